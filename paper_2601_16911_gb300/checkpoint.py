"""Checkpoint and resume of a run: the state is the coefficient (or nodal) array and the
time reached, so a checkpoint is those, the mesh description that gives them meaning, and
the step count.

A checkpoint file is an ``.npz`` holding
  * ``format``: the format tag ``cvweno-checkpoint-1``;
  * ``desc``: the problem description (the dict that ``cvweno.make_desc`` reads), as JSON;
  * ``u``: the state, float32, in the mesh's layout ``[nvar][ncell][ndof]`` (DG) or
    ``[nvar][nnode]`` (CG), exactly as the device held it;
  * ``t``, ``step``: the time reached and the number of steps taken;
  * ``crc32``: the CRC-32 of the state's bytes, checked on load.

``save`` copies the device state to the host (a synchronous device-to-host copy) and
writes the file through a temporary name, so an interrupted save leaves the previous
checkpoint in place.  ``load`` returns the description and a host array; ``resume``
makes the mesh and puts the state back on the device.  Resuming reproduces the
uninterrupted run bit for bit: the state is stored exactly and the step is a pure
function of the state and dt.
"""
from __future__ import annotations

import json
import os
import zlib

import numpy as np

FORMAT = "cvweno-checkpoint-1"


class CheckpointError(RuntimeError):
    pass


def save(path: str, desc: dict, u, t: float, step: int = 0) -> None:
    """Write the state ``u`` (a torch tensor on any device, or an array) at time ``t``."""
    arr = u.detach().to("cpu").numpy() if hasattr(u, "detach") else np.asarray(u)
    if arr.dtype != np.float32:
        raise CheckpointError(f"state must be float32, got {arr.dtype}")
    arr = np.ascontiguousarray(arr)
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, format=np.array(FORMAT), desc=np.array(json.dumps(desc, sort_keys=True)), u=arr,
                 t=np.array(float(t)), step=np.array(int(step)),
                 crc32=np.array(zlib.crc32(arr.tobytes()) & 0xFFFFFFFF, dtype=np.uint32))
    os.replace(tmp, path)


def load(path: str):
    """(desc, u as a float32 host array, t, step); raises CheckpointError on a file of
    another format or a state whose checksum does not match."""
    with np.load(path, allow_pickle=False) as z:
        if "format" not in z.files or str(z["format"]) != FORMAT:
            raise CheckpointError(f"{path}: not a {FORMAT} file")
        u = z["u"]
        if (zlib.crc32(u.tobytes()) & 0xFFFFFFFF) != int(z["crc32"]):
            raise CheckpointError(f"{path}: state checksum mismatch")
        desc = json.loads(str(z["desc"]))
        desc["bc"] = tuple(desc["bc"])
        return desc, u, float(z["t"]), int(z["step"])


def resume(path: str, device: str = "cuda"):
    """(mesh, state on the device, t, step) from a checkpoint."""
    import torch

    from . import cvweno as cv

    desc, u, t, step = load(path)
    mesh = cv.Mesh(desc)
    if tuple(u.shape) != tuple(mesh.state_shape):
        mesh.close()
        raise CheckpointError(f"{path}: state shape {u.shape} does not match the mesh's {mesh.state_shape}")
    return mesh, torch.from_numpy(u).to(device), t, step

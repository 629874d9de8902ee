"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on the
same FP32-rounded input and compare what the method makes unique."""
import numpy as np
import torch

from oracle import oracle as O
from paper_2601_16911_gb300 import cvweno as cv

# The stated bar for every floating-point stage output is 1e-5 (the FP32 path against the
# FP64 oracle on the same FP32-rounded input):
RES_TOL = 1e-5    # per-stage residual: max |r_gpu - r_oracle| / max |r_oracle|
# Per-cell sensor gamma_e in [0, 1], absolute: 1e-5 is about 170 FP32 ulps at 1.  The FP32
# sensor is a few hundred FMAs deep (Taylor data, vertex and cell Jiang-Shu weights,
# Gram-form semi-norms); over every parity case of both kernel forms, the largest
# difference measured on a GB300 was 2.6e-7.
GAMMA_TOL = 1e-5
# SC weights alpha_q (eq. alphaq), relative to the cell's largest, on cells that both
# sides mark troubled: the same bar; the largest measured was 3.4e-7.
ALPHA_TOL = 1e-5


def to_gpu(u):
    return torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()


def rounded(u64):
    """The FP32 input both sides see (the oracle reads it back in FP64)."""
    return np.ascontiguousarray(u64, dtype=np.float32).astype(np.float64)


def nonflat_mask(u, rel=1e-6):
    """Cells whose non-mean modes are not at rounding level (gamma of a flat cell is
    the ratio of two rounding errors and is not unique)."""
    nm = np.abs(u[0, :, 1:]).max(axis=1)
    return nm > rel * max(nm.max(), 1e-300)


def borderline_override(d, gamma_ref, troubled_ref, width=1e-4):
    """Cells whose oracle gamma sits within `width` of C_gamma: the SC decision is
    taken by rounding; force the GPU to the oracle's decision there."""
    ov = np.full(gamma_ref.shape, -1, np.int32)
    near = np.abs(gamma_ref - d["c_gamma"]) < width
    ov[near] = troubled_ref[near]
    return ov, int(near.sum())


def residual_pair(d, u64, mesh=None):
    """Oracle and GPU full-stage outputs on the same FP32 input."""
    u = rounded(u64)
    ref = O.residual(d, u)
    own = mesh is None
    mesh = mesh or cv.Mesh(d)
    ov, nflip = borderline_override(d, ref["gamma"], ref["troubled"])
    out = mesh.residual_ex(to_gpu(u), troubled_override=torch.from_numpy(ov).cuda())
    torch.cuda.synchronize()
    mesh.status_check()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    if own:
        mesh.close()
    return u, ref, got, nflip


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

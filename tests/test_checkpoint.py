"""Checkpoint files (paper_2601_16911_gb300.checkpoint): the state round-trips exactly,
with its description, time and step; a corrupted state or a file of another format is
refused; an interrupted save leaves the previous checkpoint in place."""
import os

import numpy as np
import pytest

from paper_2601_16911_gb300 import checkpoint as ck
from paper_2601_16911_gb300 import inputs as I


def state(seed=0, shape=(1, 20, 9)):
    return np.random.default_rng(seed).standard_normal(shape).astype(np.float32)


def test_round_trip_is_exact(tmp_path):
    d, _ = I.kpp(3, n=5, degree=2)
    u = state()
    p = str(tmp_path / "run.npz")
    ck.save(p, d, u, t=0.125, step=7)
    d2, u2, t, step = ck.load(p)
    assert d2 == d
    assert u2.dtype == np.float32 and np.array_equal(u2.view(np.uint32), u.view(np.uint32))
    assert t == 0.125 and step == 7


def test_torch_tensor_is_accepted(tmp_path):
    torch = pytest.importorskip("torch")
    d, _ = I.burgers1d_step(1, nx=8, degree=1)
    u = torch.from_numpy(state(1, (1, 8, 2)))
    p = str(tmp_path / "run.npz")
    ck.save(p, d, u, t=0.5)
    assert np.array_equal(ck.load(p)[1], u.numpy())


def test_corrupted_state_is_refused(tmp_path):
    d, _ = I.kpp(3, n=5, degree=2)
    p = str(tmp_path / "run.npz")
    ck.save(p, d, state(), t=1.0)
    with np.load(p) as z:
        fields = {k: z[k] for k in z.files}
    fields["u"] = fields["u"].copy()
    fields["u"].flat[3] += 1.0
    np.savez(p, **fields)
    with pytest.raises(ck.CheckpointError, match="checksum"):
        ck.load(p)


def test_other_files_are_refused(tmp_path):
    p = str(tmp_path / "other.npz")
    np.savez(p, u=state())
    with pytest.raises(ck.CheckpointError, match="not a"):
        ck.load(p)


def test_non_float32_state_is_refused(tmp_path):
    d, _ = I.kpp(3, n=5, degree=2)
    with pytest.raises(ck.CheckpointError):
        ck.save(str(tmp_path / "x.npz"), d, state().astype(np.float64), t=0.0)


def test_save_replaces_atomically(tmp_path):
    d, _ = I.kpp(3, n=5, degree=2)
    p = str(tmp_path / "run.npz")
    ck.save(p, d, state(0), t=1.0, step=1)
    ck.save(p, d, state(1), t=2.0, step=2)
    assert not os.path.exists(p + ".tmp")
    assert ck.load(p)[3] == 2

"""Host-side bookkeeping of bench.py (no GPU): the launch counts it reports, the table of
dominant kernels, and the algorithmic FMA counts behind the roofline figures."""
import pytest

import bench
from paper_2601_16911_gb300 import inputs as I


def test_launches_per_rk_step():
    # a 1D DG mesh of one tile (at most 128 cells) runs the whole step in one launch
    assert bench.launches_per_rk_step(dict(dim=1, nx=128, kind=I.DG)) == 1
    assert bench.launches_per_rk_step(dict(dim=1, nx=129, kind=I.DG)) == 3
    assert bench.launches_per_rk_step(dict(dim=2, nx=256, kind=I.DG)) == 3
    # CG: cells + node phase per stage in 2D; cells, node right-hand side, two sweeps in 1D
    assert bench.launches_per_rk_step(dict(dim=2, nx=256, kind=I.CG)) == 6
    assert bench.launches_per_rk_step(dict(dim=1, nx=128, kind=I.CG)) == 12


@pytest.mark.parametrize("workload", sorted(bench.DOMINANT))
def test_dominant_kernel_table_matches_the_workload(workload):
    label, kernel, pos, per_stage, stages = bench.DOMINANT[workload]
    probs = {lab: d for lab, d, _, _ in bench.problems(workload, 16 if workload != "burgers1d" else None)}
    assert label in probs
    assert stages in (1, 3) and 0 <= pos < per_stage
    if stages == 3:
        # one launch per step: the variant must be a one-tile 1D DG mesh
        assert bench.launches_per_rk_step(probs[label]) == 1
    else:
        assert bench.launches_per_rk_step(probs[label]) == 3 * per_stage


def test_method_count_is_the_per_stage_formula():
    # stages (a)-(e) of 2D scalar DG Q_p, n = p + 1, troubled fraction tf:
    # (8n^3 + 4n^2) + 4n^2 + (8n^3 + 6n^4) + tf 2n^5 + 14n^3 + 20n^2; Q3 at tf = 0.0701 is
    # 4047.6 FMA per cell
    assert bench.fma_per_cell(3, 0.0701) == pytest.approx(4047.5648)
    for p in (1, 2, 4):
        n = p + 1
        assert bench.fma_per_cell(p, 0.0) == 8 * n**3 + 8 * n**2 + 8 * n**3 + 6 * n**4 + 14 * n**3 + 20 * n**2


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cg_halo_recomputation_is_reported_apart(p):
    # the CG cell kernel's roofline uses the method's count; its halo recomputation (the
    # nodal -> modal map and the ring integrals of the 52 halo cells of a 128-cell tile)
    # is implementation work reported beside it
    n = p + 1
    assert bench.fma_per_cell_cg_halo(p) == pytest.approx(52 / 128 * (2 * n**3 + 4 * n**2))
    assert bench.fma_face_terms(p) == 20 * n**2


def test_every_traffic_key_names_its_sources():
    for key in bench.KERNEL_SOURCES:
        assert len(bench.kernel_source_sha(key)) == 16

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


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cg_cell_count_drops_exactly_the_face_part(p):
    # the CG cell kernel's count is the DG count of stages (a)-(e) without the face part of
    # (e), plus its own nodal work, which does not depend on the troubled fraction
    n = p + 1
    for tf in (0.0, 0.3):
        extra = bench.fma_per_cell_cg_cells(p, tf) - (bench.fma_per_cell(p, tf) - bench.fma_face_terms(p))
        assert extra == pytest.approx(180 / 128 * 2 * n**3 + 4 * n**3 + 52 / 128 * 4 * n**2 + 4 * n**3 + 8 * n**2)
    assert bench.fma_face_terms(p) == 20 * n**2


def test_every_traffic_key_names_its_sources():
    for key in bench.KERNEL_SOURCES:
        assert len(bench.kernel_source_sha(key)) == 16

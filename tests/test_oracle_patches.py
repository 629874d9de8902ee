"""Brute-force pins of the oracle's geometric vertex patches (Sec. 3.2: the patch
E(x_i) is the set of cells containing the vertex x_i) against an index-arithmetic
enumeration written here, on tiny meshes with periodic and transmissive sides."""
import itertools

import pytest

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I


def brute_patches_2d(nx, ny, perx, pery):
    vx = nx if perx else nx + 1
    vy = ny if pery else ny + 1
    out = {}
    for J in range(vy):
        for Iv in range(vx):
            s = set()
            # (di, dj) offset of the cell relative to the vertex; the corner of that
            # cell touching the vertex is (1 - di', 1 - dj') in (cx, cy)
            for di, dj in itertools.product((-1, 0), (-1, 0)):
                i, j = Iv + di, J + dj
                if perx:
                    i %= nx
                if pery:
                    j %= ny
                if 0 <= i < nx and 0 <= j < ny:
                    cx, cy = (1 if di == -1 else 0), (1 if dj == -1 else 0)
                    s.add((i + nx * j, cx + 2 * cy))
            out[Iv + vx * J] = s
    return out


def brute_patches_1d(nx, per):
    vx = nx if per else nx + 1
    out = {}
    for Iv in range(vx):
        s = set()
        for di in (-1, 0):
            i = Iv + di
            if per:
                i %= nx
            if 0 <= i < nx:
                s.add((i, 1 if di == -1 else 0))
        out[Iv] = s
    return out


def oracle_sets(d):
    cnt, cell, cor, cv = O.vertex_patches(d)
    sets = {}
    for v in range(len(cnt)):
        sets[v] = {(int(cell[v, s]), int(cor[v, s])) for s in range(cnt[v])}
    return sets, cv


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 3), (2, 5), (5, 2)])
@pytest.mark.parametrize("perx,pery", [(True, True), (False, False), (True, False), (False, True)])
def test_patches_2d(nx, ny, perx, pery):
    bc = (I.PERIODIC if perx else I.TRANSMISSIVE,) * 2 + (I.PERIODIC if pery else I.TRANSMISSIVE,) * 2
    d = I.mesh(2, nx, ny, degree=1, bc=bc)
    sets, cv = oracle_sets(d)
    ref = brute_patches_2d(nx, ny, perx, pery)
    assert sets == ref
    # every cell corner points at a vertex whose patch contains that (cell, corner)
    for e in range(nx * ny):
        for c in range(4):
            assert (e, c) in sets[int(cv[e, c])]
    sizes = sorted(len(s) for s in sets.values())
    if perx and pery:
        assert sizes == [4] * (nx * ny)
    if not perx and not pery:
        assert sizes.count(1) == 4  # domain corners


@pytest.mark.parametrize("nx", [3, 4, 7])
@pytest.mark.parametrize("per", [True, False])
def test_patches_1d(nx, per):
    d = I.mesh(1, nx, degree=2, bc=I.PERIODIC if per else I.TRANSMISSIVE)
    sets, cv = oracle_sets(d)
    assert sets == brute_patches_1d(nx, per)

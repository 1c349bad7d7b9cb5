"""Host logic of the benchmark's measurement (CPU only): the candidate count
from a cell histogram against a direct count over particles and stencil
cells, the merge of x sub-cells back to width-r cells, and the counting
sort's algorithmic bytes."""
import itertools

import numpy as np
import pytest

import bench


def _direct_candidates(cell_of, ncell, periodic, reach):
    """sum over particles of the particles in the distinct stencil cells."""
    dim = len(ncell)
    counts = {}
    for c in map(tuple, cell_of):
        counts[c] = counts.get(c, 0) + 1
    total = 0
    for c in map(tuple, cell_of):
        seen = set()
        for off in itertools.product(*[range(-reach[k], reach[k] + 1) for k in range(dim)]):
            t = []
            ok = True
            for k in range(dim):
                v = c[k] + off[k]
                if periodic[k]:
                    v %= ncell[k]
                elif v < 0 or v >= ncell[k]:
                    ok = False
                    break
                t.append(v)
            if ok:
                seen.add(tuple(t))
        total += sum(counts.get(t, 0) for t in seen)
    return total


@pytest.mark.parametrize("dim,ncell,periodic,reach", [
    (2, (7, 5), (1, 0), (1, 1)),
    (3, (6, 4, 5), (1, 1, 0), (1, 1, 1)),
    (3, (12, 4, 5), (1, 1, 1), (2, 1, 1)),
    (2, (2, 6), (1, 1), (1, 1)),        # periodic axis with 2 cells: no double count
])
def test_candidates_from_cells_matches_direct_count(dim, ncell, periodic, reach):
    rng = np.random.default_rng(dim + sum(ncell))
    n = 300
    cell_of = np.stack([rng.integers(0, ncell[k], n) for k in range(dim)], 1)
    # row-major with x fastest, as the library's table
    flat = cell_of[:, 0].copy()
    stride = 1
    for k in range(1, dim):
        stride *= ncell[k - 1]
        flat = flat + stride * cell_of[:, k]
    cnt = np.bincount(flat, minlength=int(np.prod(ncell)))
    start = np.concatenate([[0], np.cumsum(cnt)]).astype(np.uint32)
    got = bench.candidates_from_cells(start, ncell if dim == 3 else (ncell[0], ncell[1]),
                                      periodic, dim, reach)
    assert got == _direct_candidates(cell_of, ncell, periodic, reach)


def test_base_candidates_merges_x_subcells():
    """Splitting every width-r cell into kx parts along x and merging them
    back gives the same count as building the width-r histogram directly."""
    rng = np.random.default_rng(3)
    base = (5, 4, 6)
    kx = 3
    n = 500
    cx = rng.integers(0, base[0] * kx, n)
    cy = rng.integers(0, base[1], n)
    cz = rng.integers(0, base[2], n)
    fine = (base[0] * kx, base[1], base[2])
    flat = cx + fine[0] * (cy + fine[1] * cz)
    cnt = np.bincount(flat, minlength=int(np.prod(fine)))
    start = np.concatenate([[0], np.cumsum(cnt)]).astype(np.uint32)
    got = bench.base_candidates(start, fine, (1, 1, 1), 3, (kx, 1, 1))
    cell_of = np.stack([cx // kx, cy, cz], 1)
    assert got == _direct_candidates(cell_of, base, (1, 1, 1), (1, 1, 1))


def test_build_bytes_counting_sort():
    # 60 bytes a particle and 8 a width-r cell (plus the end entry)
    assert bench.build_bytes(1000, 99) == 60 * 1000 + 8 * 100

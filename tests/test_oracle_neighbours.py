"""Pins of the oracle's neighbour search (CPU only).

The neighbour relation is the paper's radius-filtered sum over the shortest
separation vector (Sec. 3, Eq. 1 and the velocity-update listing); the pins
below come from outside the oracle: scipy's periodic k-d tree, exact lattice
shell counts, hand-worked minimum-image cases and the uniform-density mean.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _pairs(offsets, idx, queries=None):
    n = len(offsets) - 1
    rows = np.repeat(np.arange(n) if queries is None else queries,
                     np.diff(offsets))
    return set(zip(rows.tolist(), idx.tolist()))


@pytest.mark.parametrize("dim,periodic,n,r", [
    (2, (1, 1), 3000, 0.03), (3, (1, 1, 1), 3000, 0.08),
    (2, (1, 0), 2000, 0.05), (3, (0, 1, 0), 2500, 0.1),
    (2, (0, 0), 1500, 0.07)])
def test_brute_matches_scipy_kdtree(dim, periodic, n, r):
    """Brute force vs scipy.spatial.cKDTree (FP64 distances).

    The two may only disagree on pairs whose FP64 distance is within a few
    FP32 ulps of r (the paper's predicate is evaluated in FP32 here)."""
    scipy_spatial = pytest.importorskip("scipy.spatial")
    pos = synth.uniform_positions(n, dim, 11 + dim + n)
    box = oracle.Box(dim, periodic, radius=r)
    off, idx = oracle.neighbours_brute(box, pos)
    mine = _pairs(off, idx)
    x = pos[:, :dim].astype(np.float64)
    if all(periodic):
        tree = scipy_spatial.cKDTree(x, boxsize=1.0)
        ref = tree.query_pairs(r, output_type="ndarray")
    elif not any(periodic):
        tree = scipy_spatial.cKDTree(x)
        ref = tree.query_pairs(r, output_type="ndarray")
    else:
        # mixed: replicate the periodic axes' images and search once
        shifts = [np.array([s if periodic[k] else 0 for k, s in enumerate(v)])
                  for v in np.array(np.meshgrid(*[[-1, 0, 1]] * dim)).T.reshape(-1, dim)]
        shifts = np.unique(np.array(shifts), axis=0)
        tree = scipy_spatial.cKDTree(x)
        ref = []
        for sh in shifts:
            other = scipy_spatial.cKDTree(x + sh)
            for i, js in enumerate(tree.query_ball_tree(other, r)):
                ref.extend((i, j) for j in js if j != i)
        ref = np.array(ref)
    refset = set()
    for i, j in ref.tolist():
        refset.add((i, j))
        refset.add((j, i))

    def dist(i, j):
        d = x[j] - x[i]
        for k in range(dim):
            if periodic[k]:
                d[k] -= round(d[k])
        return math.sqrt(float((d * d).sum()))

    for (i, j) in mine ^ refset:
        assert abs(dist(i, j) - r) <= 4e-7 * r + 1e-7, (i, j, dist(i, j))
    assert len(mine ^ refset) <= 2


@pytest.mark.parametrize("dim,ratio,expect", [
    (2, 1.1, 4), (2, 1.5, 8), (3, 1.1, 6), (3, 1.5, 18), (3, 1.8, 26)])
@pytest.mark.parametrize("search", ["brute", "cells"])
def test_lattice_shell_counts(dim, ratio, expect, search):
    """Square / cubic lattice with spacing a=1/16 (exact in FP32), periodic:
    shells at a, a*sqrt(2), a*sqrt(3) give 4/8 (2-D), 6/18/26 (3-D)."""
    m = 16
    g = np.stack(np.meshgrid(*[np.arange(m)] * dim, indexing="ij"), -1).reshape(-1, dim)
    pos = synth.pack4((g / m).astype(np.float32))
    box = oracle.Box(dim, (1,) * dim, radius=ratio / m)
    if search == "brute":
        off, _ = oracle.neighbours_brute(box, pos)
    else:
        off, _ = oracle.CellList(box, pos).neighbours()
    assert np.all(np.diff(off) == expect)


def test_minimum_image_closed_cases():
    """x=0.01 and x=0.99 are 0.02 apart through the periodic face only."""
    pos = synth.pack4(np.array([[0.01, 0.5], [0.99, 0.5]], np.float32))
    for periodic, expect in [((1, 1), 1), ((0, 1), 0), ((0, 0), 0), ((1, 0), 1)]:
        box = oracle.Box(2, periodic, radius=0.03)
        off, idx = oracle.neighbours_brute(box, pos)
        assert list(np.diff(off)) == [expect, expect]
        off2, idx2 = oracle.CellList(box, pos).neighbours()
        assert np.array_equal(off, off2) and np.array_equal(idx, idx2)
    # separation exactly 0.03 is excluded (strict <), 0.029 included
    pos = synth.pack4(np.array([[0.25, 0.5], [0.28125, 0.5], [0.75, 0.5]], np.float32))
    box = oracle.Box(2, (1, 1), radius=0.03125)
    off, _ = oracle.neighbours_brute(box, pos)
    assert list(np.diff(off)) == [0, 0, 0]
    box = oracle.Box(2, (1, 1), radius=0.032)
    off, _ = oracle.neighbours_brute(box, pos)
    assert list(np.diff(off)) == [1, 1, 0]


def test_half_box_tie_is_symmetric():
    """A separation of exactly L/2 is not wrapped from either side, so the
    relation stays symmetric (reading of 'shortest vector', Sec. 3)."""
    pos = synth.pack4(np.array([[0.0, 0.0], [0.5, 0.0], [0.25, 0.0]], np.float32))
    box = oracle.Box(2, (1, 1), radius=0.75)
    off, idx = oracle.neighbours_brute(box, pos)
    s = _pairs(off, idx)
    assert all((j, i) in s for (i, j) in s)


@pytest.mark.parametrize("dim,periodic,n,r", [
    (2, (1, 1), 4000, 0.03), (3, (1, 1, 1), 4000, 0.09),
    (2, (1, 0), 3000, 0.2), (3, (1, 0, 1), 3000, 0.3),     # n_k = 4, 3
    (2, (1, 1), 2000, 0.45), (3, (1, 1, 1), 1500, 0.6),    # n_k = 2, 1
    (2, (0, 0), 2000, 0.3), (3, (0, 1, 1), 2000, 0.21)])
def test_cell_list_equals_brute_force(dim, periodic, n, r):
    pos = synth.uniform_positions(n, dim, 100 + n + dim)
    box = oracle.Box(dim, periodic, radius=r)
    a = oracle.neighbours_brute(box, pos)
    b = oracle.CellList(box, pos).neighbours()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_cell_boundary_ulps():
    """Particles one ulp either side of cell boundaries and of the periodic
    face; both searches must agree exactly."""
    r = 0.1
    rng = np.random.default_rng(5)
    base = np.array([0.0, 0.1, 0.2, 0.3, 0.5, 0.9, 1.0], np.float32)
    xs = np.concatenate([np.nextafter(base, np.float32(-1)), base,
                         np.nextafter(base, np.float32(2))]).astype(np.float32)
    xs = xs[(xs >= 0) & (xs < 1)]
    g = np.stack(np.meshgrid(xs, xs, indexing="ij"), -1).reshape(-1, 2)
    g = np.concatenate([g, rng.random((500, 2)).astype(np.float32)])
    pos = synth.pack4(g.astype(np.float32))
    for periodic in [(1, 1), (0, 1), (0, 0)]:
        for rr in [r, np.nextafter(np.float32(r), np.float32(1)), 0.0999999]:
            box = oracle.Box(2, periodic, radius=float(rr))
            a = oracle.neighbours_brute(box, pos)
            b = oracle.CellList(box, pos).neighbours()
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_symmetry_and_uniform_mean():
    """j in N(i) <=> i in N(j); mean count ~ (N-1) pi r^2 for uniform data."""
    w = synth.c1()
    box = oracle.Box(2, (1, 1), radius=w.radius)
    off, idx = oracle.neighbours_brute(box, w.pos)
    s = _pairs(off, idx)
    assert all((j, i) in s for (i, j) in s)
    assert int(off[-1]) % 2 == 0
    mean = off[-1] / w.n
    expect = (w.n - 1) * math.pi * w.radius ** 2
    # Poisson-ish: sd of the mean ~ sqrt(2*expect/N)
    assert abs(mean - expect) < 6 * math.sqrt(2 * expect / w.n)


def test_3d_uniform_mean_count():
    n = 1 << 16
    pos = synth.uniform_positions(n, 3, 77)
    r = 0.05
    box = oracle.Box(3, (1, 1, 1), radius=r)
    c = oracle.CellList(box, pos).counts()
    expect = (n - 1) * 4.0 / 3.0 * math.pi * r ** 3
    assert abs(c.mean() - expect) < 6 * math.sqrt(2 * expect / n)


def test_query_subset_matches_full():
    pos = synth.uniform_positions(5000, 3, 9)
    box = oracle.Box(3, (1, 1, 1), radius=0.07)
    q = synth.query_sample(5000, 700, 3)
    off_all, idx_all = oracle.neighbours_brute(box, pos)
    off_q, idx_q = oracle.CellList(box, pos).neighbours(q)
    for t, i in enumerate(q):
        assert np.array_equal(idx_all[off_all[i]:off_all[i + 1]],
                              idx_q[off_q[t]:off_q[t + 1]])

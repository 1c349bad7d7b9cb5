"""GPU cell list + neighbour set vs the oracle: bit-exact (GPU, C ABI).

The neighbour relation (paper Sec. 2.2.2 box search, Sec. 3 Eq. 1 predicate
over the shortest separation) must equal the oracle's set exactly.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import dev, gpu_csr_rows, host, oracle_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ab():
    import paper_1704_08907_gb300 as ab
    return ab


@pytest.fixture(scope="module")
def ctx(ab, cuda):
    c = ab.Context(0)
    yield c
    c.close()


def _compare_all(ab, ctx, dim, periodic, pos, r, lo=(0, 0, 0), hi=(1, 1, 1)):
    dom = ab.Domain(dim, periodic, r, lo, hi)
    ab.ab_build(ctx, dom, dev(pos))
    off, idx = ab.ab_pair_list(ctx)
    box = oracle.Box(dim, periodic, lo, hi, r)
    ooff, oidx = oracle.neighbours_brute(box, pos)
    off_h = host(off)
    assert np.array_equal(off_h, ooff)
    idx_h = host(idx)
    for i in range(pos.shape[0]):
        assert np.array_equal(np.sort(idx_h[off_h[i]:off_h[i + 1]]), oidx[ooff[i]:ooff[i + 1]]), i
    ab.ab_sync(ctx)
    return off_h


def test_c1_full_neighbour_set(ab, ctx):
    w = synth.c1()
    off = _compare_all(ab, ctx, 2, w.periodic, w.pos, w.radius)
    assert abs(off[-1] / w.n - (w.n - 1) * math.pi * w.radius ** 2) < 0.5


@pytest.mark.parametrize("dim,periodic,n,r", [
    (2, (1, 1), 3000, 0.03), (3, (1, 1, 1), 4000, 0.09),
    (2, (1, 0), 3000, 0.2), (3, (1, 0, 1), 3000, 0.3),     # n_k = 4, 3 (general path)
    (2, (1, 1), 2000, 0.45), (3, (1, 1, 1), 1500, 0.6),    # n_k = 2, 1
    (2, (0, 0), 2000, 0.3), (3, (0, 1, 1), 2000, 0.21),    # aperiodic, n_k = 4
    (3, (1, 1, 1), 3000, 0.19), (2, (1, 1), 3000, 0.166),  # n_k = 5, 6 (fast path edge)
    (2, (0, 1), 5000, 0.011), (3, (1, 1, 0), 5000, 0.05)])
def test_random_boxes(ab, ctx, dim, periodic, n, r):
    pos = synth.uniform_positions(n, dim, 1000 + n + dim)
    _compare_all(ab, ctx, dim, periodic, pos, r)


def test_non_unit_box_and_offsets(ab, ctx):
    rng = np.random.default_rng(3)
    lo, hi = (-2.0, 0.5, 10.0), (1.0, 2.0, 12.5)
    pts = np.stack([rng.uniform(lo[k], hi[k], 3000) for k in range(3)], 1).astype(np.float32)
    for k in range(3):
        pts[pts[:, k] >= np.float32(hi[k]), k] = np.float32(lo[k])
    _compare_all(ab, ctx, 3, (1, 0, 1), synth.pack4(pts), 0.23, lo, hi)


@pytest.mark.parametrize("dim,ratio,expect", [
    (2, 1.1, 4), (2, 1.5, 8), (3, 1.1, 6), (3, 1.5, 18), (3, 1.8, 26)])
def test_lattice_shells(ab, ctx, dim, ratio, expect):
    m = 16
    g = np.stack(np.meshgrid(*[np.arange(m)] * dim, indexing="ij"), -1).reshape(-1, dim)
    pos = synth.pack4((g / m).astype(np.float32))
    off = _compare_all(ab, ctx, dim, (1,) * dim, pos, ratio / m)
    assert np.all(np.diff(off) == expect)


def test_minimum_image_closed_case(ab, ctx):
    pos = synth.pack4(np.array([[0.01, 0.5], [0.99, 0.5]], np.float32))
    for periodic, expect in [((1, 1), 1), ((0, 1), 0)]:
        off = _compare_all(ab, ctx, 2, periodic, pos, 0.03)
        assert list(np.diff(off)) == [expect, expect]


def test_cell_boundary_ulps(ab, ctx):
    base = np.array([0.0, 0.1, 0.2, 0.3, 0.5, 0.9, 1.0], np.float32)
    xs = np.concatenate([np.nextafter(base, np.float32(-1)), base,
                         np.nextafter(base, np.float32(2))]).astype(np.float32)
    xs = xs[(xs >= 0) & (xs < 1)]
    g = np.stack(np.meshgrid(xs, xs, indexing="ij"), -1).reshape(-1, 2)
    rng = np.random.default_rng(5)
    g = np.concatenate([g, rng.random((500, 2)).astype(np.float32)]).astype(np.float32)
    pos = synth.pack4(g)
    for periodic in [(1, 1), (0, 1), (0, 0)]:
        for r in [0.1, float(np.nextafter(np.float32(0.1), np.float32(1))), 0.0999999]:
            _compare_all(ab, ctx, 2, periodic, pos, r)


@pytest.mark.parametrize("periodic", [(1, 1), (0, 1)])
def test_x_subcell_boundary_ulps(ab, ctx, periodic):
    """Along x the cells are split into kx parts (reach kx): particles one or
    two ulps either side of every x cell boundary, against brute force."""
    r = 0.1
    dom = ab.Domain(2, periodic, r)
    ab.ab_build(ctx, dom, dev(synth.pack4(np.array([[0.5, 0.5]], np.float32))))
    (nx, _, _), _, reach = ab.ab_cell_shape(ctx, with_reach=True)
    assert reach[0] >= 2
    b = (np.arange(nx + 1) / nx).astype(np.float32)
    xs = np.concatenate([b, np.nextafter(b, np.float32(-1)), np.nextafter(b, np.float32(2)),
                         np.nextafter(np.nextafter(b, np.float32(2)), np.float32(2))])
    xs = np.unique(xs[(xs >= 0) & (xs < 1)]).astype(np.float32)
    rng = np.random.default_rng(11)
    ys = rng.choice(np.float32([0.3, 0.3 + 1e-7, 0.35]), len(xs)).astype(np.float32)
    pos = synth.pack4(np.stack([xs, ys], 1))
    extra = rng.random((1500, 2)).astype(np.float32)
    _compare_all(ab, ctx, 2, periodic, np.concatenate([pos, synth.pack4(extra)]), r)


def test_degenerate_inputs(ab, ctx):
    # empty
    dom = ab.Domain(3, (1, 1, 1), 0.1)
    ab.ab_build(ctx, dom, torch.zeros((0, 4), dtype=torch.float32, device="cuda:0"))
    off, idx = ab.ab_pair_list(ctx)
    assert host(off).tolist() == [0] and idx.numel() == 0
    y = ab.ab_pair_sum(ctx, "count", ab.OpParams())
    assert y.numel() == 0
    # one particle, two particles, everything in one cell, coincident points
    _compare_all(ab, ctx, 3, (1, 1, 1), synth.pack4(np.array([[0.5, 0.5, 0.5]], np.float32)), 0.1)
    _compare_all(ab, ctx, 2, (1, 1), synth.pack4(np.array([[0.2, 0.2], [0.25, 0.2]], np.float32)), 0.1)
    pts = (0.5 + 0.01 * np.random.default_rng(0).random((300, 3))).astype(np.float32)
    _compare_all(ab, ctx, 3, (1, 1, 1), synth.pack4(pts), 0.2)
    pts = np.repeat(np.array([[0.3, 0.3], [0.31, 0.3]], np.float32), 5, axis=0)
    off = _compare_all(ab, ctx, 2, (1, 1), synth.pack4(pts), 0.05)
    assert np.all(np.diff(off) == 9)


def test_sort_is_stable_and_deterministic(ab, ctx):
    w = synth.c2(n=200000)
    dom = ab.Domain(3, w.periodic, w.radius)
    p = dev(w.pos)
    ab.ab_build(ctx, dom, p)
    perm1, start1 = (host(t) for t in ab.ab_cell_export(ctx))
    y1 = host(ab.ab_pair_sum(ctx, "lj", ab.OpParams(eps=1.0, sigma=0.01)))
    ab.ab_build(ctx, dom, p)
    perm2, start2 = (host(t) for t in ab.ab_cell_export(ctx))
    y2 = host(ab.ab_pair_sum(ctx, "lj", ab.OpParams(eps=1.0, sigma=0.01)))
    assert np.array_equal(perm1, perm2) and np.array_equal(start1, start2)
    assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))
    assert np.array_equal(np.sort(perm1), np.arange(w.n))
    # within every cell the original indices ascend (stable counting sort)
    starts = start1.astype(np.int64)
    assert starts[0] == 0 and starts[-1] == w.n and np.all(np.diff(starts) >= 0)
    seg = np.repeat(np.arange(len(starts) - 1), np.diff(starts))
    same = seg[1:] == seg[:-1]
    assert np.all(perm1[1:][same] > perm1[:-1][same])
    (nx, ny, nz), tot, reach = ab.ab_cell_shape(ctx, with_reach=True)
    kx, ky, kz = reach
    assert 1 <= kx <= 4 and 1 <= ky <= 2 and kz == 1
    assert (nx, ny, nz) == (50 * kx, 50 * ky, 50) and tot == 125000 * kx * ky


def test_c2_full_neighbour_set(ab, ctx):
    """1,048,576 uniform points, r = 0.0197: every row equals the oracle's."""
    w = synth.c2()
    dom = ab.Domain(3, w.periodic, w.radius)
    ab.ab_build(ctx, dom, dev(w.pos))
    off, idx = ab.ab_pair_list(ctx)
    ooff, oidx = oracle.CellList(oracle_box(w), w.pos).neighbours()
    off_h = host(off)
    assert np.array_equal(off_h, ooff)
    idx_h = host(idx).astype(np.int64)
    rows = np.repeat(np.arange(w.n, dtype=np.int64), np.diff(off_h))
    key = np.sort(rows * w.n + idx_h)
    okey = np.repeat(np.arange(w.n, dtype=np.int64), np.diff(ooff)) * w.n + oidx
    assert np.array_equal(key, okey)
    mean = off_h[-1] / w.n
    assert abs(mean - (w.n - 1) * 4 / 3 * math.pi * w.radius ** 3) < 0.1


def test_c3_full_sampled_rows(ab, ctx):
    """16.7M clustered points: sampled rows of the neighbour set are exact."""
    w = synth.c3()
    dom = ab.Domain(3, w.periodic, w.radius)
    ab.ab_build(ctx, dom, dev(w.pos))
    off, idx = ab.ab_pair_list(ctx)
    q = synth.query_sample(w.n, 4096, 77)
    off_h, rows = gpu_csr_rows(off, idx, q)
    cl = oracle.CellList(oracle_box(w), w.pos)
    ooff, oidx = cl.neighbours(q)
    for t, r in enumerate(q):
        assert np.array_equal(rows[t], oidx[ooff[t]:ooff[t + 1]]), r
    assert abs(off_h[-1] / w.n - 64.0) < 2.0
    del off, idx
    torch.cuda.empty_cache()


def test_c5_full_sampled_rows(ab, ctx):
    """4M points, x periodic / y reflecting, r = 0.002."""
    w = synth.c5()
    dom = ab.Domain(2, w.periodic, w.radius)
    ab.ab_build(ctx, dom, dev(w.pos))
    off, idx = ab.ab_pair_list(ctx)
    q = np.concatenate([synth.query_sample(w.n, 4096, 5),
                        np.where((w.pos[:, 0] < 0.002) | (w.pos[:, 1] > 0.998))[0][:2048]])
    _, rows = gpu_csr_rows(off, idx, q)
    ooff, oidx = oracle.CellList(oracle_box(w), w.pos).neighbours(q)
    for t, r in enumerate(q):
        assert np.array_equal(rows[t], oidx[ooff[t]:ooff[t + 1]]), r

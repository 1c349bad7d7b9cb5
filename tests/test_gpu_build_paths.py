"""The cell-list build paths against each other (GPU, C ABI): the counting
sort as one cooperative launch and as a kernel sequence, and the stable radix
sort of the cell ids, give the same cell list bit for bit; and the bounded
waits of the single launch and of the radix sort's look-back, made to run
out without a fault or a hang."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import dev, host, oracle_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ab():
    import paper_1704_08907_gb300 as ab
    return ab


@pytest.fixture(scope="module")
def ctx(ab, cuda):
    c = ab.Context(0)
    yield c
    ab.ab_testing_build_path(c, ab.BUILD_AUTO)
    ab.ab_testing_cell_table(c, 0)
    c.close()


def _case(name):
    if name == "c2":
        w = synth.c2()
        return 3, (1, 1, 1), w.radius, w.pos
    if name == "clustered":
        w = synth.c3(n=1 << 18, n_blobs=16)
        return 3, (1, 1, 1), w.radius, w.pos
    if name == "2d_wall":
        return 2, (1, 0), 0.002, synth.uniform_positions(300000, 2, 3)
    if name == "one_cell":
        pts = np.float32(0.25) + np.float32(1e-3) * synth.uniform_positions(3000, 3, 5)[:, :3]
        return 3, (0, 0, 0), 0.3, synth.pack4(pts.astype(np.float32))
    if name == "n1":
        return 3, (1, 1, 1), 0.1, synth.uniform_positions(1, 3, 6)
    return 2, (1, 1), 0.1, synth.uniform_positions(2, 2, 7)


def _state(ab, ctx, dim, periodic, r, pos, path, packed=False):
    ab.ab_testing_build_path(ctx, int(path))
    dom = ab.Domain(dim, periodic, r)
    p = dev(pos)
    if packed:
        p = dev(np.ascontiguousarray(pos[:, :dim]))
    ab.ab_build(ctx, dom, p)
    perm, start = ab.ab_cell_export(ctx)
    cnt = ab.ab_pair_sum(ctx, "count", ab.OpParams())
    ab.ab_sync(ctx)
    return host(perm), host(start), host(cnt)


@pytest.mark.parametrize("case", ["c2", "clustered", "2d_wall", "one_cell", "n1", "n2"])
def test_single_launch_equals_kernel_sequence(ab, ctx, case):
    dim, periodic, r, pos = _case(case)
    a = _state(ab, ctx, dim, periodic, r, pos, True)
    b = _state(ab, ctx, dim, periodic, r, pos, False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # the sorted order is a permutation and the offsets end at n
    assert np.array_equal(np.sort(a[0]), np.arange(len(pos)))
    assert a[1][-1] == len(pos) and np.all(np.diff(a[1].astype(np.int64)) >= 0)


def test_single_launch_packed_positions(ab, ctx):
    w = synth.c2(n=200000)
    a = _state(ab, ctx, 3, (1, 1, 1), 0.03, w.pos, True, packed=True)
    b = _state(ab, ctx, 3, (1, 1, 1), 0.03, w.pos, False, packed=False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_single_launch_barrier_timeout_reports_and_recovers(ab, ctx):
    """Block 0 never arrives at the first grid barrier: the other blocks'
    waits give up after 20 ms, the launch ends, ab_sync reports
    AB_ERR_TIMEOUT, and the next build is correct again."""
    ab.ab_testing_build_path(ctx, ab.BUILD_COOP)
    w = synth.c1()
    dom = ab.Domain(2, w.periodic, w.radius)
    big = synth.uniform_positions(1 << 20, 2, 9)
    ab.ab_testing_build_timeout(ctx, 0, 20_000_000)
    ab.ab_build(ctx, ab.Domain(2, (1, 1), 0.002), dev(big))
    with pytest.raises(ab.AbError) as e:
        ab.ab_sync(ctx)
    assert e.value.status == 6
    ab.ab_sync(ctx)                                 # latch cleared
    ab.ab_build(ctx, dom, dev(w.pos))
    c = host(ab.ab_pair_sum(ctx, "count", ab.OpParams()))
    off, _ = oracle.neighbours_brute(oracle_box(w), w.pos)
    assert np.array_equal(c, np.diff(off).astype(np.float32))
    ab.ab_sync(ctx)


@pytest.mark.parametrize("table", [1, 2])
@pytest.mark.parametrize("case", ["c2", "clustered", "2d_wall", "one_cell", "n1", "n2"])
def test_radix_sort_equals_counting_sort(ab, ctx, case, table):
    """The radix sort of the cell ids orders particles exactly as the
    counting sort (stable by original index inside a cell): same
    permutation, same offsets of every cell and same neighbour counts, for
    the dense table (1) and the table of occupied cells (2)."""
    dim, periodic, r, pos = _case(case)
    ab.ab_testing_cell_table(ctx, table)
    a = _state(ab, ctx, dim, periodic, r, pos, ab.BUILD_RADIX)
    b = _state(ab, ctx, dim, periodic, r, pos, ab.BUILD_COOP)
    ab.ab_testing_cell_table(ctx, 0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(np.sort(a[0]), np.arange(len(pos)))


def test_radix_sort_packed_positions_and_repeat(ab, ctx):
    """Packed xyz input gives the float4 input's cell list; a second radix
    build on the same context (the next look-back epoch) gives it again."""
    w = synth.c2(n=200000)
    a = _state(ab, ctx, 3, (1, 1, 1), 0.03, w.pos, ab.BUILD_RADIX, packed=True)
    b = _state(ab, ctx, 3, (1, 1, 1), 0.03, w.pos, ab.BUILD_RADIX, packed=False)
    c = _state(ab, ctx, 3, (1, 1, 1), 0.03, w.pos, ab.BUILD_SEQUENCE, packed=False)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_radix_sort_orders_by_cell_then_index(ab, ctx):
    """On a clustered input of three digit passes, every particle sits in the
    exported range of the cell its position hashes to (the hash recomputed
    here in FP32), and inside a cell original indices increase."""
    w = synth.c3(n=1 << 18, n_blobs=16)
    ab.ab_testing_build_path(ctx, ab.BUILD_RADIX)
    ab.ab_build(ctx, ab.Domain(3, w.periodic, w.radius), dev(w.pos))
    perm, start = ab.ab_cell_export(ctx)
    ncell, n_cells, _ = ab.ab_cell_shape(ctx, with_reach=True)
    ab.ab_sync(ctx)
    ab.ab_testing_build_path(ctx, ab.BUILD_AUTO)
    assert n_cells > 1 << 20                      # more than two 10-bit digits
    perm = host(perm).astype(np.int64)
    start = host(start).astype(np.int64)
    cells = np.repeat(np.arange(len(start) - 1), np.diff(start))
    assert len(cells) == w.n
    # unit box: inv_w = n_k in FP32, cell = floor(x * n_k) clamped
    p = w.pos[perm]
    c = np.zeros(w.n, dtype=np.int64)
    stride = 1
    for k in range(3):
        u = np.floor(p[:, k] * np.float32(ncell[k])).astype(np.int64)
        c += stride * np.clip(u, 0, ncell[k] - 1)
        stride *= int(ncell[k])
    assert np.array_equal(c, cells)
    same = cells[1:] == cells[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])


def test_radix_look_back_timeout_reports_and_recovers(ab, ctx):
    """Tile 0 of the scan of the first digit's counts never publishes its
    sum: the look-back of the scan tiles after it gives up after 20 ms, the
    build ends, ab_sync reports AB_ERR_TIMEOUT, and the next build is correct
    again."""
    ab.ab_testing_build_path(ctx, ab.BUILD_RADIX)
    w = synth.c1()
    dom = ab.Domain(2, w.periodic, w.radius)
    big = synth.uniform_positions(1 << 20, 2, 9)
    ab.ab_testing_build_timeout(ctx, 0, 20_000_000)
    ab.ab_build(ctx, ab.Domain(2, (1, 1), 0.002), dev(big))
    with pytest.raises(ab.AbError) as e:
        ab.ab_sync(ctx)
    assert e.value.status == 6
    ab.ab_sync(ctx)                                 # latch cleared
    ab.ab_build(ctx, dom, dev(w.pos))
    c = host(ab.ab_pair_sum(ctx, "count", ab.OpParams()))
    off, _ = oracle.neighbours_brute(oracle_box(w), w.pos)
    assert np.array_equal(c, np.diff(off).astype(np.float32))
    ab.ab_sync(ctx)
    ab.ab_testing_build_path(ctx, ab.BUILD_AUTO)


@pytest.mark.parametrize("case", ["c2", "clustered", "2d_wall", "one_cell", "n1", "n2"])
def test_compact_table_equals_dense_table(ab, ctx, case):
    """The table of occupied cells orders particles and finds stencil rows
    exactly as the dense table: same permutation, same offsets of every
    cell, same pair sums bit for bit."""
    dim, periodic, r, pos = _case(case)
    ab.ab_testing_build_path(ctx, ab.BUILD_AUTO)
    out = {}
    for mode in (1, 2):
        ab.ab_testing_cell_table(ctx, mode)
        dom = ab.Domain(dim, periodic, r)
        ab.ab_build(ctx, dom, dev(pos))
        perm, start = ab.ab_cell_export(ctx)
        cnt = ab.ab_pair_sum(ctx, "count", ab.OpParams())
        wt = dev(synth.weights(len(pos), 3, "normal"))
        y = ab.ab_pair_sum(ctx, "gauss", ab.OpParams(s=1.0 / (r / 3) ** 2), w=wt)
        E, G, e = ab.ab_pair_energy_grad(ctx, "lj", ab.OpParams(eps=1.0, sigma=r / 3))
        ab.ab_sync(ctx)
        out[mode] = [host(t) for t in (perm, start, cnt, y, E, G)] + [float(e)]
    ab.ab_testing_cell_table(ctx, 0)
    for a, b in zip(out[1], out[2]):
        assert np.array_equal(np.asarray(a), np.asarray(b), equal_nan=True)


def test_compact_table_is_chosen_for_clustered_points(ab, ctx):
    """Automatic choice: the clustered workload's lattice has more than 4
    cells a particle, so the compact table is used; its neighbour counts
    match the oracle on sampled rows."""
    w = synth.c3(n=1 << 18, n_blobs=16)
    ab.ab_testing_cell_table(ctx, 0)
    ab.ab_testing_build_path(ctx, ab.BUILD_AUTO)
    ab.ab_build(ctx, ab.Domain(3, w.periodic, w.radius), dev(w.pos))
    _, ncells, _ = ab.ab_cell_shape(ctx, with_reach=True)
    assert ncells > 4 * w.n
    c = host(ab.ab_pair_sum(ctx, "count", ab.OpParams()))
    q = synth.query_sample(w.n, 2048, 7)
    off, _ = oracle.CellList(oracle_box(w), w.pos).neighbours(q)
    assert np.array_equal(c[q], np.diff(off).astype(np.float32))
    ab.ab_sync(ctx)


def test_cuda_graph_replay_equals_eager(ab, ctx):
    """The build (one cooperative launch), the soft-force pair sum and the
    Brownian step captured in a CUDA graph and replayed give the eager
    results bit for bit."""
    w = synth.c5(n=1 << 18)
    p = w.params
    dom = ab.Domain(2, w.periodic, w.radius)
    prm = ab.OpParams(k=p["k"])
    ab.ab_testing_build_path(ctx, ab.BUILD_AUTO)
    ab.ab_testing_cell_table(ctx, 0)

    def run(pos, F, t0, steps):
        for t in range(t0, t0 + steps):
            ab.ab_build(ctx, dom, pos)
            ab.ab_pair_sum(ctx, "soft", prm, out=F)
            ab.ab_bd_step(ctx, dom, pos, F, p["dt"], p["D"], p["seed"], t)

    pos_e = dev(w.pos)
    F_e = torch.empty_like(pos_e)
    run(pos_e, F_e, 0, 4)
    pos_g = dev(w.pos)
    F_g = torch.empty_like(pos_g)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        with torch.cuda.graph(g, stream=cap):
            run(pos_g, F_g, 0, 4)
    torch.cuda.current_stream().wait_stream(cap)
    pos_g.copy_(dev(w.pos))
    g.replay()
    torch.cuda.synchronize()
    ab.ab_sync(ctx)
    assert torch.equal(pos_g, pos_e) and torch.equal(F_g, F_e)

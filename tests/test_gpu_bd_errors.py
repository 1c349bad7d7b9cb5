"""Brownian step parity, stale detection, argument errors and the bounded
device-side wait (GPU, C ABI)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import dev, host, oracle_box
from oracle import brownian, philox

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


def _periodic_diff(a, b, periodic, L=1.0):
    d = np.abs(a.astype(np.float64) - b.astype(np.float64))
    for k, p in enumerate(periodic):
        if p:
            d[:, k] = np.minimum(d[:, k], L - d[:, k])
    return d


def test_bd_step_full_size_one_step(ab, ctx):
    """One Euler-Maruyama step of the 4M-particle workload: the library's
    soft-force pair sum and step against the oracle's own pair sum and step.
    The positions may differ by two FP32 roundings plus dt times the pair-sum
    error bar (1e-5 of sum |t|, per particle)."""
    w = synth.c5()
    p = w.params
    dom = ab.Domain(2, w.periodic, w.radius)
    pos = dev(w.pos)
    ab.ab_build(ctx, dom, pos)
    F = ab.ab_pair_sum(ctx, "soft", ab.OpParams(k=p["k"]))
    ab.ab_bd_step(ctx, dom, pos, F, p["dt"], p["D"], p["seed"], 7)
    out = host(pos)
    box = oracle_box(w)
    off, idx = oracle.CellList(box, w.pos).neighbours()
    Fo = oracle.pair_values("soft", box, w.pos, off, idx, params={"k": p["k"]})
    den = oracle.abs_terms("soft", box, w.pos, off, idx, params={"k": p["k"]})
    ref = brownian.bd_step(w.pos, Fo, 2, w.periodic, w.lo, w.hi, p["dt"], p["D"], p["seed"], 7)
    d = _periodic_diff(out[:, :2], ref[:, :2], w.periodic)
    tol = 4e-7 + p["dt"] * 1e-5 * np.maximum(np.abs(Fo[:, :2]), den[:, :2])
    assert np.all(d <= tol)
    assert np.all(out[:, :2] >= 0) and np.all(out[:, 0] < 1) and np.all(out[:, 1] <= 1)


def test_bd_noise_words_match_philox(ab, ctx):
    """With dt = 0 the step is x + sqrt(2D dt) z = x: use dt tiny and D large
    to read z back and compare with the oracle's Philox/Box-Muller normals."""
    n = 100000
    pos0 = np.zeros((n, 4), np.float32)
    pos0[:, :3] = 0.5
    dom = ab.Domain(3, (0, 0, 0), 0.1, (-1e6, -1e6, -1e6), (1e6, 1e6, 1e6))
    pos = dev(pos0)
    dt, D = 1.0, 0.5          # sqrt(2 D dt) = 1
    ab.ab_bd_step(ctx, dom, pos, None, dt, D, 1704094, 3)
    z = host(pos)[:, :3].astype(np.float64) - 0.5
    ref = philox.particle_normals(np.arange(n), 3, 1704094)
    assert np.max(np.abs(z - ref)) <= 2e-6 * np.maximum(1.0, np.abs(ref)).max()


def test_stale_after_move(ab, ctx):
    w = synth.c1()
    dom = ab.Domain(2, w.periodic, w.radius)
    pos = dev(w.pos)
    ab.ab_build(ctx, dom, pos)
    ab.ab_bd_step(ctx, dom, pos, None, 1e-5, 1e-2, 1, 0)
    with pytest.raises(ab.AbError) as e:
        ab.ab_pair_sum(ctx, "count", ab.OpParams())
    assert e.value.status == 3
    ab.ab_build(ctx, dom, pos)
    ab.ab_pair_sum(ctx, "count", ab.OpParams())


def test_argument_errors(ab, ctx):
    w = synth.c1()
    pos = dev(w.pos)
    for bad in [ab.Domain(4, (1, 1), 0.1), ab.Domain(2, (1, 1), 0.0),
                ab.Domain(2, (1, 1), float("nan")), ab.Domain(2, (1, 1), 0.1, (0, 0), (0, 1))]:
        with pytest.raises(ab.AbError) as e:
            ab.ab_build(ctx, bad, pos)
        assert e.value.status == 1
    dom = ab.Domain(2, w.periodic, w.radius)
    ab.ab_build(ctx, dom, pos)
    with pytest.raises(ab.AbError) as e:          # GAUSS without weights
        ab.ab_pair_sum(ctx, "gauss", ab.OpParams(s=1.0))
    assert e.value.status == 1
    wt = dev(w.w)
    with pytest.raises(ab.AbError) as e:          # output aliases the weights
        ab.ab_pair_sum(ctx, "gauss", ab.OpParams(s=1.0), w=wt, out=wt)
    assert e.value.status == 2
    g = dev(synth.weights(w.n, 2))
    gpos = torch.empty((w.n, 4), dtype=torch.float32, device="cuda:0")
    with pytest.raises(ab.AbError) as e:          # gradient output aliases grad_out
        ab.ab_pair_sum_bwd(ctx, "gauss", ab.OpParams(s=1.0), wt, g, gpos, g)
    assert e.value.status == 2
    # the sorted copy is the library's: overwriting the caller's positions
    # after the build is allowed and does not change the result
    c0 = host(ab.ab_pair_sum(ctx, "count", ab.OpParams()))
    f = ab.ab_pair_sum(ctx, "expf", ab.OpParams(c=1.0), out=pos)
    c1 = host(ab.ab_pair_sum(ctx, "count", ab.OpParams()))
    assert np.array_equal(c0, c1) and f.data_ptr() == pos.data_ptr()
    with pytest.raises(ab.AbError) as e:          # no adjoint for EXPF
        ab.ab_pair_sum_bwd(ctx, "expf", ab.OpParams(), None, wt)
    assert e.value.status == 7
    with pytest.raises(ab.AbError) as e:          # capacity
        ab.ab_pair_list(ctx, cap=10)
    assert e.value.status == 8
    ab.ab_sync(ctx)


def test_scan_wait_times_out_without_hanging(ab, ctx):
    """A tile that never publishes: the successor's wait gives up after the
    limit, the kernel finishes, ab_sync reports AB_ERR_TIMEOUT, and the
    context keeps working."""
    ab.ab_testing_scan_timeout(ctx, 5 * 4096, 2, 20_000_000)
    with pytest.raises(ab.AbError) as e:
        ab.ab_sync(ctx)
    assert e.value.status == 6
    ab.ab_sync(ctx)                               # latch cleared
    w = synth.c1()
    ab.ab_build(ctx, ab.Domain(2, w.periodic, w.radius), dev(w.pos))
    c = host(ab.ab_pair_sum(ctx, "count", ab.OpParams()))
    box = oracle_box(w)
    off, _ = oracle.neighbours_brute(box, w.pos)
    assert np.array_equal(c, np.diff(off).astype(np.float32))


def test_bd_time_loop_statistics(ab, ctx):
    """1000 steps of the Brownian loop (rebuild + soft force + step, every
    step) on 4M points in the dilute limit (r = 2e-5, so almost no pair
    interacts): per-axis mean squared displacement 2 D t within 1%, every x
    in [0, 1) and every y in [0, 1] (periodic x, reflecting y)."""
    w = synth.c5()
    p = w.params
    r = 2e-5
    dom = ab.Domain(2, w.periodic, r)
    prm = ab.OpParams(k=p["k"])
    pos0 = w.pos.copy()
    pos0[:, 1] = np.float32(0.25) + np.float32(0.5) * pos0[:, 1]   # away from the walls
    pos = dev(pos0)
    F = torch.empty_like(pos)
    steps = 1000
    for t in range(steps):
        ab.ab_build(ctx, dom, pos)
        ab.ab_pair_sum(ctx, "soft", prm, out=F)
        ab.ab_bd_step(ctx, dom, pos, F, p["dt"], p["D"], p["seed"], t)
    ab.ab_sync(ctx)
    out = host(pos)
    assert np.all(out[:, 0] >= 0) and np.all(out[:, 0] < 1)
    assert np.all(out[:, 1] >= 0) and np.all(out[:, 1] <= 1)
    d = out[:, :2].astype(np.float64) - pos0[:, :2].astype(np.float64)
    d[:, 0] -= np.round(d[:, 0])                       # minimum image along periodic x
    msd = (d * d).mean(0)
    expect = 2 * p["D"] * p["dt"] * steps
    assert np.all(np.abs(msd / expect - 1) < 0.01), msd / expect

"""The paper's molecular-dynamics step (Sec. 3, Eqs. 1-3) through the C ABI:
EXPF pair sum + semi-implicit Euler update, against the oracle (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import dev, host
from oracle import md

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


def _pdiff(a, b, periodic):
    d = np.abs(a.astype(np.float64) - b.astype(np.float64))
    for k, p in enumerate(periodic):
        if p:
            d[:, k] = np.minimum(d[:, k], 1.0 - d[:, k])
    return d


@pytest.mark.parametrize("n", [4096, 65536])
def test_paper_step_against_oracle(ab, ctx, n):
    """One step of the paper's example (r = sqrt(3/N), c = 1e-3, dt = 1) from
    rest: each side computes its own force (Eq. 1) and applies Eqs. 2-3."""
    w = synth.paper_shape(n)
    c = w.params["c"]
    dom = ab.Domain(2, (1, 1), w.radius)
    pos, vel = dev(w.pos), torch.zeros((n, 4), dtype=torch.float32, device="cuda:0")
    ab.ab_build(ctx, dom, pos)
    F = ab.ab_pair_sum(ctx, "expf", ab.OpParams(c=c))
    ab.ab_md_step(ctx, dom, pos, vel, F, 1.0)
    box = oracle.Box(2, (1, 1), (0, 0), (1, 1), w.radius)
    off, idx = oracle.neighbours_brute(box, w.pos) if n <= 4096 else oracle.CellList(box, w.pos).neighbours()
    Fo = oracle.pair_values("expf", box, w.pos, off, idx, params={"c": c})
    den = oracle.abs_terms("expf", box, w.pos, off, idx, params={"c": c})
    po, vo = md.md_step(w.pos, np.zeros_like(w.pos), Fo, 2, (1, 1), (0, 0), (1, 1), 1.0)
    v, p = host(vel), host(pos)
    # velocity = the force sum: the pair-sum bar (1e-5 of max(|y|, sum |t|))
    tol_v = 1e-5 * np.maximum(np.abs(vo[:, :2]), den[:, :2]) + 1e-12
    assert np.all(np.abs(v[:, :2] - vo[:, :2]) <= tol_v)
    # position: that error plus two FP32 roundings of a coordinate in [0, 1)
    assert np.all(_pdiff(p[:, :2], po[:, :2], (1, 1)) <= tol_v + 2.4e-7)
    assert np.all((p[:, :2] >= 0) & (p[:, :2] < 1))


def test_walls_and_wraps_against_oracle(ab, ctx):
    """Seeded synthetic state pushed through periodic faces and walls."""
    n = 200000
    g = np.random.default_rng(41)
    pos = synth.pack4(g.uniform(0, 1, (n, 3)).astype(np.float32))
    vel = synth.pack4(g.uniform(-0.2, 0.2, (n, 3)).astype(np.float32))
    acc = synth.pack4(g.uniform(-0.05, 0.05, (n, 3)).astype(np.float32))
    periodic = (1, 0, 1)
    dom = ab.Domain(3, periodic, 0.1)
    for dt in (1.0, 0.37):
        p, v = dev(pos), dev(vel)
        ab.ab_md_step(ctx, dom, p, v, dev(acc), dt)
        po, vo = md.md_step(pos, vel, acc, 3, periodic, (0, 0, 0), (1, 1, 1), dt)
        ph, vh = host(p), host(v)
        assert _pdiff(ph[:, :3], po[:, :3], periodic).max() <= 3e-7
        assert np.abs(vh[:, :3] - vo[:, :3]).max() <= 6e-8
        assert np.array_equal(np.sign(vh[:, 1]), np.sign(vo[:, 1]))   # wall reversals agree
        assert np.all((ph[:, :3] >= 0) & (ph[:, :3] <= 1))


def test_time_loop_conserves_momentum(ab, ctx):
    """50 steps of the paper's loop: EXPF is antisymmetric, so the total
    momentum stays 0 up to FP32 rounding of the per-particle sums."""
    n = 65536
    w = synth.paper_shape(n)
    dom = ab.Domain(2, (1, 1), w.radius)
    pos, vel = dev(w.pos), torch.zeros((n, 4), dtype=torch.float32, device="cuda:0")
    prm = ab.OpParams(c=w.params["c"])
    bound = 0.0
    for _ in range(50):
        ab.ab_build(ctx, dom, pos)
        F = ab.ab_pair_sum(ctx, "expf", prm)
        bound += float(F[:, :2].abs().double().sum()) * 2.0 ** -22
        ab.ab_md_step(ctx, dom, pos, vel, F, 1.0)
    ab.ab_sync(ctx)
    v = host(vel)[:, :2].astype(np.float64)
    assert np.abs(v.sum(axis=0)).max() <= bound + np.abs(v).sum() * 2.0 ** -22
    assert np.abs(v).max() > 0


def test_md_step_errors_and_stale(ab, ctx):
    n = 1000
    dom = ab.Domain(2, (1, 1), 0.05)
    pos = dev(synth.uniform_positions(n, 2, 3))
    vel = torch.zeros((n, 4), dtype=torch.float32, device="cuda:0")
    acc = torch.zeros((n, 4), dtype=torch.float32, device="cuda:0")
    ab.ab_build(ctx, dom, pos)
    ab.ab_md_step(ctx, dom, pos, vel, acc, 1.0)
    with pytest.raises(ab.AbError) as e:
        ab.ab_pair_sum(ctx, "count", ab.OpParams())
    assert e.value.status == ab._abi.AB_ERR_STALE
    with pytest.raises(ab.AbError) as e:
        ab.ab_md_step(ctx, dom, pos, pos, acc, 1.0)
    assert e.value.status == ab._abi.AB_ERR_ALIAS
    with pytest.raises(ab.AbError) as e:
        ab.ab_md_step(ctx, dom, pos, vel, acc, float("nan"))
    assert e.value.status == ab._abi.AB_ERR_INVALID_ARG
    ab.ab_sync(ctx)


def test_linear_spring_md_step_against_oracle(ab, ctx):
    """The molecular-dynamics example program of Sec. 1: point particles
    interacting via a linear spring force, here AB_OP_SOFT (rest length r:
    f_i = sum_j -k (r - d) dx_ij / d for d < r), advanced by Eqs. 2-3 in 3-D.
    One step from a seeded moving state against the oracle's force sum and
    step."""
    n, r, k, dt = 20000, 0.05, 50.0, 1.0e-3
    periodic = (1, 1, 1)
    pos = synth.uniform_positions(n, 3, 21)
    vel = synth.pack4(np.random.default_rng(22).uniform(-0.05, 0.05, (n, 3)).astype(np.float32))
    dom = ab.Domain(3, periodic, r)
    p, v = dev(pos), dev(vel)
    ab.ab_build(ctx, dom, p)
    F = ab.ab_pair_sum(ctx, "soft", ab.OpParams(k=k))
    ab.ab_md_step(ctx, dom, p, v, F, dt)
    box = oracle.Box(3, periodic, (0, 0, 0), (1, 1, 1), r)
    off, idx = oracle.CellList(box, pos).neighbours()
    Fo = oracle.pair_values("soft", box, pos, off, idx, params={"k": k})
    den = oracle.abs_terms("soft", box, pos, off, idx, params={"k": k})
    po, vo = md.md_step(pos, vel, Fo, 3, periodic, (0, 0, 0), (1, 1, 1), dt)
    vh, ph = host(v)[:, :3].astype(np.float64), host(p)[:, :3]
    # the pair-sum bar on dt * F plus FP32 roundings of v, dt * F and their sum
    tol_v = dt * 1e-5 * np.maximum(np.abs(Fo[:, :3]), den[:, :3]) + 2.0 ** -22 * (
        np.abs(vo[:, :3]) + np.abs(vel[:, :3]) + dt * np.abs(Fo[:, :3]))
    assert np.all(np.abs(vh - vo[:, :3]) <= tol_v + 1e-12)
    # position: dt times that, plus two FP32 roundings of a coordinate in [0, 1)
    assert np.all(_pdiff(ph, po[:, :3], periodic) <= dt * tol_v + 2.4e-7)
    assert np.abs(vh - vel[:, :3]).max() > 0   # the springs did act


def test_linear_spring_time_loop_conserves_momentum(ab, ctx):
    """20 steps of the linear-spring loop from rest: the spring force is
    antisymmetric pair by pair, so the total momentum stays 0 up to FP32
    rounding of the per-particle sums and updates."""
    n, r, k, dt = 50000, 0.04, 50.0, 1.0e-3
    dom = ab.Domain(3, (1, 1, 1), r)
    pos = dev(synth.uniform_positions(n, 3, 23))
    vel = torch.zeros((n, 4), dtype=torch.float32, device="cuda:0")
    prm = ab.OpParams(k=k)
    bound = 0.0
    for _ in range(20):
        ab.ab_build(ctx, dom, pos)
        F = ab.ab_pair_sum(ctx, "soft", prm)
        bound += dt * float(F[:, :3].abs().double().sum()) * 2.0 ** -22
        ab.ab_md_step(ctx, dom, pos, vel, F, dt)
    ab.ab_sync(ctx)
    v = host(vel)[:, :3].astype(np.float64)
    assert np.abs(v.sum(axis=0)).max() <= bound + np.abs(v).sum() * 2.0 ** -22
    assert np.abs(v).max() > 0

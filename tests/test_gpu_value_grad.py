"""Forward values and the adjoint in one walk (ab_pair_sum_value_grad)
against the separate forward and adjoint calls, bit for bit, and against the
FP64 oracle (GPU, C ABI)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import dev, host, oracle_box, rel_err

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


def _case(name):
    if name == "gauss_clustered":
        w = synth.c3(n=1 << 18, n_blobs=16)
        return "gauss", 3, w.periodic, w.radius, w.pos, w.params, w.w, w.g
    if name == "gauss_2d_wall":
        pos = synth.uniform_positions(200000, 2, 31)
        return ("gauss", 2, (1, 0), 0.006, pos, {"s": 1.0 / 0.002 ** 2},
                synth.weights(200000, 32, "normal"), synth.weights(200000, 33, "normal"))
    if name == "gauss_general":
        pos = synth.uniform_positions(20000, 3, 34)
        return ("gauss", 3, (1, 1, 1), 0.26, pos, {"s": 30.0},
                synth.weights(20000, 35, "normal"), synth.weights(20000, 36, "normal"))
    if name == "lj_c2":
        w = synth.c2()
        return "lj", 3, w.periodic, w.radius, w.pos, w.params, None, w.g
    pos = synth.uniform_positions(300000, 2, 37)
    return ("lj", 2, (0, 1), 0.004, pos, {"eps": 1.0, "sigma": 0.002}, None,
            synth.weights(300000, 38))


@pytest.mark.parametrize("name", ["gauss_clustered", "gauss_2d_wall", "gauss_general", "lj_c2",
                                  "lj_2d_wall"])
def test_value_grad_equals_separate_calls_bitwise(ab, ctx, name):
    op, dim, periodic, r, pos, params, w, g = _case(name)
    prm = ab.OpParams(**{k: v for k, v in params.items() if k in ("s", "eps", "sigma")})
    ab.ab_build(ctx, ab.Domain(dim, periodic, r), dev(pos))
    n = pos.shape[0]
    f32 = dict(dtype=torch.float32, device="cuda:0")
    f64 = dict(dtype=torch.float64, device="cuda:0")
    wd = dev(w) if w is not None else None
    gd = dev(g)
    y_sep = torch.empty(n, **f32)
    e_sep = torch.empty((), **f64)
    ab.ab_pair_sum(ctx, op, prm, w=wd, out=y_sep, energy=e_sep if op == "lj" else None)
    gp_sep = torch.empty((n, 4), **f32)
    gw_sep = torch.empty(n, **f32) if op == "gauss" else None
    gs_sep = torch.empty((), **f64) if op == "gauss" else None
    ab.ab_pair_sum_bwd(ctx, op, prm, wd, gd, gp_sep, gw_sep, gs_sep)
    y = torch.empty(n, **f32)
    e = torch.empty((), **f64) if op == "lj" else None
    gp = torch.empty((n, 4), **f32)
    gw = torch.empty(n, **f32) if op == "gauss" else None
    gs = torch.empty((), **f64) if op == "gauss" else None
    ab.ab_pair_sum_value_grad(ctx, op, prm, wd, gd, out=y, energy=e, grad_pos4=gp,
                              grad_w=gw, grad_s=gs)
    ab.ab_sync(ctx)
    assert torch.equal(y, y_sep) and torch.equal(gp, gp_sep)
    if op == "gauss":
        assert torch.equal(gw, gw_sep) and torch.equal(gs, gs_sep)
    else:
        assert torch.equal(e, e_sep)


def test_value_grad_against_oracle(ab, ctx):
    w = synth.c1()
    g = synth.weights(w.n, 41, "normal")
    ab.ab_build(ctx, ab.Domain(2, w.periodic, w.radius), dev(w.pos))
    y, _, gp, gw, gs = ab.ab_pair_sum_value_grad(
        ctx, "gauss", ab.OpParams(s=w.params["s"]), dev(w.w), dev(g),
        out=torch.empty(w.n, dtype=torch.float32, device="cuda:0"),
        grad_pos4=torch.empty((w.n, 4), dtype=torch.float32, device="cuda:0"),
        grad_w=torch.empty(w.n, dtype=torch.float32, device="cuda:0"),
        grad_s=torch.empty((), dtype=torch.float64, device="cuda:0"))
    box = oracle_box(w)
    off, idx = oracle.neighbours_brute(box, w.pos)
    ref = oracle.pair_values("gauss", box, w.pos, off, idx, w=w.w, params=w.params)[:, 0]
    den = oracle.abs_terms("gauss", box, w.pos, off, idx, w=w.w, params=w.params)[:, 0]
    assert rel_err(host(y), ref, den) <= 1e-5
    rp, rw, rs = oracle.pair_grads("gauss", box, w.pos, off, idx, g, w=w.w, params=w.params)
    dp, dw, ds = oracle.abs_grad_terms("gauss", box, w.pos, off, idx, g, w=w.w, params=w.params)
    assert rel_err(host(gp)[:, :2], rp[:, :2], dp[:, :2]) <= 1e-5
    assert rel_err(host(gw), rw, dw) <= 1e-5
    assert abs(float(gs) - rs.sum()) <= 1e-5 * ds.sum()


def test_value_grad_errors(ab, ctx):
    pos = synth.uniform_positions(1000, 3, 9)
    ab.ab_build(ctx, ab.Domain(3, (1, 1, 1), 0.1), dev(pos))
    g = torch.ones(1000, dtype=torch.float32, device="cuda:0")
    with pytest.raises(ab.AbError) as e:
        ab.ab_pair_sum_value_grad(ctx, "expf", ab.OpParams(), None, g,
                                  out=torch.empty((1000, 4), dtype=torch.float32, device="cuda:0"))
    assert e.value.status == ab._abi.AB_ERR_UNSUPPORTED
    with pytest.raises(ab.AbError) as e:      # the output is the upstream gradient
        ab.ab_pair_sum_value_grad(ctx, "lj", ab.OpParams(sigma=0.01), None, g, out=g)
    assert e.value.status == ab._abi.AB_ERR_ALIAS
    buf = torch.empty((1000, 4), dtype=torch.float32, device="cuda:0")
    with pytest.raises(ab.AbError) as e:      # two outputs overlap
        ab.ab_pair_sum_value_grad(ctx, "lj", ab.OpParams(sigma=0.01), None, g,
                                  out=buf.view(-1)[:1000], grad_pos4=buf)
    assert e.value.status == ab._abi.AB_ERR_ALIAS
    ab.ab_sync(ctx)

"""Pins of the oracle's pair operators and adjoints (CPU only).

Closed forms for two and three particles, Newton's third law for the
symmetric pair forces (paper Sec. 3, Eq. 1), the energy/force relation and
central finite differences in FP64 for every adjoint.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _pos(pts):
    return synth.pack4(np.asarray(pts, np.float32))


def test_lj_two_particles_closed_form():
    d = 0.015
    sig, eps = 0.01, 1.0
    pos = _pos([[0.5, 0.5, 0.5], [0.5 + d, 0.5, 0.5]])
    box = oracle.Box(3, (1, 1, 1), radius=0.0197)
    off, idx = oracle.neighbours_brute(box, pos)
    e = oracle.pair_values("lj", box, pos, off, idx,
                           params={"eps": eps, "sigma": sig})[:, 0]
    dd = float(np.float32(0.5 + d)) - float(np.float32(0.5))
    phi = eps * ((sig / dd) ** 12 - (sig / dd) ** 6)
    assert np.allclose(e, [phi / 2, phi / 2], rtol=1e-13)
    # force on particle 0 along +x is -dphi/dd (repulsive at d < 2^(1/6) sig)
    g = np.ones(2)
    dpos, _, _ = oracle.pair_grads("lj", box, pos, off, idx, g,
                                   params={"eps": eps, "sigma": sig})
    dphi = eps * (-12 * sig ** 12 / dd ** 13 + 6 * sig ** 6 / dd ** 7)
    # dE/dx_0 = dphi/dd * d(dd)/dx_0 = -dphi
    assert math.isclose(dpos[0, 0], -dphi, rel_tol=1e-12)
    assert math.isclose(dpos[1, 0], dphi, rel_tol=1e-12)


def test_gauss_three_point_line():
    """x = 0.1, 0.125, 0.15625 on a line; r = 0.04 links 0-1 and 1-2 only."""
    xs = [0.1, 0.125, 0.15625]
    pos = _pos([[x, 0.5] for x in xs])
    w = np.array([0.5, -2.0, 3.0], np.float32)
    s = 400.0
    box = oracle.Box(2, (0, 0), radius=0.04)
    off, idx = oracle.neighbours_brute(box, pos)
    assert list(np.diff(off)) == [1, 2, 1]
    y = oracle.pair_values("gauss", box, pos, off, idx, w=w, params={"s": s})[:, 0]
    x64 = [float(np.float32(x)) for x in xs]
    k01 = math.exp(-s * (x64[1] - x64[0]) ** 2)
    k12 = math.exp(-s * (x64[2] - x64[1]) ** 2)
    assert np.allclose(y, [-2.0 * k01, 0.5 * k01 + 3.0 * k12, -2.0 * k12], rtol=1e-14)


@pytest.mark.parametrize("op,params", [("expf", {"c": 1e-3}), ("soft", {"k": 1e4})])
def test_force_two_particles_closed_form(op, params):
    r = 0.1
    pos = _pos([[0.2, 0.3], [0.25, 0.34]])
    box = oracle.Box(2, (1, 1), radius=r)
    off, idx = oracle.neighbours_brute(box, pos)
    f = oracle.pair_values(op, box, pos, off, idx, params=params)
    p = pos.astype(np.float64)
    dx = p[1, :2] - p[0, :2]
    d = math.hypot(*dx)
    r32 = float(np.float32(r))      # the radius is an FP32 parameter
    mag = -params["c"] * math.exp(-d) if op == "expf" else -params["k"] * (r32 - d)
    assert np.allclose(f[0, :2], mag * dx / d, rtol=1e-13)
    assert np.allclose(f[1, :2], -mag * dx / d, rtol=1e-13)
    # repulsive: particle 0 is pushed away from particle 1
    assert np.dot(f[0, :2], dx) < 0


def test_force_through_periodic_face():
    """The pair across the face sees the short separation 0.02, not 0.98."""
    pos = _pos([[0.01, 0.5], [0.99, 0.5]])
    box = oracle.Box(2, (1, 1), radius=0.03)
    off, idx = oracle.neighbours_brute(box, pos)
    f = oracle.pair_values("expf", box, pos, off, idx, params={"c": 1.0})
    d = float(np.float32(0.01)) + 1.0 - float(np.float32(0.99))
    # dx_01 = x1 - x0 through the face = -d, so f_0 = -exp(-d) * (-1) > 0
    assert math.isclose(f[0, 0], math.exp(-d), rel_tol=1e-12)
    assert math.isclose(f[1, 0], -math.exp(-d), rel_tol=1e-12)


@pytest.mark.parametrize("op,params", [("expf", {"c": 1e-3}), ("soft", {"k": 1e4})])
def test_newton_third_law_forces(op, params):
    pos = synth.uniform_positions(3000, 2, 21)
    box = oracle.Box(2, (1, 1), radius=0.04)
    off, idx = oracle.neighbours_brute(box, pos)
    f = oracle.pair_values(op, box, pos, off, idx, params=params)
    tot = np.abs(f).sum()
    assert np.all(np.abs(f.sum(0)) <= 1e-13 * tot)


def test_newton_third_law_lj_gradient():
    w = synth.c2(n=20000)
    box = oracle.Box(3, (1, 1, 1), radius=0.08)
    off, idx = oracle.neighbours_brute(box, w.pos)
    g = np.ones(w.n)
    dpos, _, _ = oracle.pair_grads("lj", box, w.pos, off, idx, g, params=w.params)
    assert np.all(np.abs(dpos.sum(0)) <= 1e-12 * np.abs(dpos).sum())


def _fd_case(dim, n, r, seed, periodic=(1, 1, 1)):
    pos = synth.uniform_positions(n, dim, seed)
    box = oracle.Box(dim, periodic[:dim], radius=r)
    off, idx = oracle.neighbours_brute(box, pos)
    return pos, box, off, idx


@pytest.mark.parametrize("dim", [2, 3])
def test_lj_adjoint_finite_differences(dim):
    """dL/dx for L = sum_i g_i E_i against FP64 central differences over the
    fixed neighbour set."""
    pos, box, off, idx = _fd_case(dim, 300, 0.2 if dim == 3 else 0.1, 5 + dim)
    params = {"eps": 1.0, "sigma": 0.02}
    rng = np.random.default_rng(1)
    g = rng.uniform(0.5, 1.5, len(pos))
    p64 = pos.astype(np.float64)
    dpos, _, _ = oracle.pair_grads("lj", box, pos, off, idx, g, params=params)

    def L(p):
        return float(g @ oracle.pair_values64("lj", box, p, off, idx, params=params)[:, 0])

    for i in rng.choice(len(pos), 12, replace=False):
        for k in range(dim):
            h = 1e-7
            pp = p64.copy(); pp[i, k] += h
            pm = p64.copy(); pm[i, k] -= h
            fd = (L(pp) - L(pm)) / (2 * h)
            assert math.isclose(fd, dpos[i, k], rel_tol=1e-5, abs_tol=1e-6 * abs(dpos).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_gauss_adjoint_finite_differences(dim):
    pos, box, off, idx = _fd_case(dim, 300, 0.15, 17 + dim, periodic=(1, 0, 1))
    rng = np.random.default_rng(2)
    w = rng.standard_normal(len(pos))
    g = rng.standard_normal(len(pos))
    s = 30.0
    p64 = pos.astype(np.float64)
    dpos, dw, dsp = oracle.pair_grads("gauss", box, pos, off, idx, g, w=w, params={"s": s})

    def L(p=p64, ww=w, ss=s):
        return float(g @ oracle.pair_values64("gauss", box, p, off, idx, w=ww,
                                               params={"s": ss})[:, 0])

    for i in rng.choice(len(pos), 10, replace=False):
        for k in range(dim):
            h = 1e-6
            pp = p64.copy(); pp[i, k] += h
            pm = p64.copy(); pm[i, k] -= h
            fd = (L(p=pp) - L(p=pm)) / (2 * h)
            assert math.isclose(fd, dpos[i, k], rel_tol=1e-6, abs_tol=1e-7 * abs(dpos).max())
        wp = w.copy(); wp[i] += 1e-3
        wm = w.copy(); wm[i] -= 1e-3
        fd = (L(ww=wp) - L(ww=wm)) / 2e-3
        assert math.isclose(fd, dw[i], rel_tol=1e-9, abs_tol=1e-12)
    fd = (L(ss=s + 1e-4) - L(ss=s - 1e-4)) / 2e-4
    assert math.isclose(fd, dsp.sum(), rel_tol=1e-7)


def test_gauss_dw_is_forward_with_g_as_weights():
    """Transpose identity: the kernel is symmetric, so dL/dw = K g."""
    w = synth.c1()
    box = oracle.Box(2, (1, 1), radius=w.radius)
    off, idx = oracle.neighbours_brute(box, w.pos)
    g = synth.weights(w.n, 3)
    _, dw, _ = oracle.pair_grads("gauss", box, w.pos, off, idx, g, w=w.w, params=w.params)
    y = oracle.pair_values("gauss", box, w.pos, off, idx, w=g, params=w.params)[:, 0]
    assert np.allclose(dw, y, rtol=1e-13, atol=1e-15)


def test_expf_is_minus_gradient_of_exp_potential():
    """Eq. 1 force is -grad of U = sum_{i<j} c exp(-d_ij) on the fixed set."""
    pos, box, off, idx = _fd_case(2, 200, 0.1, 31)
    c = 0.7
    f = oracle.pair_values("expf", box, pos, off, idx, params={"c": c})
    p64 = pos.astype(np.float64)
    rows = np.repeat(np.arange(len(pos)), np.diff(off))

    def U(p):
        dx = p[idx, :2] - p[rows, :2]
        dx -= np.round(dx)
        d = np.sqrt((dx * dx).sum(1))
        return 0.5 * c * np.exp(-d).sum()

    rng = np.random.default_rng(4)
    for i in rng.choice(len(pos), 10, replace=False):
        for k in range(2):
            h = 1e-5
            pp = p64.copy(); pp[i, k] += h
            pm = p64.copy(); pm[i, k] -= h
            fd = -(U(pp) - U(pm)) / (2 * h)
            assert math.isclose(fd, f[i, k], rel_tol=1e-6, abs_tol=1e-9)


def test_abs_terms_bound_values():
    w = synth.c1()
    box = oracle.Box(2, (1, 1), radius=w.radius)
    off, idx = oracle.neighbours_brute(box, w.pos)
    y = oracle.pair_values("gauss", box, w.pos, off, idx, w=w.w, params=w.params)
    a = oracle.abs_terms("gauss", box, w.pos, off, idx, w=w.w, params=w.params)
    assert np.all(np.abs(y[:, 0]) <= a[:, 0] + 1e-15)


# ---- the error-metric denominators (absmode), pinned by hand-computed values
# Each denominator is the sum of the magnitudes of a row's elementary terms;
# a wrong one (a sign kept, a part dropped) changes these numbers.

def _line3(xs, dim=2):
    pts = [[x, 0.5, 0.5][:dim] for x in xs]
    return _pos(pts), [float(np.float32(x)) for x in xs]


def test_abs_terms_gauss_three_point_line():
    pos, x = _line3([0.1, 0.125, 0.15625])
    w = np.array([0.5, -2.0, 3.0], np.float32)
    s = 400.0
    box = oracle.Box(2, (0, 0), radius=0.04)
    off, idx = oracle.neighbours_brute(box, pos)
    a = oracle.abs_terms("gauss", box, pos, off, idx, w=w, params={"s": s})[:, 0]
    k01 = math.exp(-s * (x[1] - x[0]) ** 2)
    k12 = math.exp(-s * (x[2] - x[1]) ** 2)
    assert np.allclose(a, [2.0 * k01, 0.5 * k01 + 3.0 * k12, 2.0 * k12], rtol=1e-14)


def test_abs_terms_lj_three_point_line():
    """LJ counts the repulsive and attractive halves in magnitude:
    1/2 eps (sr12 + sr6) per pair; the middle particle has two pairs."""
    sig, eps = 0.01, 1.5
    pos, x = _line3([0.5, 0.511, 0.5235], dim=3)
    box = oracle.Box(3, (1, 1, 1), radius=0.0197)
    off, idx = oracle.neighbours_brute(box, pos)
    assert list(np.diff(off)) == [1, 2, 1]
    prm = {"eps": eps, "sigma": sig}
    a = oracle.abs_terms("lj", box, pos, off, idx, params=prm)[:, 0]

    def half(d):
        sr6 = (sig / d) ** 6
        return 0.5 * eps * (sr6 * sr6 + sr6)

    h01, h12 = half(x[1] - x[0]), half(x[2] - x[1])
    assert np.allclose(a, [h01, h01 + h12, h12], rtol=1e-12)
    # the value itself subtracts the halves
    y = oracle.pair_values("lj", box, pos, off, idx, params=prm)[:, 0]
    v01 = 0.5 * eps * ((sig / (x[1] - x[0])) ** 12 - (sig / (x[1] - x[0])) ** 6)
    assert math.isclose(y[0], v01, rel_tol=1e-12)


def test_abs_terms_expf_and_soft_two_particles():
    r = 0.1
    pos = _pos([[0.2, 0.3], [0.25, 0.34]])
    box = oracle.Box(2, (1, 1), radius=r)
    off, idx = oracle.neighbours_brute(box, pos)
    p = pos.astype(np.float64)
    dx = p[1, :2] - p[0, :2]
    d = math.hypot(*dx)
    r32 = float(np.float32(r))
    c, k = 1e-3, 1e4
    ae = oracle.abs_terms("expf", box, pos, off, idx, params={"c": c})
    assert np.allclose(ae[0, :2], c * math.exp(-d) * np.abs(dx) / d, rtol=1e-13)
    assert np.allclose(ae[1, :2], ae[0, :2], rtol=1e-13)
    # SOFT: the k r and k d parts of k (r - d) in magnitude: k (r + d)
    asf = oracle.abs_terms("soft", box, pos, off, idx, params={"k": k})
    assert np.allclose(asf[0, :2], k * (r32 + d) * np.abs(dx) / d, rtol=1e-13)
    assert np.allclose(asf[1, :2], asf[0, :2], rtol=1e-13)


def test_abs_terms_sph_two_particles():
    """Density: |m_j| W(d) + |m_i| W(0); force: |m_j| (|A_i| + |A_j|) |W'(d)/d| |dx|."""
    r = 0.1
    pos = _pos([[0.2, 0.3, 0.4], [0.24, 0.33, 0.41]])
    box = oracle.Box(3, (1, 1, 1), radius=r)
    off, idx = oracle.neighbours_brute(box, pos)
    p = pos.astype(np.float64)
    dx = p[1, :3] - p[0, :3]
    d = math.sqrt(float(dx @ dx))
    r32 = float(np.float32(r))
    a_n = 21.0 / (2.0 * math.pi * r32 ** 3)
    q = d / r32
    W = a_n * (1 - q) ** 4 * (1 + 4 * q)
    m = np.array([0.5, -1.25])
    rho = oracle.abs_terms("sph_density", box, pos, off, idx, w=m)[:, 0]
    assert np.allclose(rho, [1.25 * W + 0.5 * a_n, 0.5 * W + 1.25 * a_n], rtol=1e-13)
    A = np.array([-0.75, 2.0])
    wv = np.stack([m, A], 1)
    af = oracle.abs_terms("sph_force", box, pos, off, idx, w=wv)
    gradcoef = 20.0 * a_n * (1 - q) ** 3 / r32 ** 2
    assert np.allclose(af[0, :3], 1.25 * (0.75 + 2.0) * gradcoef * np.abs(dx), rtol=1e-12)
    assert np.allclose(af[1, :3], 0.5 * (0.75 + 2.0) * gradcoef * np.abs(dx), rtol=1e-12)


def test_abs_grad_terms_gauss_two_particles():
    """Adjoint denominators: position (|g_i w_j| + |g_j w_i|) 2 s k |dx|,
    weight |g_j| k, lengthscale |g_i w_j| k d^2."""
    pos = _pos([[0.3, 0.5], [0.32, 0.515]])
    box = oracle.Box(2, (0, 0), radius=0.05)
    off, idx = oracle.neighbours_brute(box, pos)
    p = pos.astype(np.float64)
    dx = p[1, :2] - p[0, :2]
    d2 = float(dx @ dx)
    s = 300.0
    kij = math.exp(-s * d2)
    w = np.array([1.5, -0.5])
    g = np.array([-2.0, 0.25])
    ap, aw, as_ = oracle.abs_grad_terms("gauss", box, pos, off, idx, g, w=w, params={"s": s})
    cpos = (abs(g[0] * w[1]) + abs(g[1] * w[0])) * 2 * s * kij
    assert np.allclose(ap[0, :2], cpos * np.abs(dx), rtol=1e-13)
    assert np.allclose(ap[1, :2], cpos * np.abs(dx), rtol=1e-13)
    assert np.allclose(aw, [abs(g[1]) * kij, abs(g[0]) * kij], rtol=1e-13)
    assert np.allclose(as_, [abs(g[0] * w[1]) * kij * d2, abs(g[1] * w[0]) * kij * d2],
                       rtol=1e-13)
    # the signed value of the position gradient for comparison
    vp, _, _ = oracle.pair_grads("gauss", box, pos, off, idx, g, w=w, params={"s": s})
    cv = (g[0] * w[1] + g[1] * w[0]) * 2 * s * kij
    assert np.allclose(vp[0, :2], cv * dx, rtol=1e-13)


def test_abs_grad_terms_lj_two_particles():
    """1/2 (g_i + g_j) eps (12 sr12 + 6 sr6) / d^2 |dx| per pair."""
    sig, eps = 0.01, 2.0
    pos = _pos([[0.5, 0.5, 0.5], [0.512, 0.505, 0.5]])
    box = oracle.Box(3, (1, 1, 1), radius=0.0197)
    off, idx = oracle.neighbours_brute(box, pos)
    p = pos.astype(np.float64)
    dx = p[1, :3] - p[0, :3]
    d2 = float(dx @ dx)
    sr6 = (sig * sig / d2) ** 3
    g = np.array([0.75, 1.25])
    a, _, _ = oracle.abs_grad_terms("lj", box, pos, off, idx, g, params={"eps": eps, "sigma": sig})
    ca = 0.5 * (g[0] + g[1]) * eps * (12 * sr6 * sr6 + 6 * sr6) / d2
    assert np.allclose(a[0, :3], ca * np.abs(dx), rtol=1e-12)
    assert np.allclose(a[1, :3], ca * np.abs(dx), rtol=1e-12)


@pytest.mark.parametrize("op", ["gauss", "lj", "expf", "soft", "sph_density", "sph_force"])
def test_abs_terms_bound_every_operator(op):
    w = synth.c2(n=3000)
    box = oracle.Box(3, (1, 1, 1), radius=0.09)
    off, idx = oracle.neighbours_brute(box, w.pos)
    rng = np.random.default_rng(5)
    wt = None
    if op in ("gauss", "sph_density"):
        wt = rng.standard_normal(w.n)
    elif op == "sph_force":
        wt = np.stack([rng.random(w.n), rng.standard_normal(w.n)], 1)
    prm = {"s": 200.0, "eps": 1.0, "sigma": 0.01, "c": 1.0, "k": 10.0}
    y = oracle.pair_values(op, box, w.pos, off, idx, w=wt, params=prm)
    a = oracle.abs_terms(op, box, w.pos, off, idx, w=wt, params=prm)
    assert np.all(np.abs(y) <= a * (1 + 1e-12) + 1e-300)

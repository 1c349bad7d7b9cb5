"""Pins of the dense kernel-operator oracle (CPU only)."""
import math

import numpy as np

import synth
from oracle import dense


def test_s_zero_gives_column_sums():
    w = synth.c4(m=64, n=200, nrhs=8)
    y = dense.matvec(w.X, w.Y, w.W, 0.0)
    assert np.allclose(y, np.tile(w.W.astype(np.float64).sum(0), (64, 1)), rtol=1e-13)


def test_identity_case():
    """X = Y on a coarse lattice with s large: K = I to FP64 precision."""
    g = np.stack(np.meshgrid(*[np.arange(5) / 5.0] * 3, indexing="ij"), -1).reshape(-1, 3)
    X = g.astype(np.float32)
    W = np.random.default_rng(0).standard_normal((len(X), 4))
    y = dense.matvec(X, X, W, 5000.0)      # exp(-5000*0.04) = 1e-87
    assert np.allclose(y, W, rtol=1e-14, atol=1e-80)


def test_tiny_case_double_loop():
    rng = np.random.default_rng(3)
    X = rng.random((4, 3)).astype(np.float32)
    Y = rng.random((5, 3)).astype(np.float32)
    W = rng.standard_normal((5, 2))
    s = 3.0
    out = np.zeros((4, 2))
    for i in range(4):
        for j in range(5):
            d2 = sum((float(X[i, k]) - float(Y[j, k])) ** 2 for k in range(3))
            for c in range(2):
                out[i, c] += math.exp(-s * d2) * W[j, c]
    assert np.allclose(dense.matvec(X, Y, W, s), out, rtol=1e-14)


def test_adjoints_finite_differences():
    rng = np.random.default_rng(7)
    m, n, c = 40, 50, 5
    X = rng.random((m, 3))
    Y = rng.random((n, 3))
    W = rng.standard_normal((n, c))
    G = rng.standard_normal((m, c))
    s = 20.0

    def L(X=X, Y=Y, W=W, s=s):
        return float((G * dense.matvec(X, Y, W, s)).sum())

    dW = dense.grad_W(X, Y, G, s)
    dX = dense.grad_X(X, Y, W, G, s)
    dY = dense.grad_Y(X, Y, W, G, s)
    ds = dense.grad_s(X, Y, W, G, s)
    h = 1e-6
    for (i, k) in [(0, 0), (7, 2), (39, 1)]:
        Xp = X.copy(); Xp[i, k] += h
        Xm = X.copy(); Xm[i, k] -= h
        assert math.isclose((L(X=Xp) - L(X=Xm)) / (2 * h), dX[i, k], rel_tol=1e-6, abs_tol=1e-8)
    for (j, k) in [(0, 0), (13, 1), (49, 2)]:
        Yp = Y.copy(); Yp[j, k] += h
        Ym = Y.copy(); Ym[j, k] -= h
        assert math.isclose((L(Y=Yp) - L(Y=Ym)) / (2 * h), dY[j, k], rel_tol=1e-6, abs_tol=1e-8)
    for (j, k) in [(0, 0), (21, 4)]:
        Wp = W.copy(); Wp[j, k] += 1e-3
        Wm = W.copy(); Wm[j, k] -= 1e-3
        assert math.isclose((L(W=Wp) - L(W=Wm)) / 2e-3, dW[j, k], rel_tol=1e-9)
    assert math.isclose((L(s=s + 1e-5) - L(s=s - 1e-5)) / 2e-5, ds, rel_tol=1e-6)
    # chain rule to the lengthscale, s = 1/(2 l^2)
    l = 1.0 / math.sqrt(2 * s)
    dl = dense.grad_lengthscale(ds, l)
    sl = lambda ll: 1.0 / (2 * ll * ll)
    fd = (L(s=sl(l + 1e-7)) - L(s=sl(l - 1e-7))) / 2e-7
    assert math.isclose(fd, dl, rel_tol=1e-5)


def test_row_and_column_subsets():
    w = synth.c4(m=300, n=400, nrhs=6)
    rows = np.array([0, 17, 299])
    full = dense.matvec(w.X, w.Y, w.W, w.s)
    assert np.allclose(dense.matvec(w.X, w.Y, w.W, w.s, rows=rows), full[rows], rtol=1e-14)
    dW = dense.grad_W(w.X, w.Y, w.G, w.s)
    assert np.allclose(dense.grad_W(w.X, w.Y, w.G, w.s, cols=rows), dW[rows], rtol=1e-13)

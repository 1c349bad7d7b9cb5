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


def test_adjoint_abs_terms_hand_computed():
    """One x, two y, two right-hand sides: the elementary terms of dL/dx_ik
    are -2 s G_ic W_jc K_j (x_k - y_jk), one per (j, c); the denominators sum
    their magnitudes."""
    X = np.array([[0.25, 0.5, 0.75]])
    Y = np.array([[0.5, 0.25, 0.75], [0.0, 1.0, 0.5]])
    W = np.array([[1.5, -0.5], [-2.0, 0.25]])
    G = np.array([[0.5, -3.0]])
    s = 2.0
    K = [math.exp(-s * sum((X[0, k] - Y[j, k]) ** 2 for k in range(3))) for j in range(2)]
    aX = [sum(2 * s * abs(G[0, c] * W[j, c]) * K[j] * abs(X[0, k] - Y[j, k])
              for j in range(2) for c in range(2)) for k in range(3)]
    vX = [sum(-2 * s * G[0, c] * W[j, c] * K[j] * (X[0, k] - Y[j, k])
              for j in range(2) for c in range(2)) for k in range(3)]
    assert np.allclose(dense.grad_X_abs(X, Y, W, G, s)[0], aX, rtol=1e-14)
    assert np.allclose(dense.grad_X(X, Y, W, G, s)[0], vX, rtol=1e-13)
    aY = [[sum(2 * s * abs(G[0, c] * W[j, c]) * K[j] * abs(X[0, k] - Y[j, k])
               for c in range(2)) for k in range(3)] for j in range(2)]
    assert np.allclose(dense.grad_Y_abs(X, Y, W, G, s), aY, rtol=1e-14)
    aS = sum(abs(G[0, c] * W[j, c]) * K[j] * sum((X[0, k] - Y[j, k]) ** 2 for k in range(3))
             for j in range(2) for c in range(2))
    assert math.isclose(dense.grad_s_abs(X, Y, W, G, s), aS, rel_tol=1e-14)


def test_adjoint_abs_terms_equal_magnitude_when_signs_agree():
    """Positive G, W and every y below every x in each coordinate: all the
    elementary terms of dX (and of dY) share one sign, so the denominator
    equals |dX| (|dY|) exactly up to rounding."""
    rng = np.random.default_rng(11)
    X = 0.6 + 0.4 * rng.random((20, 3))
    Y = 0.5 * rng.random((30, 3))
    W = rng.random((30, 4)) + 0.1
    G = rng.random((20, 4)) + 0.1
    s = 3.0
    assert np.allclose(dense.grad_X_abs(X, Y, W, G, s), np.abs(dense.grad_X(X, Y, W, G, s)),
                       rtol=1e-12)
    assert np.allclose(dense.grad_Y_abs(X, Y, W, G, s), np.abs(dense.grad_Y(X, Y, W, G, s)),
                       rtol=1e-12)
    assert math.isclose(dense.grad_s_abs(X, Y, W, G, s), abs(dense.grad_s(X, Y, W, G, s)),
                        rel_tol=1e-12)


def test_adjoint_abs_terms_bound_and_exceed_mixed_signs():
    w = synth.c4(m=60, n=80, nrhs=8, seed_offset=4)
    for fn, fa in ((dense.grad_X, dense.grad_X_abs), (dense.grad_Y, dense.grad_Y_abs)):
        v = fn(w.X, w.Y, w.W, w.G, w.s)
        a = fa(w.X, w.Y, w.W, w.G, w.s)
        assert np.all(np.abs(v) <= a * (1 + 1e-12))
        # signs of G, W and x - y are mixed: cancellation makes most
        # elements strictly smaller than the sum of magnitudes
        assert np.mean(np.abs(v) < 0.9 * a) > 0.5

"""Dense kernel operator and its adjoint in FP64 (TEST INFRASTRUCTURE).

Only tests, the smoke check and the benchmark's CPU legs may use this module.

The paper's RBF-interpolation, Kansa and Gaussian-process examples (Sec. 1,
Sec. 1.1) apply a dense kernel matrix to vectors; Sec. 2.2.2 names fast
summation of such global operators as Level-2 work.  The operator here is

    K_ij = exp(-s * |x_i - y_j|^2),        Y_out = K W,

the Gaussian (squared-exponential) kernel with s = 1/(2 l^2) for lengthscale
l.  Its adjoint for an upstream gradient G = dL/dY_out is

    dL/dW   = K^T G
    A_ij    = (G_i . W_j) K_ij
    dL/dx_i = -2 s sum_j A_ij (x_i - y_j)
    dL/dy_j = +2 s sum_i A_ij (x_i - y_j)
    dL/ds   = -sum_ij A_ij |x_i - y_j|^2
    dL/dl   = dL/ds * ds/dl = dL/ds * (-1 / l^3)

Everything is the plain definition evaluated in FP64 from the FP32 inputs,
one row block at a time (rows are independent; the blocking only bounds
memory).  Pinned by: the s = 0 case (K = all ones, so K W = column sums of
W), the well-separated identity case (X = Y, s large, K W = W), a pure-Python
double loop on a tiny case, and central finite differences of the forward
for every adjoint.
"""
from __future__ import annotations

import numpy as np


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def sqdist(X, Y):
    """|x_i - y_j|^2 by direct differences, FP64, shape [m, n]."""
    X = _f64(X)
    Y = _f64(Y)
    d = X[:, None, :] - Y[None, :, :]
    return np.einsum("ijk,ijk->ij", d, d)


def kernel(X, Y, s):
    return np.exp(-float(s) * sqdist(X, Y))


def matvec(X, Y, W, s, rows=None, block=256):
    """FP64 ``K(X[rows], Y) W``; ``rows`` selects output rows (default all)."""
    X = _f64(X)
    Y = _f64(Y)
    W = _f64(W)
    if rows is not None:
        X = X[np.asarray(rows)]
    out = np.zeros((X.shape[0], W.shape[1]))
    for a in range(0, X.shape[0], block):
        out[a:a + block] = kernel(X[a:a + block], Y, s) @ W
    return out


def matvec_abs(X, Y, W, s, rows=None, block=256):
    """sum_j K_ij |W_jc| -- the denominator of the dense error metric."""
    return matvec(X, Y, np.abs(_f64(W)), s, rows, block)


def grad_W(X, Y, G, s, cols=None, block=256):
    """dL/dW = K^T G, optionally only for the Y-rows ``cols``."""
    X = _f64(X)
    Y = _f64(Y)
    G = _f64(G)
    if cols is not None:
        Y = Y[np.asarray(cols)]
    out = np.zeros((Y.shape[0], G.shape[1]))
    for a in range(0, X.shape[0], block):
        out += kernel(X[a:a + block], Y, s).T @ G[a:a + block]
    return out


def grad_X(X, Y, W, G, s, rows=None, block=256):
    """dL/dx_i for the rows ``rows`` (default all)."""
    X = _f64(X)
    Y = _f64(Y)
    W = _f64(W)
    G = _f64(G)
    if rows is not None:
        X = X[np.asarray(rows)]
        G = G[np.asarray(rows)]
    out = np.zeros(X.shape)
    for a in range(0, X.shape[0], block):
        Xb = X[a:a + block]
        A = (G[a:a + block] @ W.T) * kernel(Xb, Y, s)
        out[a:a + block] = -2.0 * s * (Xb * A.sum(1)[:, None] - A @ Y)
    return out


def grad_Y(X, Y, W, G, s, cols=None, block=256):
    """dL/dy_j for the Y-rows ``cols`` (default all)."""
    X = _f64(X)
    Y = _f64(Y)
    W = _f64(W)
    G = _f64(G)
    if cols is not None:
        Y = Y[np.asarray(cols)]
        W = W[np.asarray(cols)]
    out = np.zeros(Y.shape)
    for a in range(0, X.shape[0], block):
        Xb = X[a:a + block]
        A = (G[a:a + block] @ W.T) * kernel(Xb, Y, s)          # [b, n]
        out += 2.0 * s * (A.T @ Xb - Y * A.sum(0)[:, None])
    return out


def grad_X_abs(X, Y, W, G, s, rows=None, block=256):
    """Per-element denominator of the dX error metric: the magnitudes of the
    elementary terms of dL/dx_ik summed,

        2 s sum_j sum_c |G_ic| |W_jc| K_ij |x_ik - y_jk|,

    one term per (j, c) of dL/dx_ik = -2 s sum_j sum_c G_ic W_jc K_ij
    (x_ik - y_jk).  It bounds |dL/dx_ik| and equals it when every term has
    the same sign."""
    X = _f64(X)
    Y = _f64(Y)
    W = np.abs(_f64(W))
    G = np.abs(_f64(G))
    if rows is not None:
        X = X[np.asarray(rows)]
        G = G[np.asarray(rows)]
    out = np.zeros(X.shape)
    for a in range(0, X.shape[0], block):
        Xb = X[a:a + block]
        B = (G[a:a + block] @ W.T) * kernel(Xb, Y, s)            # [b, n]
        for k in range(X.shape[1]):
            out[a:a + block, k] = 2.0 * s * (B * np.abs(Xb[:, k, None] - Y[None, :, k])).sum(1)
    return out


def grad_Y_abs(X, Y, W, G, s, cols=None, block=256):
    """Per-element denominator of the dY error metric:
    2 s sum_i sum_c |G_ic| |W_jc| K_ij |x_ik - y_jk| (see grad_X_abs)."""
    X = _f64(X)
    Y = _f64(Y)
    W = np.abs(_f64(W))
    G = np.abs(_f64(G))
    if cols is not None:
        Y = Y[np.asarray(cols)]
        W = W[np.asarray(cols)]
    out = np.zeros(Y.shape)
    for a in range(0, X.shape[0], block):
        Xb = X[a:a + block]
        B = (G[a:a + block] @ W.T) * kernel(Xb, Y, s)            # [b, n]
        for k in range(Y.shape[1]):
            out[:, k] += 2.0 * s * (B * np.abs(Xb[:, k, None] - Y[None, :, k])).sum(0)
    return out


def grad_s(X, Y, W, G, s, block=256):
    """dL/ds = -sum_ij (G_i . W_j) K_ij d_ij^2 over all pairs."""
    X = _f64(X)
    Y = _f64(Y)
    W = _f64(W)
    G = _f64(G)
    tot = 0.0
    for a in range(0, X.shape[0], block):
        D2 = sqdist(X[a:a + block], Y)
        A = (G[a:a + block] @ W.T) * np.exp(-s * D2)
        tot -= float((A * D2).sum())
    return tot


def grad_s_abs(X, Y, W, G, s, block=256):
    """Denominator of the ds error metric: sum_ij sum_c |G_ic| |W_jc| K_ij d_ij^2,
    the magnitudes of the elementary terms of dL/ds summed."""
    return -grad_s(X, Y, np.abs(_f64(W)), np.abs(_f64(G)), s, block)


def grad_lengthscale(ds, lengthscale):
    """Chain rule for s = 1/(2 l^2): ds/dl = -1/l^3."""
    return ds * (-1.0 / lengthscale ** 3)

"""Kernel-system solve (K(X, X) + sigma^2 I) W = B (TEST INFRASTRUCTURE).

Only tests, the smoke check and the benchmark's CPU legs may use this module.

RBF interpolation with a nugget and the Gaussian-process posterior mean
(paper Sec. 1.1) both need the weights W of this symmetric positive definite
system, K_ij = exp(-s |x_i - x_j|^2).  Two routes, in FP64:

  direct(X, B, s, sigma2)  -- the textbook dense solve (Cholesky through
                              numpy.linalg.solve);
  cg(X, B, s, sigma2, tol, max_iter)  -- Hestenes and Stiefel's conjugate
      gradients, one independent iteration per column of B, from W = 0:
          r = b, p = r
          repeat: alpha = r.r / p.Ap;  w += alpha p;  r -= alpha Ap;
                  stop if ||r|| <= tol ||b||;  beta = r'.r' / r.r;
                  p = r' + beta p
      A column that has stopped keeps its w.

Pinned by: agreement with the direct solve; exact interpolation at the nodes
(sigma2 = 0, K w = y reproduces y); termination within n iterations in the
SPD case (exact-arithmetic bound, checked on a small system); the recurrence
residual tracking the true residual b - A w.
"""
from __future__ import annotations

import numpy as np

from . import dense


def system_matrix(X, s, sigma2):
    K = dense.kernel(X, X, s)
    return K + float(sigma2) * np.eye(K.shape[0])


def direct(X, B, s, sigma2):
    return np.linalg.solve(system_matrix(X, s, sigma2), np.asarray(B, np.float64))


def cg(X, B, s, sigma2, tol, max_iter, A=None):
    """Returns (W, iterations, per-column relative residual of the recurrence)."""
    if A is None:
        A = system_matrix(X, s, sigma2)
    B = np.asarray(B, np.float64)
    W = np.zeros_like(B)
    R = B.copy()
    P = R.copy()
    bb = np.einsum("ij,ij->j", B, B)
    rs = bb.copy()
    active = rs > 0
    it = 0
    while active.any() and it < max_iter:
        AP = A @ P
        pap = np.einsum("ij,ij->j", P, AP)
        alpha = np.where(active & (pap > 0), rs / np.where(pap > 0, pap, 1.0), 0.0)
        W += alpha * P
        R -= alpha * AP
        rs_new = np.einsum("ij,ij->j", R, R)
        beta = np.where(active, rs_new / np.where(rs > 0, rs, 1.0), 0.0)
        rs = np.where(active, rs_new, rs)
        active = active & (rs_new > tol * tol * bb)
        P = np.where(active, R + beta * P, 0.0)
        it += 1
    return W, it, np.sqrt(rs / np.where(bb > 0, bb, 1.0))

"""Central finite differences of pair-sum losses in FP64 (TEST INFRASTRUCTURE).

Only tests, the smoke check and the benchmark's CPU legs may use this module.

The adjoints of the pair sums (the reverse-mode derivatives the hot path
computes from the cell list) are checked against derivatives that need no
adjoint at all: the loss is evaluated at perturbed inputs and differenced.
For the Gaussian pair sum of the paper's radius-filtered form (Sec. 3, the
sum over neighbours of a kernel of the separation),

    L = sum_q g_q y_q,   y_q = sum_{j in N(q)} w_j exp(-s |dx_qj|^2),

a particle i's coordinates enter only the terms of y_i and the terms for i in
y_j of its neighbours j, so

    L_i(x_i) = sum_{j in N(i)} (g_i w_j + g_j w_i) exp(-s |x_j - x_i|^2)

holds every term that changes when x_i moves; dL/dx_ik is the central
difference of L_i.  The neighbour set is held fixed (the derivative of the
radius filter is zero almost everywhere), and the separation is the minimum
image chosen by the FP32 rule of the neighbour predicate, then formed in FP64.

Pinned by: agreement with the analytic adjoint of ``oracle.pair_grads`` on
small cases (tests/test_oracle_fd.py), and the finite differences of the
whole loss there.
"""
from __future__ import annotations

import numpy as np


def _image_shift(box, k, xi32, xj32):
    """Shift (-L, 0, +L) the FP32 minimum-image rule adds to x_j - x_i."""
    if not box.periodic[k]:
        return np.zeros(xi32.shape)
    L32 = np.float32(box.hi[k] - box.lo[k])
    half = np.float32(np.float32(0.5) * L32)
    d = (xj32 - xi32).astype(np.float32)
    return np.where(d > half, -float(L32), np.where(d < -half, float(L32), 0.0))


def gauss_position_grad_fd(box, pos, offsets, idx, queries, w, g, s, h=1e-7):
    """dL/dx_i (float64[nq, 3]) for L = sum_q g_q y_q of the Gaussian pair
    sum, by central differences of L_i with step h, for each query i.

    ``offsets, idx``: neighbour CSR of the queries (rows in query order, j
    as original indices).  ``pos``: float32[n, 4]; ``w, g``: float[n]."""
    pos = np.asarray(pos, np.float32)
    q = np.asarray(queries, np.int64)
    offsets = np.asarray(offsets, np.int64)
    idx = np.asarray(idx, np.int64)
    w = np.asarray(w, np.float64)
    g = np.asarray(g, np.float64)
    rows = np.repeat(np.arange(len(q)), np.diff(offsets))
    i = q[rows]
    j = idx
    dx = np.zeros((len(j), 3))
    for k in range(box.dim):
        xi32, xj32 = pos[i, k], pos[j, k]
        dx[:, k] = (xj32.astype(np.float64) - xi32.astype(np.float64)) + \
            _image_shift(box, k, xi32, xj32)
    c = g[i] * w[j] + g[j] * w[i]
    out = np.zeros((len(q), 3))
    for k in range(box.dim):
        lp = np.zeros(len(q))
        lm = np.zeros(len(q))
        dp = dx.copy()
        dp[:, k] -= h          # x_i + h moves x_j - x_i by -h
        dm = dx.copy()
        dm[:, k] += h
        np.add.at(lp, rows, c * np.exp(-s * (dp * dp).sum(1)))
        np.add.at(lm, rows, c * np.exp(-s * (dm * dm).sum(1)))
        out[:, k] = (lp - lm) / (2.0 * h)
    return out

"""Pins of the finite-difference helper (CPU only): it must agree with the
oracle's analytic Gaussian adjoint, and with finite differences of the whole
loss, on small cases with periodic and non-periodic axes."""
import numpy as np
import pytest

import oracle
import synth
from oracle import fd


@pytest.mark.parametrize("dim,periodic", [(3, (1, 1, 1)), (3, (1, 0, 1)), (2, (0, 1))])
def test_fd_matches_analytic_adjoint(dim, periodic):
    pos = synth.uniform_positions(400, dim, 40 + dim)
    box = oracle.Box(dim, periodic[:dim], radius=0.15)
    off, idx = oracle.neighbours_brute(box, pos)
    rng = np.random.default_rng(9)
    w = rng.standard_normal(len(pos))
    g = rng.standard_normal(len(pos))
    s = 1.0 / 0.05 ** 2
    ref, _, _ = oracle.pair_grads("gauss", box, pos, off, idx, g, w=w, params={"s": s})
    den, _, _ = oracle.abs_grad_terms("gauss", box, pos, off, idx, g, w=w, params={"s": s})
    got = fd.gauss_position_grad_fd(box, pos, off, idx, np.arange(len(pos)), w, g, s, h=1e-7)
    err = np.abs(got[:, :dim] - ref[:, :dim]) / np.maximum(den[:, :dim], 1e-300)
    assert err.max() <= 1e-7, err.max()


def test_fd_local_loss_equals_whole_loss_difference():
    """L_i holds every term of L that contains x_i: the whole-loss central
    difference (oracle FP64 evaluation at perturbed positions) agrees."""
    pos = synth.uniform_positions(300, 3, 77)
    box = oracle.Box(3, (1, 1, 1), radius=0.2)
    off, idx = oracle.neighbours_brute(box, pos)
    rng = np.random.default_rng(3)
    w = rng.standard_normal(len(pos))
    g = rng.standard_normal(len(pos))
    s = 100.0
    q = np.array([0, 57, 123, 299])
    offq = np.concatenate([[0], np.cumsum(np.diff(off)[q])])
    idxq = np.concatenate([idx[off[i]:off[i + 1]] for i in q])
    got = fd.gauss_position_grad_fd(box, pos, offq, idxq, q, w, g, s, h=1e-7)
    p64 = pos.astype(np.float64)

    def L(p):
        return float(g @ oracle.pair_values64("gauss", box, p, off, idx, w=w,
                                               params={"s": s})[:, 0])

    for a, i in enumerate(q):
        for k in range(3):
            h = 1e-6
            pp = p64.copy(); pp[i, k] += h
            pm = p64.copy(); pm[i, k] -= h
            whole = (L(pp) - L(pm)) / (2 * h)
            assert abs(whole - got[a, k]) <= 1e-6 * max(abs(whole), 1e-3)

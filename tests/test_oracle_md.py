"""Pins of the oracle's molecular-dynamics step (paper Sec. 3, Eqs. 2-3)."""
import numpy as np

import oracle
import synth
from oracle import md


def _state(xy, v):
    p = synth.pack4(np.asarray(xy, np.float32))
    q = synth.pack4(np.asarray(v, np.float32))
    return p, q


def test_free_flight_and_rest():
    p, v = _state([[0.2, 0.3], [0.5, 0.5]], [[0.0, 0.0], [0.01, -0.02]])
    p1, v1 = md.md_step(p, v, np.zeros((2, 4)), 2, (1, 1), (0, 0), (1, 1), 1.0)
    assert np.array_equal(p1[0], p[0]) and np.array_equal(v1, v)
    assert np.allclose(p1[1, :2], [0.51, 0.48], atol=1e-7)


def test_constant_acceleration_closed_form():
    """Semi-implicit Euler: v_k = k dt a, x_k = x_0 + dt^2 a k (k+1) / 2."""
    a, dt, K = 1e-4, 0.5, 40
    p, v = _state([[0.1, 0.1]], [[0.0, 0.0]])
    acc = np.array([[a, 0.0, 0.0, 0.0]])
    for _ in range(K):
        p, v = md.md_step(p, v, acc, 2, (0, 0), (0, 0), (1, 1), dt)
    assert abs(float(v[0, 0]) - K * dt * a) < 1e-9
    assert abs(float(p[0, 0]) - (0.1 + dt * dt * a * K * (K + 1) / 2)) < 2e-7
    assert float(p[0, 1]) == np.float32(0.1)


def test_wrap_and_reflect_closed_cases():
    p, v = _state([[0.95, 0.95]], [[0.1, 0.1]])
    p1, v1 = md.md_step(p, v, np.zeros((1, 4)), 2, (1, 0), (0, 0), (1, 1), 1.0)
    assert abs(float(p1[0, 0]) - 0.05) < 1e-7 and float(v1[0, 0]) == np.float32(0.1)
    assert abs(float(p1[0, 1]) - 0.95) < 1e-7 and float(v1[0, 1]) == np.float32(-0.1)
    p, v = _state([[0.02, 0.02]], [[-0.05, -0.05]])
    p1, v1 = md.md_step(p, v, np.zeros((1, 4)), 2, (1, 0), (0, 0), (1, 1), 1.0)
    assert abs(float(p1[0, 0]) - 0.97) < 1e-7
    assert abs(float(p1[0, 1]) - 0.03) < 1e-7 and float(v1[0, 1]) == np.float32(0.05)


def test_momentum_conserved_with_pair_forces():
    """EXPF is antisymmetric (f_ij = -f_ji), so sum_i a_i = 0 and the total
    momentum of a periodic system stays at its initial value (here 0)."""
    w = synth.paper_shape(4096)
    box = oracle.Box(2, (1, 1), (0, 0), (1, 1), w.radius)
    pos = w.pos.copy()
    vel = np.zeros_like(pos)
    for _ in range(3):
        off, idx = oracle.neighbours_brute(box, pos)
        F = oracle.pair_values("expf", box, pos, off, idx, params={"c": w.params["c"]})
        assert np.abs(F[:, :2].sum(axis=0)).max() < 1e-12 * np.abs(F[:, :2]).sum()
        pos, vel = md.md_step(pos, vel, F, 2, (1, 1), (0, 0), (1, 1), 1.0)
    # conserved up to the FP32 rounding of the stored velocities (<= |v| 2^-24
    # per particle and step)
    v64 = vel[:, :2].astype(np.float64)
    assert np.abs(v64.sum(axis=0)).max() <= 3 * np.abs(v64).sum() * 2.0 ** -24

"""Pins of the Philox generator, Box-Muller and the Brownian step (CPU)."""
import math

import numpy as np
import pytest

from oracle import brownian, philox

M = np.uint64(0xFFFFFFFFFFFFFFFF)


def _inc(ctr):
    v = sum(int(x) << (64 * i) for i, x in enumerate(ctr))
    v = (v + 1) % (1 << 256)
    return np.array([(v >> (64 * i)) & int(M) for i in range(4)], dtype=np.uint64)


@pytest.mark.parametrize("key", [(0, 0), (5, 7), (2**64 - 1, 3), (1704094, 0)])
@pytest.mark.parametrize("ctr", [(0, 0, 0, 0), (2**64 - 1, 0, 0, 0),
                                 (2**64 - 1, 2**64 - 1, 5, 9), (123, 456, 0, 0)])
def test_philox_matches_numpy_bit_generator(key, ctr):
    """numpy.random.Philox is Philox4x64-10; it advances the counter by one
    before producing a block."""
    key = np.array(key, dtype=np.uint64)
    ctr = np.array(ctr, dtype=np.uint64)
    bg = np.random.Philox(key=key, counter=ctr)
    ref = bg.random_raw(8)
    c1 = _inc(ctr)
    c2 = _inc(c1)
    mine = np.concatenate([philox.philox4x64_10(c1, key), philox.philox4x64_10(c2, key)])
    assert np.array_equal(ref, mine)


def test_philox_vectorised_matches_numpy_many():
    key = np.array([99, 1], dtype=np.uint64)
    ctrs = np.zeros((64, 4), dtype=np.uint64)
    ctrs[:, 0] = np.arange(64, dtype=np.uint64) * np.uint64(7919)
    ctrs[:, 1] = np.uint64(12)
    out = philox.philox4x64_10(ctrs, key)
    for t in range(64):
        prev = ctrs[t].copy()
        prev[0] = prev[0] - np.uint64(1) if prev[0] > 0 else M
        if ctrs[t][0] == 0:
            prev[1] -= np.uint64(1)
        ref = np.random.Philox(key=key, counter=prev).random_raw(4)
        assert np.array_equal(ref, out[t])


def test_box_muller_identities_and_distribution():
    stats = pytest.importorskip("scipy.stats")
    b = philox.particle_block(np.arange(200000), 3, 1704094)
    u1 = philox.uniform24(b[:, 0])
    u2 = philox.uniform24(b[:, 1])
    assert u1.dtype == np.float32 and u1.min() > 0 and u1.max() <= 1
    z0, z1 = philox.box_muller(u1, u2)
    assert np.allclose(z0 ** 2 + z1 ** 2, -2 * np.log(u1.astype(np.float64)), rtol=1e-12, atol=1e-12)
    ang = np.mod(np.arctan2(z1, z0), 2 * np.pi)
    ref = np.mod(2 * np.pi * u2.astype(np.float64), 2 * np.pi)
    dif = np.abs(ang - ref)
    dif = np.minimum(dif, 2 * np.pi - dif)
    assert np.all(dif[np.sqrt(z0**2 + z1**2) > 1e-6] < 1e-9)
    for z in (z0, z1):
        assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 0.01


def test_bd_no_force_no_noise_is_identity():
    pos = np.random.default_rng(0).random((100, 4)).astype(np.float32)
    pos[:, 2:] = 0
    out = brownian.bd_step(pos, np.zeros((100, 4)), 2, (1, 0, 0), (0, 0, 0), (1, 1, 1),
                           1e-5, 0.0, 1, 0)
    assert np.array_equal(out, pos)


def test_bd_reflect_and_wrap_closed_cases():
    pos = np.array([[0.999, 0.001, 0, 0], [0.001, 0.999, 0, 0]], np.float32)
    F = np.array([[0.01, -0.003, 0, 0], [-0.003, 0.002, 0, 0]]) / 1e-1
    out = brownian.bd_step(pos, F, 2, (1, 0, 0), (0, 0, 0), (1, 1, 1), 0.1, 0.0, 1, 0)
    x0 = float(np.float32(0.999)) + 0.01 - 1.0
    y0 = -(float(np.float32(0.001)) - 0.003)
    x1 = float(np.float32(0.001)) - 0.003 + 1.0
    y1 = 2.0 - (float(np.float32(0.999)) + 0.002)
    assert np.allclose(out[:, :2], [[x0, y0], [x1, y1]], rtol=0, atol=1e-7)


def test_bd_free_diffusion_msd():
    """<dx^2> = 2 D t per axis for free particles (no force), over 20 steps."""
    n = 200000
    rng = np.random.default_rng(2)
    pos = np.zeros((n, 4), np.float32)
    pos[:, :2] = 0.25 + 0.5 * rng.random((n, 2)).astype(np.float32)
    D, dt, steps = 1e-2, 1e-5, 20
    p = pos.copy()
    for t in range(steps):
        p = brownian.bd_step(p, np.zeros((n, 4)), 2, (1, 0, 0), (0, 0, 0), (1, 1, 1),
                             dt, D, 1704094, t)
    d = (p[:, :2] - pos[:, :2]).astype(np.float64)
    msd = (d * d).mean(0)
    expect = 2 * D * dt * steps
    assert np.all(np.abs(msd / expect - 1) < 0.02)

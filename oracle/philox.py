"""Philox4x64-10 and Box-Muller in numpy (TEST INFRASTRUCTURE).

Only tests, the smoke check and the benchmark's CPU legs may use this module.

Philox (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11) is a counter-based generator: a keyed bijection of a
4 x 64-bit counter made of 10 rounds.  Each round multiplies two counter
words by fixed odd constants, keeps the high and low halves of the 128-bit
products, XORs the high halves with the other two words and the round key,
and permutes; the 2 x 64-bit key is advanced by two Weyl constants between
rounds.  The Brownian step draws, for particle i at step t, the block
philox(counter = (i, t, 0, 0), key = (seed, 0)).

Pinned by: numpy's own ``numpy.random.Philox`` bit generator (a library
implementation of the same published algorithm), compared word for word on
arbitrary keys and counters, including carries.

Box-Muller (Box & Muller 1958): u1, u2 uniform in (0, 1] give
z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2), two
independent standard normals.  Uniforms are taken from the top 24 bits of a
64-bit word w as u = ((w >> 40) + 1) * 2^-24, exact in FP32.  Pinned by a
Kolmogorov-Smirnov test against scipy's normal CDF and by the identities
z0^2 + z1^2 = -2 ln u1 and atan2(z1, z0) = 2 pi u2 (mod 2 pi).
"""
from __future__ import annotations

import numpy as np

_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)
PHILOX_M0 = np.uint64(0xD2E7470EE14C6C93)
PHILOX_M1 = np.uint64(0xCA5A826395121157)
PHILOX_W0 = np.uint64(0x9E3779B97F4A7C15)
PHILOX_W1 = np.uint64(0xBB67AE8584CAA73B)


def mulhilo64(a, b):
    """(high, low) 64-bit halves of the 128-bit product a*b (uint64 arrays)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a0, a1 = a & _M32, a >> _S32
    b0, b1 = b & _M32, b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _M32) + (p10 & _M32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64_10(ctr, key):
    """Philox4x64 with 10 rounds.

    ctr: uint64[..., 4]; key: uint64[..., 2] (broadcast).  Returns
    uint64[..., 4].
    """
    with np.errstate(over="ignore"):
        c = [np.asarray(ctr, dtype=np.uint64)[..., t].copy() for t in range(4)]
        k0 = np.asarray(key, dtype=np.uint64)[..., 0].copy()
        k1 = np.asarray(key, dtype=np.uint64)[..., 1].copy()
        for rnd in range(10):
            if rnd > 0:
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
            hi0, lo0 = mulhilo64(PHILOX_M0, c[0])
            hi1, lo1 = mulhilo64(PHILOX_M1, c[2])
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        return np.stack(c, axis=-1)


def uniform24(words):
    """u = ((w >> 40) + 1) * 2^-24 in (0, 1], returned as float32 (exact)."""
    k = (np.asarray(words, dtype=np.uint64) >> np.uint64(40)).astype(np.float64)
    return ((k + 1.0) * 2.0 ** -24).astype(np.float32)


def box_muller(u1, u2):
    """Two standard normals from two uniforms in (0,1], evaluated in FP64."""
    u1 = np.asarray(u1, dtype=np.float64)
    u2 = np.asarray(u2, dtype=np.float64)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def particle_block(idx, step, seed):
    """Philox block of particle ``idx`` at ``step`` (uint64[len(idx), 4])."""
    idx = np.asarray(idx, dtype=np.uint64)
    ctr = np.zeros(idx.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = idx
    ctr[..., 1] = np.uint64(step)
    key = np.array([np.uint64(seed), np.uint64(0)], dtype=np.uint64)
    return philox4x64_10(ctr, key)


def particle_normals(idx, step, seed):
    """Three standard normals per particle: (z0, z1) from words 0, 1 and z2
    from words 2, 3 (cosine branch).  Returns float64[len(idx), 3]."""
    b = particle_block(idx, step, seed)
    z0, z1 = box_muller(uniform24(b[..., 0]), uniform24(b[..., 1]))
    z2, _ = box_muller(uniform24(b[..., 2]), uniform24(b[..., 3]))
    return np.stack([z0, z1, z2], axis=-1)

"""One Euler-Maruyama Brownian-dynamics step (TEST INFRASTRUCTURE).

Only tests, the smoke check and the benchmark's CPU legs may use this module.

The paper lists Brownian dynamics among the particle methods it supports
(Sec. 1, Sec. 1.1) and names the fast-moving Brownian case as the reason for
a rebuilt search structure (Sec. 2.2.1).  The step, per axis k of particle i:

    x' = x + dt F_k + sqrt(2 D dt) z_k,    z = Philox/Box-Muller normals,

then on a periodic axis x' is wrapped into [lo, hi) (x' -= L floor((x'-lo)/L),
and a value that equals hi after rounding to FP32 becomes lo); on a
non-periodic axis it is reflected once at the walls (x' < lo -> 2 lo - x',
x' > hi -> 2 hi - x').  Evaluated in FP64 from FP32 inputs and rounded to
FP32 at the end.

Pinned by: closed cases (no force and no noise leaves x unchanged; a
particle pushed across a wall is reflected to the mirror point; across a
periodic face it re-enters on the other side), and the diffusion law
<dx^2> = 2 D t per axis over many free particles.  Trajectory-level parity
over many steps is unpinned: trajectories of interacting particles diverge.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox


def bd_step(pos, force, dim, periodic, lo, hi, dt, D, seed, step,
            noise=None):
    """Return the next float32[n,4] positions (pad copied through)."""
    pos = np.asarray(pos, dtype=np.float32)
    F = np.asarray(force, dtype=np.float64)
    n = pos.shape[0]
    if noise is None:
        noise = philox.particle_normals(np.arange(n), step, seed)
    amp = math.sqrt(2.0 * D * dt)
    out = pos.copy()
    for k in range(dim):
        x = pos[:, k].astype(np.float64) + dt * F[:, k] + amp * noise[:, k]
        l, h = float(np.float32(lo[k])), float(np.float32(hi[k]))
        L = h - l
        if periodic[k]:
            x = x - L * np.floor((x - l) / L)
            x32 = x.astype(np.float32)
            x32[x32 >= np.float32(h)] = np.float32(l)
        else:
            x = np.where(x < l, 2 * l - x, x)
            x = np.where(x > h, 2 * h - x, x)
            x32 = x.astype(np.float32)
        out[:, k] = x32
    return out

"""Semi-implicit Euler step of the paper's molecular-dynamics example
(TEST INFRASTRUCTURE).

Only tests, the smoke check and the benchmark's CPU legs may use this module.

The paper's worked example (Sec. 3) evolves velocities and positions with
accelerations a_i = sum_j f_ij (the exponential force of Eq. 1) by a
semi-implicit Euler step with dt = 1 (Eqs. 2-3): first v_i += a_i, then
r_i += v_i with the new velocity.  Generalised to a step dt:

    v' = v + dt a,    x' = x + dt v'.

On a periodic axis x' is wrapped into [lo, hi) (x' -= L floor((x'-lo)/L), and
a value equal to hi after rounding to FP32 becomes lo); on a non-periodic
axis a particle past a wall is reflected once (x' < lo -> 2 lo - x',
x' > hi -> 2 hi - x') and that velocity component reversed.  Evaluated in
FP64 from FP32 inputs and rounded to FP32 at the end.

Pinned by: closed forms (free flight; constant acceleration gives
v_k = k dt a and x_k = x_0 + dt^2 a k (k+1)/2 after k steps), the wrap and
reflection closed cases, and conservation of total momentum when the
accelerations are an antisymmetric pair sum (Newton's third law).
"""
from __future__ import annotations

import numpy as np


def md_step(pos, vel, acc, dim, periodic, lo, hi, dt):
    """Return (pos', vel') as float32[n,4] (fourth component copied)."""
    pos = np.asarray(pos, dtype=np.float32)
    vel = np.asarray(vel, dtype=np.float32)
    A = np.asarray(acc, dtype=np.float64)
    out_p, out_v = pos.copy(), vel.copy()
    for k in range(dim):
        v = vel[:, k].astype(np.float64) + dt * A[:, k]          # Eq. 2
        x = pos[:, k].astype(np.float64) + dt * v                 # Eq. 3
        l, h = float(np.float32(lo[k])), float(np.float32(hi[k]))
        L = h - l
        if periodic[k]:
            x = x - L * np.floor((x - l) / L)
            x32 = x.astype(np.float32)
            x32[x32 >= np.float32(h)] = np.float32(l)
        else:
            below, above = x < l, x > h
            x = np.where(below, 2 * l - x, x)
            v = np.where(below, -v, v)
            above = x > h
            x = np.where(above, 2 * h - x, x)
            v = np.where(above, -v, v)
            x32 = x.astype(np.float32)
        out_p[:, k] = x32
        out_v[:, k] = v.astype(np.float32)
    return out_p, out_v

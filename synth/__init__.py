"""Seeded synthetic inputs shaped like the paper's particle workloads.

This module only draws random numbers and lays them out; it contains none of
the method's arithmetic (no cells, distances, kernels or sums), so both the
CUDA path and the CPU oracle may consume what it produces.

Positions follow the paper's illustrative example (Sec. 3): points drawn
uniformly in the unit hypercube, every axis periodic.  They are drawn in FP64
with ``numpy.random.Generator(PCG64(seed))`` and rounded to FP32; a coordinate
that rounds up to the upper bound 1.0 is folded to 0.0 so every coordinate lies
in ``[0, 1)``.  Positions are packed as ``float32[n, 4]`` with the unused
components zero (``z`` for 2-D, and the pad).

Workloads (the radius, operator parameters and sizes):

* ``c1``: d=2, N=4096, uniform, both axes periodic, r=0.03, w~U(-1,1),
  Gaussian width h=0.01 (s=1/h^2).
* ``c2``: d=3, N=2^20, uniform periodic cube, r=0.0197, truncated
  Lennard-Jones with sigma=0.01, eps=1.
* ``c3``: d=3, N=2^24, 1024 Gaussian blobs (centres uniform, sd 0.01, equal
  weight) wrapped into the periodic cube, w~N(0,1), Gaussian pair kernel with
  h=r/3, r chosen for 64 neighbours mean.
* ``c4``: dense kernel operator, X and Y each 65,536 points uniform in
  [0,1]^3, W~N(0,1) with 64 columns, lengthscale 0.1.
* ``c5``: d=2 Brownian dynamics, N=2^22 uniform in the unit square, x periodic,
  y reflecting, soft repulsion within r=0.002, dt=1e-5.
* ``paper``: the shape of the paper's benchmark (Sec. 3, Fig. 3 left): d=2
  periodic unit square, r=sqrt(3/N), exponential force with c=1e-3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1704089

# Radius giving 64 neighbours mean for the clustered 16.7M-point workload.
# Found by bisection on the oracle's neighbour counts of a 65,536-point query
# sample against all points (script: tests/golden/make_c3_radius.py, output
# tests/golden/c3_radius.json).  Stored here as a plain number so that this
# module carries no neighbour arithmetic.
C3_RADIUS = 0.0034309213515371084


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _to_f32_unit(x64: np.ndarray) -> np.ndarray:
    """Round FP64 coordinates in [0,1) to FP32, folding 1.0 back to 0.0."""
    x = x64.astype(np.float32)
    x[x >= np.float32(1.0)] = np.float32(0.0)
    return x


def pack4(coords: np.ndarray) -> np.ndarray:
    """Pack ``[n, d]`` FP32 coordinates into ``float32[n, 4]`` (zero pad)."""
    n, d = coords.shape
    out = np.zeros((n, 4), dtype=np.float32)
    out[:, :d] = coords
    return out


def uniform_positions(n: int, dim: int, seed: int) -> np.ndarray:
    """``float32[n,4]`` positions uniform in the unit hypercube."""
    g = _rng(seed)
    return pack4(_to_f32_unit(g.random((n, dim))))


def blob_positions(n: int, n_blobs: int, sd: float, seed: int) -> np.ndarray:
    """Equal-weight Gaussian blobs with uniform centres, wrapped mod 1 (3-D)."""
    g = _rng(seed)
    centres = g.random((n_blobs, 3))
    per = n // n_blobs
    assert per * n_blobs == n
    pts = np.repeat(centres, per, axis=0) + sd * g.standard_normal((n, 3))
    pts -= np.floor(pts)
    return pack4(_to_f32_unit(pts))


@dataclass
class PairWorkload:
    name: str
    dim: int
    n: int
    pos: np.ndarray                  # float32[n,4]
    periodic: tuple = (1, 1, 1)
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    radius: float = 0.0
    op: str = "count"
    params: dict = field(default_factory=dict)
    w: np.ndarray | None = None      # float32[n] per-particle weight
    g: np.ndarray | None = None      # float32[n] upstream gradient (adjoint tests)


def c1(seed_offset: int = 0) -> PairWorkload:
    """2-D, N=4096, r=0.03, count + Gaussian sum (h=0.01)."""
    seed = BASE_SEED + 1 + seed_offset
    n = 4096
    pos = uniform_positions(n, 2, seed)
    w = _rng(seed + 100).uniform(-1.0, 1.0, n).astype(np.float32)
    return PairWorkload("c1", 2, n, pos, (1, 1, 0), radius=0.03, op="gauss",
                        params={"s": 1.0 / (0.01 ** 2)}, w=w)


def c2(n: int = 1 << 20, seed_offset: int = 0) -> PairWorkload:
    """3-D uniform periodic cube, r=0.0197, truncated Lennard-Jones."""
    seed = BASE_SEED + 2 + seed_offset
    pos = uniform_positions(n, 3, seed)
    g = _rng(seed + 100).uniform(0.5, 1.5, n).astype(np.float32)
    return PairWorkload("c2", 3, n, pos, (1, 1, 1), radius=0.0197, op="lj",
                        params={"eps": 1.0, "sigma": 0.01}, g=g)


def c3(n: int = 1 << 24, n_blobs: int = 1024, seed_offset: int = 0,
       radius: float | None = None) -> PairWorkload:
    """3-D clustered: Gaussian blobs (sd 0.01) in the periodic cube."""
    seed = BASE_SEED + 3 + seed_offset
    pos = blob_positions(n, n_blobs, 0.01, seed)
    r = C3_RADIUS if radius is None else radius
    w = _rng(seed + 100).standard_normal(n).astype(np.float32)
    g = _rng(seed + 200).standard_normal(n).astype(np.float32)
    return PairWorkload("c3", 3, n, pos, (1, 1, 1), radius=r, op="gauss",
                        params={"s": 1.0 / (r / 3.0) ** 2}, w=w, g=g)


@dataclass
class DenseWorkload:
    name: str
    X: np.ndarray      # float32[m,3]
    Y: np.ndarray      # float32[n,3]
    W: np.ndarray      # float32[n,nrhs]
    G: np.ndarray      # float32[m,nrhs]  upstream gradient
    lengthscale: float

    @property
    def s(self) -> float:
        # squared-exponential convention exp(-d^2 / (2 l^2))
        return 1.0 / (2.0 * self.lengthscale ** 2)


def c4(m: int = 65536, n: int = 65536, nrhs: int = 64, seed_offset: int = 0,
       lengthscale: float = 0.1) -> DenseWorkload:
    seed = BASE_SEED + 4 + seed_offset
    g = _rng(seed)
    X = g.random((m, 3)).astype(np.float32)
    Y = g.random((n, 3)).astype(np.float32)
    W = g.standard_normal((n, nrhs)).astype(np.float32)
    G = g.standard_normal((m, nrhs)).astype(np.float32)
    return DenseWorkload("c4", X, Y, W, G, lengthscale)


def c5(n: int = 1 << 22, seed_offset: int = 0) -> PairWorkload:
    """2-D Brownian dynamics: x periodic, y reflecting, soft repulsion."""
    seed = BASE_SEED + 5 + seed_offset
    pos = uniform_positions(n, 2, seed)
    return PairWorkload("c5", 2, n, pos, (1, 0, 0), radius=0.002, op="soft",
                        params={"k": 1.0e4, "dt": 1.0e-5, "D": 1.0e-2,
                                "seed": seed})


def paper_shape(n: int, seed_offset: int = 0) -> PairWorkload:
    """The paper's benchmark shape: 2-D periodic, r=sqrt(3/N), exp force."""
    seed = BASE_SEED + 6 + seed_offset
    pos = uniform_positions(n, 2, seed)
    return PairWorkload("paper", 2, n, pos, (1, 1, 0), radius=math.sqrt(3.0 / n),
                        op="expf", params={"c": 1.0e-3})


def weights(n: int, seed: int, kind: str = "uniform") -> np.ndarray:
    g = _rng(seed)
    if kind == "uniform":
        return g.uniform(-1.0, 1.0, n).astype(np.float32)
    return g.standard_normal(n).astype(np.float32)


def query_sample(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct particle indices (sorted int64) drawn without replacement."""
    g = _rng(seed)
    return np.sort(g.choice(n, size=min(k, n), replace=False)).astype(np.int64)

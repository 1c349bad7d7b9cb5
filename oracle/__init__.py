"""CPU oracle for the particle pair sum and the dense kernel operator.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call, link or execute anything under ``oracle/``.  It shares no code with the
CUDA library and never imports it.

Contents
--------
* ``oracle.c`` (loaded here through ctypes): the FP32 neighbour predicate,
  an O(N) brute-force search, an independent linked-list cell list, and the
  pair operators and their adjoints in FP64 (paper Sec. 1 problem statement,
  Sec. 2.2.1-2.2.2, Sec. 3 Eq. 1).
* ``dense.py``: the dense kernel operator ``Y = K(X,Y) W`` and its adjoint in
  FP64 numpy (RBF / Gaussian-process examples, Sec. 1.1).
* ``philox.py``: the Philox4x64-10 counter-based generator (Salmon et al.,
  SC'11) and the Box-Muller transform.
* ``brownian.py``: one Euler-Maruyama step with periodic / reflecting axes.

Parity status of each function is listed in the module docstrings
("pinned by ..." or "parity unpinned").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
          "-fno-fast-math", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or \
            os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            F = ctypes.c_float
            box = [I, P, P, P, F]
            lib.or_brute_counts.argtypes = box + [I64, P, I64, P, P]
            lib.or_brute_list.argtypes = box + [I64, P, I64, P, P, P]
            lib.or_cells_build.argtypes = box + [I64, P]
            lib.or_cells_build.restype = P
            lib.or_cells_free.argtypes = [P]
            lib.or_cells_shape.argtypes = [P, P]
            lib.or_cells_counts.argtypes = [P, I64, P, P]
            lib.or_cells_list.argtypes = [P, I64, P, P, P]
            lib.or_pair_eval.argtypes = [I, I, P, I, P, P, P, I64, P, P, I64,
                                         P, P, P, P]
            lib.or_pair_grad.argtypes = [I, I, P, I, P, P, P, I64, P, P, P,
                                         I64, P, P, P, P, P, P]
            lib.or_num_threads.restype = I
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().or_num_threads())


OPS = {"count": 0, "gauss": 1, "lj": 2, "expf": 3, "soft": 4, "sph_density": 5,
       "sph_force": 6}


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Box:
    """Box ``[lo, hi)`` in ``dim`` dimensions with per-axis periodicity."""

    def __init__(self, dim, periodic, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                 radius=0.0):
        self.dim = int(dim)
        self.periodic = np.ascontiguousarray(
            [int(bool(p)) for p in (list(periodic) + [0, 0, 0])[:3]], np.int32)
        self.lo = np.ascontiguousarray((list(lo) + [0, 0, 0])[:3], np.float32)
        self.hi = np.ascontiguousarray((list(hi) + [1, 1, 1])[:3], np.float32)
        self.radius = float(np.float32(radius))

    def args(self):
        return (self.dim, _ptr(self.periodic), _ptr(self.lo), _ptr(self.hi),
                ctypes.c_float(self.radius))


def _pos32(pos):
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    assert pos.ndim == 2 and pos.shape[1] == 4, "positions are float32[n,4]"
    return pos


def _queries(n, queries):
    if queries is None:
        return np.arange(n, dtype=np.int64)
    return np.ascontiguousarray(queries, dtype=np.int64)


def _csr(counts):
    offsets = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return offsets


def neighbours_brute(box: Box, pos, queries=None):
    """Neighbour CSR of each query by the plain definition (O(N) per query).

    Returns ``(offsets int64[nq+1], idx int32[nnz])``; rows ascending in j.
    """
    lib = _load()
    pos = _pos32(pos)
    n = pos.shape[0]
    q = _queries(n, queries)
    counts = np.zeros(len(q), dtype=np.int64)
    lib.or_brute_counts(*box.args(), n, _ptr(pos), len(q), _ptr(q), _ptr(counts))
    offsets = _csr(counts)
    idx = np.zeros(int(offsets[-1]), dtype=np.int32)
    lib.or_brute_list(*box.args(), n, _ptr(pos), len(q), _ptr(q), _ptr(offsets),
                      _ptr(idx))
    return offsets, idx


class CellList:
    """The oracle's own linked-list cell list (FP64 cell index)."""

    def __init__(self, box: Box, pos):
        self._lib = _load()
        self.box = box
        self.pos = _pos32(pos)          # kept alive: the C side borrows it
        self.n = self.pos.shape[0]
        self._h = self._lib.or_cells_build(*box.args(), self.n, _ptr(self.pos))
        if not self._h:
            raise MemoryError("oracle cell list allocation failed")

    def shape(self):
        out = np.zeros(3, dtype=np.int32)
        self._lib.or_cells_shape(self._h, _ptr(out))
        return tuple(int(v) for v in out)

    def counts(self, queries=None):
        q = _queries(self.n, queries)
        counts = np.zeros(len(q), dtype=np.int64)
        self._lib.or_cells_counts(self._h, len(q), _ptr(q), _ptr(counts))
        return counts

    def neighbours(self, queries=None):
        q = _queries(self.n, queries)
        offsets = _csr(self.counts(q))
        idx = np.zeros(int(offsets[-1]), dtype=np.int32)
        self._lib.or_cells_list(self._h, len(q), _ptr(q), _ptr(offsets), _ptr(idx))
        return offsets, idx

    def close(self):
        if self._h:
            self._lib.or_cells_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _params(params, radius):
    p = dict(params or {})
    return np.ascontiguousarray(
        [p.get("s", 0.0), p.get("eps", 1.0), p.get("sigma", 1.0),
         p.get("c", 1.0), p.get("k", 1.0), radius], np.float64)


def _eval(op, absmode, box, pos64, offsets, idx, queries, w, params):
    lib = _load()
    n = pos64.shape[0]
    q = _queries(n, queries)
    w64 = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    if OPS[op] in (1, 5, 6) and w64 is None:
        raise ValueError(f"{op} needs per-particle values w")
    if OPS[op] == 6 and (w64.ndim != 2 or w64.shape[1] != 2):
        raise ValueError("sph_force needs w = (m, P/rho^2) as float[n, 2]")
    out = np.zeros((len(q), 4), dtype=np.float64)
    prm = _params(params, box.radius)
    lib.or_pair_eval(OPS[op], absmode, _ptr(prm), box.dim, _ptr(box.periodic),
                     _ptr(box.lo), _ptr(box.hi), n, _ptr(pos64), _ptr(w64),
                     len(q), _ptr(q), _ptr(np.ascontiguousarray(offsets, np.int64)),
                     _ptr(np.ascontiguousarray(idx, np.int32)), _ptr(out))
    return out


def _grad(op, absmode, box, pos64, offsets, idx, g, queries, w, params):
    lib = _load()
    n = pos64.shape[0]
    q = _queries(n, queries)
    g64 = np.ascontiguousarray(g, dtype=np.float64)
    w64 = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros((len(q), 4), dtype=np.float64)
    gw = gs = None
    if OPS[op] == 1:
        if w64 is None:
            raise ValueError("gauss needs weights")
        gw = np.zeros(len(q), dtype=np.float64)
        gs = np.zeros(len(q), dtype=np.float64)
    elif OPS[op] != 2:
        raise ValueError(f"no adjoint for {op}")
    prm = _params(params, box.radius)
    lib.or_pair_grad(OPS[op], absmode, _ptr(prm), box.dim, _ptr(box.periodic),
                     _ptr(box.lo), _ptr(box.hi), n, _ptr(pos64), _ptr(w64),
                     _ptr(g64), len(q), _ptr(q),
                     _ptr(np.ascontiguousarray(offsets, np.int64)),
                     _ptr(np.ascontiguousarray(idx, np.int32)), _ptr(out),
                     _ptr(gw), _ptr(gs))
    return out, gw, gs


def pair_values(op, box: Box, pos, offsets, idx, queries=None, w=None,
                params=None):
    """FP64 pair sums over a neighbour CSR; returns ``float64[nq,4]``.

    Scalar operators (count, gauss, lj) use column 0; the force operators
    (expf = paper Eq. 1, soft) fill the first ``dim`` columns.
    """
    return _eval(op, 0, box, np.ascontiguousarray(_pos32(pos), np.float64),
                 offsets, idx, queries, w, params)


def pair_values64(op, box: Box, pos64, offsets, idx, queries=None, w=None,
                  params=None):
    """As :func:`pair_values` but from FP64 positions over a fixed CSR."""
    return _eval(op, 0, box, np.ascontiguousarray(pos64, np.float64), offsets,
                 idx, queries, w, params)


def pair_grads(op, box: Box, pos, offsets, idx, g, queries=None, w=None,
               params=None, pos64=None):
    """FP64 adjoint of a pair sum for upstream gradient ``g``.

    Returns ``(dpos float64[nq,4], dw float64[nq] or None, ds_part float64[nq]
    or None)``; ``ds = ds_part.sum()`` over all particles.  ``pos64`` may give
    FP64 positions (finite-difference tests); the neighbour CSR is then taken
    as fixed.
    """
    p64 = (np.ascontiguousarray(_pos32(pos), np.float64) if pos64 is None
           else np.ascontiguousarray(pos64, np.float64))
    return _grad(op, 0, box, p64, offsets, idx, g, queries, w, params)


def abs_terms(op, box: Box, pos, offsets, idx, queries=None, w=None,
              params=None):
    """Per-query sum of |term| for a forward pair sum: ``float64[nq,4]``.

    This is the denominator of the pair-sum error metric
    ``|y - y_ref| / max(|y_ref|, sum |t|)``.
    """
    return _eval(op, 1, box, np.ascontiguousarray(_pos32(pos), np.float64),
                 offsets, idx, queries, w, params)


def abs_grad_terms(op, box: Box, pos, offsets, idx, g, queries=None, w=None,
                   params=None):
    """Per-query sums of |term| for the adjoint (same layout as pair_grads)."""
    return _grad(op, 1, box, np.ascontiguousarray(_pos32(pos), np.float64),
                 offsets, idx, g, queries, w, params)

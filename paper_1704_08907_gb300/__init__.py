"""GB300 (sm_103a) particle-interaction library after arXiv:1704.08907.

Thin Python binding of the C ABI in ``include/aboria_gpu.h``: the functions
below carry the C names and only marshal torch tensors into device pointers.
Every step of the computation runs in the CUDA library; importing this
package without the built library raises ``ImportError`` (no CPU fallback).

Paper map: cell-list build (Sec. 2.2.1), box search and radius-filtered
pair sums (Sec. 2.2.2, Sec. 3 Eq. 1), dense kernel operators for RBF / GP
(Sec. 1.1), Brownian dynamics (Sec. 1).
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi
from ._abi import (AB_OP_COUNT, AB_OP_EXPF, AB_OP_GAUSS, AB_OP_LJ,  # noqa: F401
                   AB_OP_SOFT, AB_OP_SPH_DENSITY, AB_OP_SPH_FORCE, AB_PREC_BF16, AB_PREC_BF16X3, AB_PREC_FP32,
                   AB_PREC_TF32, AB_PREC_TF32X3)

_lib = _abi.load()

OPS = {"count": AB_OP_COUNT, "gauss": AB_OP_GAUSS, "lj": AB_OP_LJ,
       "expf": AB_OP_EXPF, "soft": AB_OP_SOFT, "sph_density": AB_OP_SPH_DENSITY,
       "sph_force": AB_OP_SPH_FORCE}
PRECS = {"fp32": AB_PREC_FP32, "tf32x3": AB_PREC_TF32X3, "bf16x3": AB_PREC_BF16X3,
         "tf32": AB_PREC_TF32, "bf16": AB_PREC_BF16}


def lib_path() -> str:
    return _abi.LIB_PATH


class AbError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        msg = _lib.ab_status_string(status).decode()
        super().__init__(f"{msg} (status {status})" + (f": {detail}" if detail else ""))


def _check(status: int, ctx: "Context | None" = None):
    if status != _abi.AB_OK:
        detail = _lib.ab_last_error(ctx.handle).decode() if ctx is not None else ""
        raise AbError(status, detail)


def Domain(dim, periodic, radius, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> _abi.ab_domain:
    """The hypercube [lo, hi) with per-axis periodicity and cut-off radius."""
    d = _abi.ab_domain()
    d.dim = int(dim)
    per = (list(periodic) + [0, 0, 0])[:3]
    lo = (list(lo) + [0.0, 0.0, 0.0])[:3]
    hi = (list(hi) + [1.0, 1.0, 1.0])[:3]
    for k in range(3):
        d.periodic[k] = int(bool(per[k]))
        d.lo[k] = float(lo[k])
        d.hi[k] = float(hi[k])
    d.radius = float(radius)
    return d


def OpParams(s=0.0, eps=1.0, sigma=1.0, c=1.0, k=1.0) -> _abi.ab_op_params:
    p = _abi.ab_op_params()
    p.s, p.eps, p.sigma, p.c, p.k = float(s), float(eps), float(sigma), float(c), float(k)
    return p


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, shape_tail=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape [n, {shape_tail}]")
    return t


class Context:
    """Owns an ``ab_ctx`` (workspace, cell list) on one device."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        _check(_lib.ab_create(ctypes.byref(h), int(device), ctypes.c_void_p(s)))
        self.handle = h
        self.n = 0
        self.dim = 0
        self.build_seq = 0

    def _stream(self):
        _lib.ab_set_stream(self.handle, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def close(self):
        if getattr(self, "handle", None):
            _lib.ab_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ab_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def ab_destroy(ctx: Context):
    ctx.close()


def ab_sync(ctx: Context):
    _check(_lib.ab_sync(ctx.handle), ctx)


def ab_build(ctx: Context, dom: _abi.ab_domain, pos4: torch.Tensor):
    """Cell-list build (hash, scan, stable scatter) of ``pos4`` float32[n,4],
    or of positions packed as float32[n,dim] (``ab_build_packed``)."""
    if pos4.dim() == 2 and pos4.shape[1] == dom.dim:
        pos = _dev(pos4, torch.float32, (dom.dim,), "pos")
        ctx._stream()
        _check(_lib.ab_build_packed(ctx.handle, ctypes.byref(dom), pos.shape[0], _ptr(pos)), ctx)
    else:
        pos4 = _dev(pos4, torch.float32, (4,), "pos4")
        ctx._stream()
        _check(_lib.ab_build(ctx.handle, ctypes.byref(dom), pos4.shape[0], _ptr(pos4)), ctx)
    ctx.n = pos4.shape[0]
    ctx.dim = dom.dim
    ctx.build_seq += 1
    return ctx.build_seq


def ab_cell_shape(ctx: Context, with_reach: bool = False):
    """(cells per axis, total cells[, stencil reach per axis])."""
    nc = (ctypes.c_int32 * 3)()
    reach = (ctypes.c_int32 * 3)()
    tot = ctypes.c_int64()
    _check(_lib.ab_cell_shape(ctx.handle, nc, ctypes.byref(tot), reach), ctx)
    if with_reach:
        return tuple(nc), tot.value, tuple(reach)
    return tuple(nc), tot.value


def ab_cell_export(ctx: Context):
    """(perm uint32 as int32[n], cell_start int32[n_cells+1]) on the device."""
    _, tot = ab_cell_shape(ctx)
    perm = torch.empty(ctx.n, dtype=torch.int32, device=ctx.device)
    start = torch.empty(tot + 1, dtype=torch.int32, device=ctx.device)
    ctx._stream()
    _check(_lib.ab_cell_export(ctx.handle, _ptr(perm), _ptr(start)), ctx)
    return perm, start


def ab_pair_sum(ctx: Context, op, params, w=None, out=None, energy=None):
    """Pair sum over the last cell list; returns ``out`` (allocated if None)."""
    op = OPS.get(op, op)
    vec = op in (AB_OP_EXPF, AB_OP_SOFT, AB_OP_SPH_FORCE)
    if out is None:
        shape = (ctx.n, 4) if vec else (ctx.n,)
        out = torch.empty(shape, dtype=torch.float32, device=ctx.device)
    _dev(out, torch.float32, None, "out")
    _dev(w, torch.float32, None, "w")
    _dev(energy, torch.float64, None, "energy")
    ctx._stream()
    _check(_lib.ab_pair_sum(ctx.handle, op, ctypes.byref(params), _ptr(w), _ptr(out),
                            _ptr(energy)), ctx)
    return out


def ab_pair_sum_bwd(ctx: Context, op, params, w, grad_out, grad_pos4=None, grad_w=None,
                    grad_s=None):
    op = OPS.get(op, op)
    for t, nm, dt in [(w, "w", torch.float32), (grad_out, "grad_out", torch.float32),
                      (grad_pos4, "grad_pos4", torch.float32), (grad_w, "grad_w", torch.float32),
                      (grad_s, "grad_s", torch.float64)]:
        _dev(t, dt, None, nm)
    ctx._stream()
    _check(_lib.ab_pair_sum_bwd(ctx.handle, op, ctypes.byref(params), _ptr(w), _ptr(grad_out),
                                _ptr(grad_pos4), _ptr(grad_w), _ptr(grad_s)), ctx)
    return grad_pos4, grad_w, grad_s


def ab_pair_sum_value_grad(ctx: Context, op, params, w, grad_out, out=None, energy=None,
                           grad_pos4=None, grad_w=None, grad_s=None):
    """Forward values and the adjoint for upstream gradient grad_out in one
    walk (GAUSS, LJ); outputs as ab_pair_sum and ab_pair_sum_bwd."""
    op = OPS.get(op, op)
    for t, nm, dt in [(w, "w", torch.float32), (grad_out, "grad_out", torch.float32),
                      (out, "out", torch.float32), (energy, "energy", torch.float64),
                      (grad_pos4, "grad_pos4", torch.float32), (grad_w, "grad_w", torch.float32),
                      (grad_s, "grad_s", torch.float64)]:
        _dev(t, dt, None, nm)
    ctx._stream()
    _check(_lib.ab_pair_sum_value_grad(ctx.handle, op, ctypes.byref(params), _ptr(w),
                                       _ptr(grad_out), _ptr(out), _ptr(energy), _ptr(grad_pos4),
                                       _ptr(grad_w), _ptr(grad_s)), ctx)
    return out, energy, grad_pos4, grad_w, grad_s


def ab_pair_energy_grad(ctx: Context, op, params, E=None, grad_pos4=None, energy=None):
    """Energy and the gradient of the total energy in one walk (LJ):
    returns (E float32[n], dE_total/dx float32[n,4], total energy float64)."""
    op = OPS.get(op, op)
    if E is None:
        E = torch.empty(ctx.n, dtype=torch.float32, device=ctx.device)
    if grad_pos4 is None:
        grad_pos4 = torch.empty((ctx.n, 4), dtype=torch.float32, device=ctx.device)
    if energy is None:
        energy = torch.empty((), dtype=torch.float64, device=ctx.device)
    _dev(E, torch.float32, None, "E")
    _dev(grad_pos4, torch.float32, (4,), "grad_pos4")
    _dev(energy, torch.float64, None, "energy")
    ctx._stream()
    _check(_lib.ab_pair_energy_grad(ctx.handle, op, ctypes.byref(params), _ptr(E), _ptr(grad_pos4),
                                    _ptr(energy)), ctx)
    return E, grad_pos4, energy


def ab_pair_energy_grad_packed(ctx: Context, op, params, E=None, grad_pos=None, energy=None):
    """ab_pair_energy_grad with the gradient as float32[n, dim]."""
    op = OPS.get(op, op)
    if E is None:
        E = torch.empty(ctx.n, dtype=torch.float32, device=ctx.device)
    if grad_pos is None:
        grad_pos = torch.empty((ctx.n, ctx.dim), dtype=torch.float32, device=ctx.device)
    if energy is None:
        energy = torch.empty((), dtype=torch.float64, device=ctx.device)
    _dev(E, torch.float32, None, "E")
    _dev(grad_pos, torch.float32, (ctx.dim,), "grad_pos")
    _dev(energy, torch.float64, None, "energy")
    ctx._stream()
    _check(_lib.ab_pair_energy_grad_packed(ctx.handle, op, ctypes.byref(params), _ptr(E),
                                           _ptr(grad_pos), _ptr(energy)), ctx)
    return E, grad_pos, energy


def ab_pair_list(ctx: Context, cap: int | None = None):
    """Neighbour CSR (offsets int64[n+1], idx int32[nnz]) in caller order."""
    offsets = torch.empty(ctx.n + 1, dtype=torch.int64, device=ctx.device)
    nnz = ctypes.c_int64()
    ctx._stream()
    if cap is None:
        st = _lib.ab_pair_list(ctx.handle, _ptr(offsets), None, 0, ctypes.byref(nnz))
        if st not in (_abi.AB_OK, _abi.AB_ERR_CAPACITY):
            _check(st, ctx)
        cap = nnz.value
    idx = torch.empty(max(cap, 1), dtype=torch.int32, device=ctx.device)
    _check(_lib.ab_pair_list(ctx.handle, _ptr(offsets), _ptr(idx), cap, ctypes.byref(nnz)), ctx)
    return offsets, idx[:nnz.value]


def ab_kernel_matvec(ctx: Context, X, Y, W, s, prec="fp32", out=None):
    prec = PRECS.get(prec, prec)
    _dev(X, torch.float32, (4,), "X")
    _dev(Y, torch.float32, (4,), "Y")
    _dev(W, torch.float32, None, "W")
    m, n, nrhs = X.shape[0], Y.shape[0], W.shape[1]
    if out is None:
        out = torch.empty((m, nrhs), dtype=torch.float32, device=ctx.device)
    _dev(out, torch.float32, None, "out")
    ctx._stream()
    _check(_lib.ab_kernel_matvec(ctx.handle, m, n, _ptr(X), _ptr(Y), nrhs, _ptr(W),
                                 float(s), prec, _ptr(out)), ctx)
    return out


def ab_kernel_matvec_bwd(ctx: Context, X, Y, W, s, prec, G, dW=None, dX=None, dY=None,
                         ds=None):
    prec = PRECS.get(prec, prec)
    m, n, nrhs = X.shape[0], Y.shape[0], W.shape[1]
    for t, nm, dt in [(X, "X", torch.float32), (Y, "Y", torch.float32),
                      (W, "W", torch.float32), (G, "G", torch.float32),
                      (dW, "dW", torch.float32), (dX, "dX", torch.float32),
                      (dY, "dY", torch.float32), (ds, "ds", torch.float64)]:
        _dev(t, dt, None, nm)
    ctx._stream()
    _check(_lib.ab_kernel_matvec_bwd(ctx.handle, m, n, _ptr(X), _ptr(Y), nrhs, _ptr(W),
                                     float(s), prec, _ptr(G), _ptr(dW), _ptr(dX), _ptr(dY),
                                     _ptr(ds)), ctx)
    return dW, dX, dY, ds


def ab_kernel_solve(ctx: Context, X, B, s, sigma2, prec="fp32", tol=1e-5, max_iter=1000,
                    W=None):
    """Solve (K(X, X) + sigma2 I) W = B by conjugate gradients (Sec. 1.1).
    Returns (W, iterations, largest relative residual)."""
    prec = PRECS.get(prec, prec)
    _dev(X, torch.float32, (4,), "X")
    _dev(B, torch.float32, None, "B")
    n, nrhs = X.shape[0], B.shape[1]
    if W is None:
        W = torch.empty((n, nrhs), dtype=torch.float32, device=ctx.device)
    _dev(W, torch.float32, None, "W")
    it = ctypes.c_int32()
    rr = ctypes.c_float()
    ctx._stream()
    _check(_lib.ab_kernel_solve(ctx.handle, n, _ptr(X), nrhs, _ptr(B), float(s), float(sigma2),
                                prec, float(tol), int(max_iter), _ptr(W), ctypes.byref(it),
                                ctypes.byref(rr)), ctx)
    return W, it.value, rr.value


def ab_bd_step(ctx: Context, dom, pos4, force4, dt, D, seed, step):
    _dev(pos4, torch.float32, (4,), "pos4")
    _dev(force4, torch.float32, (4,), "force4")
    ctx._stream()
    _check(_lib.ab_bd_step(ctx.handle, ctypes.byref(dom), pos4.shape[0], _ptr(pos4),
                           _ptr(force4), float(dt), float(D), int(seed), int(step)), ctx)


def ab_md_step(ctx: Context, dom, pos4, vel4, acc4, dt=1.0):
    """Semi-implicit Euler step (Sec. 3, Eqs. 2-3): v += dt a, x += dt v."""
    for t, nm in [(pos4, "pos4"), (vel4, "vel4"), (acc4, "acc4")]:
        _dev(t, torch.float32, (4,), nm)
    ctx._stream()
    _check(_lib.ab_md_step(ctx.handle, ctypes.byref(dom), pos4.shape[0], _ptr(pos4), _ptr(vel4),
                           _ptr(acc4), float(dt)), ctx)


def ab_testing_scan_timeout(ctx: Context, items: int, skip_tile: int, limit_ns: int):
    ctx._stream()
    _check(_lib.ab_testing_scan_timeout(ctx.handle, int(items), int(skip_tile),
                                        int(limit_ns)), ctx)


def ab_testing_cell_table(ctx: Context, mode: int):
    """Testing hook: 0 automatic, 1 dense table, 2 table of occupied cells."""
    _check(_lib.ab_testing_cell_table(ctx.handle, int(mode)), ctx)


BUILD_SEQUENCE, BUILD_COOP, BUILD_RADIX, BUILD_AUTO = range(4)


def ab_testing_build_path(ctx: Context, path: int):
    """Testing hook: how ab_build runs -- 0 the counting sort as a kernel
    sequence, 1 the counting sort in one cooperative launch, 2 the radix
    sort, 3 the automatic choice (the default)."""
    _check(_lib.ab_testing_build_path(ctx.handle, int(path)), ctx)


def ab_testing_build_timeout(ctx: Context, skip_block: int, limit_ns: int):
    """Testing hook: in the next build, block `skip_block` never arrives at
    the first barrier (radix sort: scan tile `skip_block` of the first digit's
    counts never publishes its sum)."""
    _check(_lib.ab_testing_build_timeout(ctx.handle, int(skip_block), int(limit_ns)), ctx)


from .autograd import GaussPairSum, KernelMatvec, LJEnergy, lj_energy_forces  # noqa: E402,F401

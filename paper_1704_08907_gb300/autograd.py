"""torch.autograd.Function wrappers over the C ABI.

The backward passes call the library's hand-written adjoint kernels, which
recompute the pairs from the cell list instead of storing a neighbour list.
"""
from __future__ import annotations

import torch

from . import (AB_OP_GAUSS, AB_OP_LJ, Context, OpParams, ab_build, ab_kernel_matvec,
               ab_kernel_matvec_bwd, ab_pair_energy_grad, ab_pair_energy_grad_packed,
               ab_pair_sum, ab_pair_sum_bwd)


def _ensure_built(abctx: Context, dom, pos4, seq):
    # another forward may have rebuilt the context's cell list since
    if abctx.build_seq != seq:
        ab_build(abctx, dom, pos4)


class LJEnergy(torch.autograd.Function):
    """Per-particle truncated Lennard-Jones energy E_i (float32[n]).

    forward(pos4 float32[n,4], abctx, dom, eps, sigma) -> E;  the adjoint
    gives dL/dpos4 = sum_j 1/2 (g_i + g_j) C_ij dx_ij (minus the force for
    L = sum_i E_i)."""

    @staticmethod
    def forward(fctx, pos4, abctx, dom, eps, sigma, energy=None):
        seq = ab_build(abctx, dom, pos4.detach())
        prm = OpParams(eps=eps, sigma=sigma)
        E = ab_pair_sum(abctx, AB_OP_LJ, prm, energy=energy)
        fctx.save_for_backward(pos4)
        fctx.abctx, fctx.dom, fctx.prm, fctx.seq = abctx, dom, prm, seq
        return E

    @staticmethod
    def backward(fctx, gE):
        (pos4,) = fctx.saved_tensors
        _ensure_built(fctx.abctx, fctx.dom, pos4.detach(), fctx.seq)
        g = torch.empty_like(pos4)
        ab_pair_sum_bwd(fctx.abctx, AB_OP_LJ, fctx.prm, None, gE.contiguous(), grad_pos4=g)
        return g, None, None, None, None, None


class GaussPairSum(torch.autograd.Function):
    """y_i = sum_{|dx_ij| < r} w_j exp(-s |dx_ij|^2); differentiable in
    positions, weights and s (s may be a 0-dim float64 tensor)."""

    @staticmethod
    def forward(fctx, pos4, w, s, abctx, dom):
        sval = float(s)
        seq = ab_build(abctx, dom, pos4.detach())
        prm = OpParams(s=sval)
        y = ab_pair_sum(abctx, AB_OP_GAUSS, prm, w=w.detach().contiguous())
        fctx.save_for_backward(pos4, w)
        fctx.abctx, fctx.dom, fctx.prm, fctx.seq = abctx, dom, prm, seq
        fctx.s_is_tensor = isinstance(s, torch.Tensor)
        return y

    @staticmethod
    def backward(fctx, gy):
        pos4, w = fctx.saved_tensors
        _ensure_built(fctx.abctx, fctx.dom, pos4.detach(), fctx.seq)
        gpos = torch.empty_like(pos4)
        gw = torch.empty_like(w)
        gs = torch.empty((), dtype=torch.float64, device=pos4.device)
        ab_pair_sum_bwd(fctx.abctx, AB_OP_GAUSS, fctx.prm, w.detach().contiguous(),
                        gy.contiguous(), grad_pos4=gpos, grad_w=gw, grad_s=gs)
        return gpos, gw, (gs if fctx.s_is_tensor else None), None, None


class KernelMatvec(torch.autograd.Function):
    """out = K(X, Y) W with K_ij = exp(-s |x_i - y_j|^2); X, Y float32[.,4]."""

    @staticmethod
    def forward(fctx, X, Y, W, s, abctx, prec="fp32"):
        sval = float(s)
        out = ab_kernel_matvec(abctx, X.detach(), Y.detach(), W.detach().contiguous(), sval, prec)
        fctx.save_for_backward(X, Y, W)
        fctx.abctx, fctx.sval, fctx.prec = abctx, sval, prec
        fctx.s_is_tensor = isinstance(s, torch.Tensor)
        return out

    @staticmethod
    def backward(fctx, G):
        X, Y, W = fctx.saved_tensors
        dW = torch.empty_like(W) if fctx.needs_input_grad[2] else None
        dX = torch.empty_like(X) if fctx.needs_input_grad[0] else None
        dY = torch.empty_like(Y) if fctx.needs_input_grad[1] else None
        ds = torch.empty((), dtype=torch.float64, device=X.device) if fctx.s_is_tensor else None
        ab_kernel_matvec_bwd(fctx.abctx, X.detach(), Y.detach(), W.detach().contiguous(),
                             fctx.sval, fctx.prec, G.contiguous(), dW=dW, dX=dX, dY=dY, ds=ds)
        return dX, dY, dW, ds, None, None


def lj_energy_forces(abctx: Context, dom, pos4: torch.Tensor, eps: float, sigma: float,
                     E=None, F=None, energy=None, g=None):
    """One rebuild + LJ energy forward + adjoint (forces = -dE/dx).

    Positions are float32[n,4] or packed float32[n,dim]; the gradient comes
    back in the same layout.  Returns (E per particle, minus-force dE/dx,
    total energy float64 scalar tensor).  Buffers may be passed in to avoid
    allocation.  With g None (the loss is the total energy) the energy and
    its gradient come from one fused walk; with an explicit upstream g the
    forward and the adjoint run separately."""
    n = pos4.shape[0]
    packed = pos4.shape[1] == dom.dim
    ab_build(abctx, dom, pos4)
    prm = OpParams(eps=eps, sigma=sigma)
    if energy is None:
        energy = torch.empty((), dtype=torch.float64, device=pos4.device)
    if F is None:
        F = torch.empty_like(pos4)
    if g is None:
        if E is None:
            E = torch.empty(n, dtype=torch.float32, device=pos4.device)
        if packed:
            ab_pair_energy_grad_packed(abctx, AB_OP_LJ, prm, E=E, grad_pos=F, energy=energy)
        else:
            ab_pair_energy_grad(abctx, AB_OP_LJ, prm, E=E, grad_pos4=F, energy=energy)
        return E, F, energy
    E = ab_pair_sum(abctx, AB_OP_LJ, prm, out=E, energy=energy)
    if packed:
        G4 = torch.empty((n, 4), dtype=torch.float32, device=pos4.device)
        ab_pair_sum_bwd(abctx, AB_OP_LJ, prm, None, g, grad_pos4=G4)
        F.copy_(G4[:, :dom.dim])
    else:
        ab_pair_sum_bwd(abctx, AB_OP_LJ, prm, None, g, grad_pos4=F)
    return E, F, energy

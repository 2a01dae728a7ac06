"""torch.autograd functions over the library's operator, solver and force kernels.

TMApply:            y = M(U) psi (eq. 2.1, full lattice).  backward: grad_psi = M^dag g (tm_mat with
                    dagger), grad_U = the su(3)-projected link gradient (tm_force, coef 1).
PseudofermionAction: S = phi^dag (M^dag M)^-1 phi.  X = M^-1 M^-dag phi from two even-odd solves
                    (M^dag z = phi, then M X = z, so Y = M X = z); backward: grad_U from tm_force with
                    psi = X, g = Y, coef = -2; grad_phi = 2 X.

Canonical complex128 tensors run in FP64, complex64 in FP32 (the solves inside the action always run
in FP64 CG or mixed CG with an FP64 result).  Gradients follow torch's convention for complex
tensors (the conjugate Wirtinger derivative times two, so dL = Re sum conj(grad) dz).
"""
from __future__ import annotations

import torch

from . import (TM_PC_ASYM, TM_PREC_F32, TM_PREC_F64, Field, Gauge, Params, force, mat, pack, prepare_rhs,
               reconstruct_odd, solve, unpack)


def _prec(t):
    return TM_PREC_F64 if t.dtype == torch.complex128 else TM_PREC_F32


def _apply_full(g, psi, dagger, prec):
    e, o = pack(g, psi, 0, prec), pack(g, psi, 1, prec)
    oe, oo = Field(g, prec), Field(g, prec)
    mat(g, oe, oo, e, o, dagger)
    out = torch.zeros_like(psi)
    unpack(g, oe, 0, canon=out)
    unpack(g, oo, 1, canon=out)
    return out


class TMApply(torch.autograd.Function):
    """y = M(U) psi.  Arguments: U [4,Lt,Lz,Ly,Lx,3,3], psi [Lt,Lz,Ly,Lx,nf,4,3] (complex, cuda), params."""

    @staticmethod
    def forward(ctx, U, psi, params: Params):
        g = Gauge(params, U.detach())
        y = _apply_full(g, psi.detach(), False, _prec(psi))
        ctx.save_for_backward(psi)
        ctx.g = g
        return y

    @staticmethod
    def backward(ctx, gy):
        (psi,) = ctx.saved_tensors
        g = ctx.g
        prec = _prec(psi)
        gy = gy.to(psi.dtype).contiguous()
        grad_psi = _apply_full(g, gy, True, prec) if ctx.needs_input_grad[1] else None
        grad_U = None
        if ctx.needs_input_grad[0]:
            pe, po = pack(g, psi.detach(), 0, prec), pack(g, psi.detach(), 1, prec)
            ge, go = pack(g, gy, 0, prec), pack(g, gy, 1, prec)
            grad_U = force(g, pe, po, ge, go, coef=1.0, project=True)
        ctx.g = None
        g.close()
        return grad_U, grad_psi, None


def solve_full(g: Gauge, b, dagger=False, tol=1e-12, solver="cg", sloppy_prec=TM_PREC_F32, maxiter=50000):
    """psi with M psi = b (or M^dag psi = b): asymmetric even-odd solve + odd reconstruction, FP64 result."""
    be, bo = pack(g, b, 0, TM_PREC_F64), pack(g, b, 1, TM_PREC_F64)
    bp = Field(g, TM_PREC_F64)
    prepare_rhs(g, bp, be, bo, TM_PC_ASYM, dagger)
    xe = Field(g, TM_PREC_F64)
    stats = solve(g, xe, bp, pc=TM_PC_ASYM, dagger=dagger, tol=tol, solver=solver, sloppy_prec=sloppy_prec,
                  maxiter=maxiter)
    xo = Field(g, TM_PREC_F64)
    reconstruct_odd(g, xo, bo, xe, dagger)
    out = torch.zeros(b.shape, dtype=torch.complex128, device=b.device)
    unpack(g, xe, 0, canon=out)
    unpack(g, xo, 1, canon=out)
    return out, stats


class PseudofermionAction(torch.autograd.Function):
    """S = phi^dag (M^dag M)^-1 phi (real scalar) with the pseudofermion force as its U-gradient."""

    @staticmethod
    def forward(ctx, U, phi, params: Params, tol=1e-12, solver="cg"):
        g = Gauge(params, U.detach())
        phi64 = phi.detach().to(torch.complex128)
        z, _ = solve_full(g, phi64, dagger=True, tol=tol, solver=solver)  # z = M^-dag phi = Y
        X, _ = solve_full(g, z, dagger=False, tol=tol, solver=solver)    # X = M^-1 z
        S = torch.vdot(phi64.reshape(-1), X.reshape(-1)).real
        ctx.save_for_backward(X, z)
        ctx.g, ctx.phi_dtype, ctx.U_dtype = g, phi.dtype, U.dtype
        return S.to(torch.float64)

    @staticmethod
    def backward(ctx, gS):
        X, Y = ctx.saved_tensors
        g = ctx.g
        grad_U = grad_phi = None
        if ctx.needs_input_grad[0]:
            xe, xo = pack(g, X, 0, TM_PREC_F64), pack(g, X, 1, TM_PREC_F64)
            ye, yo = pack(g, Y, 0, TM_PREC_F64), pack(g, Y, 1, TM_PREC_F64)
            grad_U = (force(g, xe, xo, ye, yo, coef=-2.0, project=True) * gS).to(ctx.U_dtype)
        if ctx.needs_input_grad[1]:
            grad_phi = (2.0 * X * gS).to(ctx.phi_dtype)
        ctx.g = None
        g.close()
        return grad_U, grad_phi, None, None, None

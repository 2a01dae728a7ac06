"""torch.autograd functions over the library's operator, solver and force kernels.

TMApply:            y = M(U) psi (eq. 2.1, full lattice).  backward: grad_psi = M^dag g (tm_mat with
                    dagger), grad_U = the su(3)-projected link gradient (tm_force, coef 1).
PseudofermionAction: S = phi^dag (M^dag M)^-1 phi.  X = M^-1 M^-dag phi from two even-odd solves
                    (M^dag Y = phi, then M X = Y, so Y = M X); S = Re<phi, X> from tm_dot on the two
                    parities; backward: grad_U from tm_force with psi = X, g = Y and coef = -2 dS;
                    grad_phi = 2 dS X from tm_axpby.

Canonical complex128 tensors run in FP64, complex64 in FP32 (the solves inside the action always run
in FP64 CG or mixed CG with an FP64 result).  Gradients follow torch's convention for complex
tensors (the conjugate Wirtinger derivative times two, so dL = Re sum conj(grad) dz).  Every step
on field values is a library call; this module only packs, unpacks and sequences them.

Gauge handles are reused while U is unchanged: a handle is kept per parameter set together with a
weak reference to its U and U's version counter, so repeated calls with the same (unmodified) U pack
the links once, and only in the storage precisions the call computes in (tm_gauge_create_ex).  The
FP64 links keep all 18 reals (TM_GAUGE_F64_FULL_LINKS): the FP64 operator, solves and force run on
the FP64 pipe, where rebuilding the third row costs more than reading it.  A handle dropped from the cache stays alive while an autograd graph still holds it.
"""
from __future__ import annotations

import weakref

import torch

from . import (TM_PC_ASYM, TM_PREC_F32, TM_PREC_F64, Field, Gauge, Params, axpby, dot, force, mat, pack,
               prepare_rhs, reconstruct_odd, solve, unpack)

_CACHE: dict = {}   # params key -> (weakref to U, U._version, Gauge)
_CACHE_MAX = 2


def _key(params: Params, U, precs, f64_full):
    return (params.L, params.kappa, params.mu, params.eps, params.flavor, params.t_antiperiodic, params.recon,
            U.device.index, tuple(sorted(precs)), bool(f64_full))


def gauge_for(U, params: Params, precs=(TM_PREC_F64, TM_PREC_F32), f64_full=True) -> Gauge:
    """The cached handle of (U, params) holding the links of `precs` only (FP64 ones with all 18
    reals when f64_full), created when U is new or was modified in place."""
    k = _key(params, U, precs, f64_full)
    hit = _CACHE.get(k)
    if hit is not None and hit[0]() is U and hit[1] == U._version:
        return hit[2]
    g = Gauge(params, U.detach(), precs=precs, f64_full_links=f64_full)
    _CACHE.pop(k, None)
    while len(_CACHE) >= _CACHE_MAX:
        _CACHE.pop(next(iter(_CACHE)))
    _CACHE[k] = (weakref.ref(U), U._version, g)
    return g


def clear_cache():
    _CACHE.clear()


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
        g = gauge_for(U, params, (_prec(psi),))
        y = _apply_full(g, psi.detach(), False, _prec(psi))
        ctx.save_for_backward(psi)
        ctx.g, ctx.U_dtype = g, U.dtype
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
            out = torch.empty(g.params.gauge_shape, dtype=ctx.U_dtype, device=psi.device)
            grad_U = force(g, pe, po, ge, go, coef=1.0, project=True, out=out)
        ctx.g = None
        return grad_U, grad_psi, None


def solve_fields(g: Gauge, be: Field, bo: Field, dagger=False, tol=1e-12, solver="cg", sloppy_prec=TM_PREC_F32,
                 maxiter=50000):
    """(psi_e, psi_o) with M psi = b (or M^dag psi = b) for FP64 parity fields b: the asymmetric
    even-odd solve (eq. 2.2) and the odd reconstruction (eq. 2.4)."""
    bp = Field(g, TM_PREC_F64)
    prepare_rhs(g, bp, be, bo, TM_PC_ASYM, dagger)
    xe = Field(g, TM_PREC_F64)
    stats = solve(g, xe, bp, pc=TM_PC_ASYM, dagger=dagger, tol=tol, solver=solver, sloppy_prec=sloppy_prec,
                  maxiter=maxiter)
    xo = Field(g, TM_PREC_F64)
    reconstruct_odd(g, xo, bo, xe, dagger)
    return xe, xo, stats


def solve_full(g: Gauge, b, dagger=False, tol=1e-12, solver="cg", sloppy_prec=TM_PREC_F32, maxiter=50000):
    """psi with M psi = b (or M^dag psi = b) for a canonical b: solve_fields, FP64 canonical result."""
    be, bo = pack(g, b, 0, TM_PREC_F64), pack(g, b, 1, TM_PREC_F64)
    xe, xo, stats = solve_fields(g, be, bo, dagger, tol, solver, sloppy_prec, maxiter)
    out = torch.zeros(b.shape, dtype=torch.complex128, device=b.device)
    unpack(g, xe, 0, canon=out)
    unpack(g, xo, 1, canon=out)
    return out, stats


class PseudofermionAction(torch.autograd.Function):
    """S = phi^dag (M^dag M)^-1 phi (real scalar) with the pseudofermion force as its U-gradient."""

    @staticmethod
    def forward(ctx, U, phi, params: Params, tol=1e-12, solver="cg"):
        g = gauge_for(U, params, (TM_PREC_F64, TM_PREC_F32) if solver == "mixed" else (TM_PREC_F64,))
        phi64 = phi.detach().to(torch.complex128)
        pe, po = pack(g, phi64, 0, TM_PREC_F64), pack(g, phi64, 1, TM_PREC_F64)
        ye, yo, _ = solve_fields(g, pe, po, dagger=True, tol=tol, solver=solver)  # Y = M^-dag phi
        xe, xo, _ = solve_fields(g, ye, yo, dagger=False, tol=tol, solver=solver)  # X = M^-1 Y
        S = dot(g, pe, xe) + dot(g, po, xo)  # Re<phi, X>, FP64 reductions on the device
        ctx.fields = (xe, xo, ye, yo)
        ctx.g, ctx.phi_dtype, ctx.U_dtype = g, phi.dtype, U.dtype
        return torch.tensor(S, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, gS):
        xe, xo, ye, yo = ctx.fields
        g = ctx.g
        dS = float(gS)
        grad_U = grad_phi = None
        if ctx.needs_input_grad[0]:
            out = torch.empty(g.params.gauge_shape, dtype=ctx.U_dtype, device=xe.data.device)
            grad_U = force(g, xe, xo, ye, yo, coef=-2.0 * dS, project=True, out=out)
        if ctx.needs_input_grad[1]:
            ge, go = Field(g, TM_PREC_F64), Field(g, TM_PREC_F64)
            axpby(g, ge, 2.0 * dS, xe)
            axpby(g, go, 2.0 * dS, xo)
            grad_phi = torch.zeros(g.params.spinor_shape, dtype=ctx.phi_dtype, device=xe.data.device)
            unpack(g, ge, 0, canon=grad_phi)
            unpack(g, go, 1, canon=grad_phi)
        ctx.g = ctx.fields = None
        return grad_U, grad_phi, None, None, None

"""GB300-native even-odd preconditioned Wilson twisted-mass operator (arXiv:1311.4462).

Thin Python binding over ``libtm.so`` (C ABI: include/tm.h).  Every step of the operator
runs in the library's CUDA kernels; torch only provides device memory and streams.  The
functions below carry the same names as the C entry points without the ``tm_`` prefix.
"""
from __future__ import annotations

import ctypes

from . import _lib as L
from ._lib import (TM_SOLUTION_MAT, TM_SOLUTION_MATDAG_MAT, TM_SOLVER_CG, TM_SOLVER_MIXED, TM_C64, TM_C128, TM_EPI_NONE, TM_EPI_TWINV, TM_EPI_TWINV_XPAY, TM_EPI_TWXPAY_ASYM, TM_EPI_XMAY_K2,
                   TM_EPI_TWXPAY_SYM, TM_EPI_XPAY, TM_NDEG_DOUBLET, TM_PC_ASYM, TM_PC_SYM, TM_PREC_F16, TM_PREC_F32,
                   TM_PREC_F64, TM_PREC_DF64, TM_TWIST_MINUS, TM_TWIST_PLUS, TM_GAUGE_F64_FULL_LINKS, TMError)

PRECS = {"f64": TM_PREC_F64, "f32": TM_PREC_F32, "f16": TM_PREC_F16, "df64": TM_PREC_DF64}


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Params:
    """Lattice and operator parameters (tm_params).  flavor: +1, -1 (one flavour) or 2 (doublet)."""

    def __init__(self, L, kappa, mu, eps=0.0, flavor=TM_NDEG_DOUBLET, t_antiperiodic=True, recon=12):
        self.L = tuple(int(v) for v in L)
        self.kappa, self.mu, self.eps = float(kappa), float(mu), float(eps)
        self.flavor = int(flavor)
        self.t_antiperiodic = bool(t_antiperiodic)
        self.recon = int(recon)

    @property
    def nf(self):
        return 2 if self.flavor == TM_NDEG_DOUBLET else 1

    @property
    def volume(self):
        Lx, Ly, Lz, Lt = self.L
        return Lx * Ly * Lz * Lt

    @property
    def Vh(self):
        return self.volume // 2

    @property
    def spinor_shape(self):
        Lx, Ly, Lz, Lt = self.L
        return (Lt, Lz, Ly, Lx, self.nf, 4, 3)

    @property
    def gauge_shape(self):
        Lx, Ly, Lz, Lt = self.L
        return (4, Lt, Lz, Ly, Lx, 3, 3)

    def c(self):
        p = L.tm_params()
        p.L[:] = self.L
        p.kappa, p.mu, p.epsilon = self.kappa, self.mu, self.eps
        p.flavor, p.t_antiperiodic, p.recon = self.flavor, int(self.t_antiperiodic), self.recon
        return p


class Gauge:
    """tm_gauge handle: packed links in FP64/FP32/FP16 (the handle's recon) on the current device."""

    def __init__(self, params: Params, U, stream=None, precs=None, f64_full_links=False):
        """precs: the storage precisions whose links to pack (None: all; tm_gauge_create_ex).
        f64_full_links: FP64 links with all 18 reals whatever params.recon (TM_GAUGE_F64_FULL_LINKS;
        faster FP64 operators, e.g. the true residuals of the mixed solver)."""
        torch = _torch()
        self.params = params
        self.csw = 0.0
        U = torch.as_tensor(U)
        if U.device.type != "cuda":
            U = U.to("cuda")
        U = U.to(torch.complex128).contiguous()
        assert tuple(U.shape) == params.gauge_shape, (U.shape, params.gauge_shape)
        h = ctypes.c_void_p()
        self._pc = params.c()
        bit = {TM_PREC_F64: 1, TM_PREC_F32: 2, TM_PREC_F16: 4, TM_PREC_DF64: 8}
        mask = 0 if precs is None else sum(bit[int(q)] for q in set(precs))
        if f64_full_links:
            mask |= TM_GAUGE_F64_FULL_LINKS
        L.check(L.load().tm_gauge_create_ex(ctypes.byref(self._pc), ctypes.c_void_p(U.data_ptr()), int(mask),
                                            _stream(stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            L.load().tm_gauge_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field_bytes(self, prec, nrhs=1):
        d, n = ctypes.c_size_t(), ctypes.c_size_t()
        L.check(L.load().tm_field_bytes(self.h, int(prec), int(nrhs), ctypes.byref(d), ctypes.byref(n)))
        return d.value, n.value


class Field:
    """One parity of a spinor field in the library's layout; memory from torch."""

    def __init__(self, gauge: Gauge, prec=TM_PREC_F32, nrhs=1):
        torch = _torch()
        self.gauge, self.prec, self.nrhs = gauge, int(prec), int(nrhs)
        nd, nn = gauge.field_bytes(self.prec, self.nrhs)
        self.data = torch.empty(nd, dtype=torch.uint8, device="cuda")
        self.norm = torch.empty(max(nn // 4, 1), dtype=torch.float32, device="cuda") if nn else None
        self.c = L.tm_field(self.data.data_ptr(), self.norm.data_ptr() if self.norm is not None else None, self.prec,
                            self.nrhs)

    def ref(self):
        return ctypes.byref(self.c)

    def zero_(self):
        self.data.zero_()
        if self.norm is not None:
            self.norm.zero_()
        return self


def host_buffers(gauge: Gauge, prec=TM_PREC_F32, nrhs=1):
    """Page-locked host tensors (data as uint8, norm as float32 or None) sized for a field in the
    library's layout, for tm_field_upload / tm_field_download."""
    torch = _torch()
    nd, nn = gauge.field_bytes(prec, nrhs)
    data = torch.empty(nd, dtype=torch.uint8).pin_memory()
    norm = torch.empty(nn // 4, dtype=torch.float32).pin_memory() if nn else None
    return data, norm


def upload(gauge: Gauge, field: Field, host_data, host_norm=None, stream=None) -> Field:
    """tm_field_upload: host copy of a field in the library's layout -> device Field."""
    L.check(L.load().tm_field_upload(gauge.h, field.ref(), ctypes.c_void_p(host_data.data_ptr()),
                                     ctypes.c_void_p(host_norm.data_ptr()) if host_norm is not None else None,
                                     _stream(stream)))
    return field


def download(gauge: Gauge, field: Field, host_data, host_norm=None, stream=None):
    """tm_field_download: device Field -> host copy in the library's layout."""
    L.check(L.load().tm_field_download(gauge.h, ctypes.c_void_p(host_data.data_ptr()),
                                       ctypes.c_void_p(host_norm.data_ptr()) if host_norm is not None else None,
                                       field.ref(), _stream(stream)))
    return host_data, host_norm


def pack(gauge: Gauge, canon, parity: int, prec=TM_PREC_F32, nrhs=1, out: Field = None, stream=None) -> Field:
    """tm_pack: canonical complex128/complex64 device tensor -> one parity Field."""
    torch = _torch()
    canon = torch.as_tensor(canon)
    if canon.device.type != "cuda" and not canon.is_pinned():
        canon = canon.to("cuda")  # pinned host tensors are read in place by the kernel
    canon = canon.contiguous()
    ct = L.TM_C128 if canon.dtype == torch.complex128 else L.TM_C64
    if canon.dtype not in (torch.complex128, torch.complex64):
        raise TypeError("canonical fields are complex128 or complex64")
    f = out if out is not None else Field(gauge, prec, nrhs)
    L.check(L.load().tm_pack(gauge.h, f.ref(), ctypes.c_void_p(canon.data_ptr()), ct, int(parity), _stream(stream)))
    return f


def unpack(gauge: Gauge, field: Field, parity: int, canon=None, dtype=None, stream=None):
    """tm_unpack: writes the sites of `parity` into canon (a new zero device tensor if None; a
    pinned host tensor is written in place over the CPU-GPU link)."""
    torch = _torch()
    shape = gauge.params.spinor_shape
    if field.nrhs > 1:
        shape = (field.nrhs,) + shape
    if canon is None:
        canon = torch.zeros(shape, dtype=dtype or torch.complex128, device="cuda")
    ct = L.TM_C128 if canon.dtype == torch.complex128 else L.TM_C64
    L.check(L.load().tm_unpack(gauge.h, ctypes.c_void_p(canon.data_ptr()), ct, field.ref(), int(parity),
                               _stream(stream)))
    return canon


def dslash(gauge, out: Field, inp: Field, out_parity: int, epilogue=TM_EPI_NONE, x: Field = None, stream=None):
    L.check(L.load().tm_dslash(gauge.h, out.ref(), inp.ref(), int(out_parity), int(epilogue),
                               x.ref() if x is not None else None, _stream(stream)))
    return out


def dslash_dagger(gauge, out: Field, inp: Field, out_parity: int, epilogue=TM_EPI_NONE, x: Field = None, stream=None):
    L.check(L.load().tm_dslash_dagger(gauge.h, out.ref(), inp.ref(), int(out_parity), int(epilogue),
                                      x.ref() if x is not None else None, _stream(stream)))
    return out


def precond_op(gauge, out_e: Field, in_e: Field, tmp_o: Field, pc=TM_PC_ASYM, dagger=False, stream=None):
    L.check(L.load().tm_precond_op(gauge.h, out_e.ref(), in_e.ref(), tmp_o.ref(), int(pc), int(dagger),
                                   _stream(stream)))
    return out_e


def normal_op(gauge, out_e: Field, in_e: Field, tmp_e: Field, tmp_o: Field, pc=TM_PC_ASYM, dagger=False, stream=None):
    """tm_normal_op: out_e = A^dag A in_e, A = M_pc (or M_pc^dag)."""
    L.check(L.load().tm_normal_op(gauge.h, out_e.ref(), in_e.ref(), tmp_e.ref(), tmp_o.ref(), int(pc), int(dagger),
                                  _stream(stream)))
    return out_e


def mat(gauge, out_e: Field, out_o: Field, in_e: Field, in_o: Field, dagger=False, stream=None):
    L.check(L.load().tm_mat(gauge.h, out_e.ref(), out_o.ref(), in_e.ref(), in_o.ref(), int(dagger), _stream(stream)))
    return out_e, out_o


def prepare_rhs(gauge, bprime_e: Field, b_e: Field, b_o: Field, pc=TM_PC_ASYM, dagger=False, stream=None):
    L.check(L.load().tm_prepare_rhs(gauge.h, bprime_e.ref(), b_e.ref(), b_o.ref(), int(pc), int(dagger),
                                    _stream(stream)))
    return bprime_e


def reconstruct_odd(gauge, psi_o: Field, b_o: Field, psi_e: Field, dagger=False, stream=None):
    L.check(L.load().tm_reconstruct_odd(gauge.h, psi_o.ref(), b_o.ref(), psi_e.ref(), int(dagger), _stream(stream)))
    return psi_o


def twist(gauge, out: Field, inp: Field, inverse=False, dagger=False, stream=None):
    L.check(L.load().tm_twist(gauge.h, out.ref(), inp.ref(), int(inverse), int(dagger), _stream(stream)))
    return out


def local_op(gauge, out: Field, inp: Field, parity: int, inverse=False, dagger=False, stream=None):
    """tm_local_op: out = L in (or L^-1, daggered) on the sites of `parity`; L = R, or the clover
    operator 1 + T + (R - 1) of a handle with a clover term."""
    L.check(L.load().tm_local_op(gauge.h, out.ref(), inp.ref(), int(parity), int(inverse), int(dagger),
                                 _stream(stream)))
    return out


def device_status(gauge, stream=None):
    """tm_device_status: raises TMError (TM_ERR_TIMEOUT) if a bounded device-side wait gave up."""
    L.check(L.load().tm_device_status(gauge.h, _stream(stream)))


def set_clover(gauge, csw: float, stream=None):
    """tm_gauge_set_clover: add the clover term with coefficient c_sw (0 removes it)."""
    L.check(L.load().tm_gauge_set_clover(gauge.h, float(csw), _stream(stream)))
    gauge.csw = float(csw)
    return gauge


def norm2(gauge, x: Field, stream=None) -> float:
    """tm_norm2: |x|^2 with FP64 accumulation (blocking)."""
    out = ctypes.c_double()
    L.check(L.load().tm_norm2(gauge.h, x.ref(), ctypes.byref(out), _stream(stream)))
    return out.value


def dot(gauge, a: Field, b: Field, stream=None) -> float:
    """tm_dot: Re<a, b> with FP64 accumulation (blocking)."""
    out = ctypes.c_double()
    L.check(L.load().tm_dot(gauge.h, a.ref(), b.ref(), ctypes.byref(out), _stream(stream)))
    return out.value


def axpby(gauge, out: Field, a: float, x: Field, b: float = 0.0, y: Field = None, stream=None) -> Field:
    """tm_axpby: out = a x + b y (y None: out = a x) on one parity field."""
    L.check(L.load().tm_axpby(gauge.h, out.ref(), float(a), x.ref(), float(b), y.ref() if y is not None else None,
                              _stream(stream)))
    return out


# reliable-update thresholds: the sloppy residual may fall by this factor between FP64 updates
# (FP16 storage keeps about 3 digits, FP32 about 7).  Chosen from a sweep on the 32^3x64
# doublet to 1e-10: FP32 1e-5 needs 2 updates (141 ms) where 1e-3 needs 4 (184 ms) at the same
# 78 iterations; FP16 3e-3 needs 4 updates (174 ms) where 1e-2 needs 5 and 1e-3 costs 127 iterations.
DEFAULT_DELTA = {TM_PREC_F16: 3e-3, TM_PREC_F32: 1e-5}


def solver_params(solver="cg", solution=TM_SOLUTION_MAT, pc=TM_PC_ASYM, dagger=False, tol=1e-10, maxiter=20000,
                  delta=None, sloppy_prec=TM_PREC_F32, use_x0=False, want_pc_residual=False, use_graph=False,
                  true_prec=TM_PREC_F64):
    sp = L.tm_solver_params()
    sp.solver = TM_SOLVER_MIXED if solver == "mixed" else TM_SOLVER_CG
    sp.solution, sp.pc, sp.dagger = int(solution), int(pc), int(dagger)
    sp.tol, sp.maxiter = float(tol), int(maxiter)
    sp.delta = float(delta if delta is not None else DEFAULT_DELTA.get(int(sloppy_prec), 0.1))
    sp.sloppy_prec, sp.use_x0, sp.want_pc_residual = int(sloppy_prec), int(use_x0), int(want_pc_residual)
    sp.use_graph = int(use_graph)
    sp.true_prec = int(true_prec)
    return sp


def solve_workspace_bytes(gauge, sp) -> int:
    n = ctypes.c_size_t()
    L.check(L.load().tm_solve_workspace_bytes(gauge.h, ctypes.byref(sp), ctypes.byref(n)))
    return n.value


def solve(gauge, x_e: Field, b_e: Field, stream=None, workspace=None, check=True, **kw):
    """tm_solve on the even sites (x_e, b_e: FP64 Fields).  Returns the stats as a dict
    (with 'status'); raises TMError on failure unless check=False."""
    torch = _torch()
    sp = solver_params(**kw)
    nbytes = solve_workspace_bytes(gauge, sp)
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = L.tm_solver_stats()
    status = L.load().tm_solve(gauge.h, x_e.ref(), b_e.ref(), ctypes.byref(sp), ctypes.byref(st),
                               ctypes.c_void_p(workspace.data_ptr()), nbytes, _stream(stream))
    out = {"status": status, "iterations": st.iterations, "reliable_updates": st.reliable_updates,
           "true_residual": st.true_residual, "pc_residual": st.pc_residual, "seconds": st.seconds}
    if check:
        L.check(status)
    return out


def force(gauge, psi_e: Field, psi_o: Field, g_e: Field, g_o: Field, coef=1.0, project=True, out=None, stream=None):
    """tm_force: link gradient of Re<g, M(U) psi> in the canonical gauge layout."""
    torch = _torch()
    dt = torch.complex128 if psi_e.prec == TM_PREC_F64 else torch.complex64
    if out is None:
        out = torch.empty(gauge.params.gauge_shape, dtype=dt, device="cuda")
    ct = L.TM_C128 if out.dtype == torch.complex128 else L.TM_C64
    L.check(L.load().tm_force(gauge.h, ctypes.c_void_p(out.data_ptr()), ct, psi_e.ref(), psi_o.ref(), g_e.ref(),
                              g_o.ref(), float(coef), int(project), _stream(stream)))
    return out


def autotune(gauge, cache_path=None, stream=None):
    """tm_autotune, with an optional JSON cache keyed by lattice, flavours and recon."""
    import json
    import os
    key = "L%s_nf%d_recon%d" % ("x".join(map(str, gauge.params.L)), gauge.params.nf, gauge.params.recon)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        tune_import(gauge, cache[key])
        return cache[key]
    L.check(L.load().tm_autotune(gauge.h, _stream(stream)))
    table = tune_export(gauge)
    if cache_path:
        cache[key] = table
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return table


def tune_export(gauge) -> str:
    buf = ctypes.create_string_buffer(512)
    L.check(L.load().tm_tune_export(gauge.h, buf, 512))
    return buf.value.decode()


def tune_import(gauge, text: str):
    L.check(L.load().tm_tune_import(gauge.h, text.encode()))


def precond_op_active(gauge, out_e: Field, in_e: Field, tmp_o: Field, active, pc=TM_PC_ASYM, dagger=False,
                      stream=None):
    """tm_precond_op_active: only the right-hand sides listed in `active` (ints)."""
    torch = _torch()
    lst = torch.tensor(list(active), dtype=torch.int32, device="cuda")
    L.check(L.load().tm_precond_op_active(gauge.h, out_e.ref(), in_e.ref(), tmp_o.ref(), int(pc), int(dagger),
                                          ctypes.c_void_p(lst.data_ptr()), int(lst.numel()), _stream(stream)))
    torch.cuda.current_stream().synchronize()
    return out_e


def solve_multi(gauge, x_e: Field, b_e: Field, stream=None, workspace=None, check=True, **kw):
    """tm_solve_multi: all nrhs sources of b_e at once.  Returns (status, list of per-source stats)."""
    torch = _torch()
    sp = solver_params(**kw)
    n = ctypes.c_size_t()
    L.check(L.load().tm_solve_multi_workspace_bytes(gauge.h, ctypes.byref(sp), int(x_e.nrhs), ctypes.byref(n)))
    if workspace is None or workspace.numel() < n.value:
        workspace = torch.empty(n.value, dtype=torch.uint8, device="cuda")
    stats = (L.tm_solver_stats * x_e.nrhs)()
    status = L.load().tm_solve_multi(gauge.h, x_e.ref(), b_e.ref(), ctypes.byref(sp), stats,
                                     ctypes.c_void_p(workspace.data_ptr()), n.value, _stream(stream))
    out = [{"iterations": s.iterations, "reliable_updates": s.reliable_updates, "true_residual": s.true_residual,
            "seconds": s.seconds} for s in stats]
    if check:
        L.check(status)
    return status, out


def noise_z2(gauge, field: Field, parity: int, seed: int, stream=None) -> Field:
    """tm_noise_z2: counter-based Z2 noise (right-hand side r uses seed + r)."""
    L.check(L.load().tm_noise_z2(gauge.h, field.ref(), int(parity), ctypes.c_ulonglong(int(seed)), _stream(stream)))
    return field


def g5dot(gauge, a: Field, b: Field, stream=None):
    """tm_g5dot: <a_r, gamma5 b_r> per right-hand side, as a complex numpy array."""
    import numpy as np
    n = a.nrhs
    re, im = (ctypes.c_double * n)(), (ctypes.c_double * n)()
    L.check(L.load().tm_g5dot(gauge.h, a.ref(), b.ref(), re, im, _stream(stream)))
    return np.array(list(re)) + 1j * np.array(list(im))


def version() -> str:
    return L.load().tm_version().decode()

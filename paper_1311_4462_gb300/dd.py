"""Domain decomposition of the lattice in time: the multi-GPU parallelisation of sec. 2.1.

Each rank holds one time slab of the lattice in its own gauge handle (tm_gauge_set_partition).  A
hopping launch packs the spin-projected half-spinors of its first and last time slice for the
neighbouring slabs (tm_dd_pack_faces: 12 reals per site and flavour, both flavours of a doublet in
one face), runs the interior slices while the faces travel, then the two boundary slices with the
received faces (tm_dd_dslash).  The operators of eq. 2.2-2.4 are two such launches; the CG on the
normal equations sums the ranks' FP64 reductions with one allreduce each.

This module only sequences library calls and moves bytes.  Two transports:
  LocalTransport      all slabs in this process on one GPU (faces are device-to-device copies on a
                      side stream, overlapping the interior launches); every slab's launches are
                      issued in turn, so R slabs emulate R ranks with the same per-rank kernels;
  TorchDistTransport  one slab per process, faces as torch.distributed point-to-point messages
                      (NCCL on device buffers; gloo through host copies), reductions by all_reduce.
A decomposed operator gives the same bits as the undecomposed one (the faces carry the values in
the arithmetic precision and the receiving kernel performs the same operations in the same order).
"""
from __future__ import annotations

import ctypes
import math

from . import _lib as L
from . import (TM_EPI_TWINV, TM_EPI_TWINV_XPAY, TM_EPI_TWXPAY_ASYM, TM_EPI_TWXPAY_SYM, TM_EPI_XMAY_K2, TM_EPI_XPAY,
               TM_PC_ASYM, TM_PREC_DF64, TM_PREC_F16, TM_PREC_F64, Field,
               Gauge, Params, _stream, axpby, dot, norm2, pack, twist, unpack)


def _torch():
    import torch
    return torch


class Faces:
    """The four face buffers of one slab for one precision: sent to / received from the previous and
    the next slab."""

    def __init__(self, nbytes: int, device="cuda"):
        torch = _torch()
        self.nbytes = int(nbytes)
        mk = lambda: torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.send_prev, self.send_next, self.recv_prev, self.recv_next = mk(), mk(), mk(), mk()


class Slab:
    """One rank's time slab [t0, t0 + Lt_slab) of a lattice with params.L: a partitioned handle and
    its face buffers.  U_slab: canonical links of the slab's sites, [4, Lt_slab, Lz, Ly, Lx, 3, 3]."""

    def __init__(self, params: Params, U_slab, t0: int, stream=None):
        Lx, Ly, Lz, Lt = params.L
        lt = int(U_slab.shape[1])
        self.params = params
        self.t0, self.lt = int(t0), lt
        self.local = Params((Lx, Ly, Lz, lt), params.kappa, params.mu, params.eps, params.flavor,
                            params.t_antiperiodic, params.recon)
        self.g = Gauge(self.local, U_slab, stream)
        L.check(L.load().tm_gauge_set_partition(self.g.h, self.t0, Lt))
        self._faces = {}

    def faces(self, prec) -> Faces:
        if prec not in self._faces:
            n = ctypes.c_size_t()
            L.check(L.load().tm_dd_face_bytes(self.g.h, int(prec), ctypes.byref(n)))
            self._faces[prec] = Faces(n.value)
        return self._faces[prec]

    def field(self, prec=TM_PREC_F64) -> Field:
        return Field(self.g, prec)

    def close(self):
        self.g.close()


def slab_bounds(Lt: int, nranks: int):
    """(t0, Lt_slab) per rank: equal even slabs (Lt / nranks must be an even integer >= 2)."""
    if Lt % nranks or (Lt // nranks) % 2:
        raise ValueError(f"Lt = {Lt} does not split into {nranks} even slabs")
    lt = Lt // nranks
    return [(r * lt, lt) for r in range(nranks)]


def make_slabs(params: Params, U, nranks: int, ranks=None):
    """Slabs of the canonical gauge field U [4, Lt, Lz, Ly, Lx, 3, 3] cut into nranks time slabs:
    all of them (ranks=None, for LocalTransport) or those of the listed ranks (one per process)."""
    bounds = slab_bounds(params.L[3], nranks)
    keep = range(nranks) if ranks is None else ranks
    return [Slab(params, U[:, t0:t0 + lt].contiguous(), t0) for r, (t0, lt) in enumerate(bounds) if r in keep]


def split_field(slabs, psi):
    """The slabs' parts of a canonical spinor field [Lt, Lz, Ly, Lx, nf, 4, 3]."""
    return [psi[s.t0:s.t0 + s.lt].contiguous() for s in slabs]


def pack_slabs(slabs, parts, parity, prec=TM_PREC_F64):
    return [pack(s.g, p, parity, prec) for s, p in zip(slabs, parts)]


def unpack_slabs(slabs, fields, parity, out=None):
    """Write the sites of `parity` of every slab's field into the canonical full-lattice tensor out."""
    torch = _torch()
    s0 = slabs[0]
    if out is None:
        Lx, Ly, Lz, Lt = s0.params.L
        out = torch.zeros((Lt, Lz, Ly, Lx, s0.params.nf, 4, 3), dtype=torch.complex128, device="cuda")
    for s, f in zip(slabs, fields):
        part = out[s.t0:s.t0 + s.lt]
        tmp = part.contiguous()
        unpack(s.g, f, parity, canon=tmp)
        part.copy_(tmp)
    return out


# ------------------------------------------------------------------------------- transports
class LocalTransport:
    """Every slab of the lattice lives in this process on one GPU: slab r's face for the next slab is
    copied into slab r+1's receive buffer (and the reverse), on a side stream that starts once the
    faces are packed and that the boundary launches wait for."""

    def __init__(self):
        torch = _torch()
        self.side = torch.cuda.Stream()

    def exchange(self, slabs, prec, packed_event):
        torch = _torch()
        R = len(slabs)
        self.side.wait_event(packed_event)
        with torch.cuda.stream(self.side):
            for r, s in enumerate(slabs):
                f, nxt, prv = s.faces(prec), slabs[(r + 1) % R].faces(prec), slabs[(r - 1) % R].faces(prec)
                nxt.recv_prev.copy_(f.send_next, non_blocking=True)
                prv.recv_next.copy_(f.send_prev, non_blocking=True)
        done = torch.cuda.Event()
        done.record(self.side)
        torch.cuda.current_stream().wait_event(done)

    def allreduce(self, values):
        return math.fsum(values)


class TorchDistTransport:
    """One slab per process.  Faces travel as point-to-point messages of torch.distributed: with
    NCCL straight from device memory, with gloo through host copies.  The messages to a neighbour
    are issued in a fixed order (the face for the next slab, then the one for the previous), which
    is also the order in which the neighbour posts its receives, so they match even when both
    neighbours are the same rank (two ranks)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        torch = _torch()
        self.dist, self.group = dist, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        self.host = dist.get_backend(group) == "gloo"
        self.side = torch.cuda.Stream() if torch.cuda.is_available() else None
        self._stage = {}

    def _host(self, t, key):
        torch = _torch()
        if t.device.type == "cpu":
            return t
        key = (key, t.numel())  # one pinned buffer per role and size (faces of FP64, FP32, FP16 fields)
        if key not in self._stage:
            self._stage[key] = torch.empty(t.numel(), dtype=t.dtype).pin_memory()
        return self._stage[key]

    def exchange_buffers(self, f: Faces):
        """Send f.send_next to the next rank and f.send_prev to the previous one; receive into
        f.recv_prev and f.recv_next.  Host-blocking."""
        dist = self.dist
        nxt, prv = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        if self.world == 1:
            f.recv_prev.copy_(f.send_next)
            f.recv_next.copy_(f.send_prev)
            return
        if self.host:
            sn, sp = self._host(f.send_next, "sn"), self._host(f.send_prev, "sp")
            rp, rn = self._host(f.recv_prev, "rp"), self._host(f.recv_next, "rn")
            if sn is not f.send_next:
                sn.copy_(f.send_next)
                sp.copy_(f.send_prev)
            reqs = [dist.isend(sn, nxt, group=self.group, tag=1), dist.isend(sp, prv, group=self.group, tag=2),
                    dist.irecv(rp, prv, group=self.group, tag=1), dist.irecv(rn, nxt, group=self.group, tag=2)]
            for q in reqs:
                q.wait()
            if rp is not f.recv_prev:
                f.recv_prev.copy_(rp)
                f.recv_next.copy_(rn)
        else:
            ops = [dist.P2POp(dist.isend, f.send_next, nxt, self.group), dist.P2POp(dist.isend, f.send_prev, prv, self.group),
                   dist.P2POp(dist.irecv, f.recv_prev, prv, self.group), dist.P2POp(dist.irecv, f.recv_next, nxt, self.group)]
            for q in dist.batch_isend_irecv(ops):
                q.wait()

    def exchange(self, slabs, prec, packed_event):
        torch = _torch()
        (s,) = slabs
        self.side.wait_event(packed_event)
        with torch.cuda.stream(self.side):
            if self.host:
                self.side.synchronize()  # the faces are packed before the host copies read them
            self.exchange_buffers(s.faces(prec))
        done = torch.cuda.Event()
        done.record(self.side)
        torch.cuda.current_stream().wait_event(done)

    def allreduce(self, values):
        torch = _torch()
        dev = "cpu" if self.host else "cuda"
        t = torch.tensor([math.fsum(values)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())


# ------------------------------------------------------------------------------- operators
def dslash(slabs, outs, ins, out_parity, epilogue, xs, transport, dagger=False, twist_in=False, stream=None):
    """tm_dslash / tm_dslash_dagger of the decomposed lattice: faces packed, interior slices launched,
    faces exchanged (overlapping the interior), boundary slices launched."""
    torch = _torch()
    lib = L.load()
    prec = ins[0].prec
    st = _stream(stream)
    for s, inp in zip(slabs, ins):
        f = s.faces(prec)
        L.check(lib.tm_dd_pack_faces(s.g.h, ctypes.c_void_p(f.send_prev.data_ptr()),
                                     ctypes.c_void_p(f.send_next.data_ptr()), inp.ref(), int(out_parity), int(dagger),
                                     int(twist_in), st))
    packed = torch.cuda.Event()
    packed.record(torch.cuda.current_stream())
    xs = xs if xs is not None else [None] * len(slabs)
    for s, o, inp, x in zip(slabs, outs, ins, xs):
        L.check(lib.tm_dd_dslash(s.g.h, o.ref(), inp.ref(), int(out_parity), int(epilogue),
                                 x.ref() if x is not None else None, int(dagger), int(twist_in), None, None,
                                 L.TM_DD_INTERIOR, st))
    transport.exchange(slabs, prec, packed)
    for s, o, inp, x in zip(slabs, outs, ins, xs):
        f = s.faces(prec)
        L.check(lib.tm_dd_dslash(s.g.h, o.ref(), inp.ref(), int(out_parity), int(epilogue),
                                 x.ref() if x is not None else None, int(dagger), int(twist_in),
                                 ctypes.c_void_p(f.recv_prev.data_ptr()), ctypes.c_void_p(f.recv_next.data_ptr()),
                                 L.TM_DD_BOUNDARY, st))
    return outs


def precond_op(slabs, outs, ins, tmps, transport, pc=TM_PC_ASYM, dagger=False):
    """tm_precond_op on the decomposed lattice: M_asym (eq. 2.2) or M_sym (eq. 2.3), or an adjoint."""
    if pc == TM_PC_ASYM:
        dslash(slabs, tmps, ins, 1, TM_EPI_TWINV, None, transport, dagger)
        return dslash(slabs, outs, tmps, 0, TM_EPI_TWXPAY_ASYM, ins, transport, dagger)
    if not dagger:
        dslash(slabs, tmps, ins, 1, TM_EPI_TWINV, None, transport, False)
        return dslash(slabs, outs, tmps, 0, TM_EPI_TWXPAY_SYM, ins, transport, False)
    # adjoint of the symmetric operator: R^-dag_ee on the input, then x - kappa^2 H^dag t.  The
    # input twist is the first launch's prologue, or (DF64, and the FP16 doublet, as tm_precond_op
    # does it) an elementwise pass into outs, which the last launch overwrites.
    prec = ins[0].prec
    if prec == TM_PREC_DF64 or (prec == TM_PREC_F16 and slabs[0].params.nf == 2):
        for s, o, i in zip(slabs, outs, ins):
            twist(s.g, o, i, inverse=True, dagger=True)
        dslash(slabs, tmps, outs, 1, TM_EPI_TWINV, None, transport, True)
    else:
        dslash(slabs, tmps, ins, 1, TM_EPI_TWINV, None, transport, True, twist_in=True)
    return dslash(slabs, outs, tmps, 0, TM_EPI_XMAY_K2, ins, transport, True)


def prepare_rhs(slabs, bps, bes, bos, transport, pc=TM_PC_ASYM, dagger=False):
    """tm_prepare_rhs on the decomposed lattice: b'_e = b_e + kappa H_eo R^-1_oo b_o (SYM without
    dagger: R^-1_ee of that), the R^-1 twist applied to b_o by the input prologue."""
    epi = TM_EPI_TWINV_XPAY if (pc != TM_PC_ASYM and not dagger) else TM_EPI_XPAY
    return dslash(slabs, bps, bos, 0, epi, bes, transport, dagger, twist_in=True)


def reconstruct_odd(slabs, psios, bos, psies, transport, dagger=False):
    """tm_reconstruct_odd on the decomposed lattice: psi_o = R^-1_oo (b_o + kappa H_oe psi_e) (eq. 2.4)."""
    return dslash(slabs, psios, psies, 1, TM_EPI_TWINV_XPAY, bos, transport, dagger)


def _fields(slabs, prec=TM_PREC_F64):
    return [s.field(prec) for s in slabs]


def cg(slabs, xs, bs, transport, pc=TM_PC_ASYM, dagger=False, tol=1e-10, maxiter=20000, sloppy_prec=None,
       delta=1e-5):
    """CG on the normal equations A^dag A x = A^dag b of the decomposed even-odd operator A = M_pc
    (A = M_pc^dag when dagger), FP64 fields x, b, x starting from zero: the solve_type NORMOP of
    sec. 2.2 with every reduction summed over the ranks.

    sloppy_prec None: FP64 CG; it stops when the recursive residual reaches tol, recomputes the true
    residual |A^dag b - A^dag A x| / |A^dag b| and restarts from it (at most four times) while it is
    above tol.  sloppy_prec TM_PREC_F32: the reliable-update mixed CG of sec. 3 (ref. [Clark:2009wm])
    as tm_solve runs it -- FP32 search direction, residual and solution increment, and when the
    sloppy residual has fallen by delta since the last update (or meets tol) the increment is added
    to the FP64 x and the true residual recomputed in FP64.  Returns a dict with iterations,
    reliable updates / restarts, true_residual and converged."""
    ar = transport.allreduce
    tol2 = tol * tol
    bh, r, Ap, te, to = (_fields(slabs) for _ in range(5))

    def normal(out, inp, tes, tos):
        precond_op(slabs, tes, inp, tos, transport, pc, dagger)
        precond_op(slabs, out, tes, tos, transport, pc, not dagger)

    def n2(fs):
        return ar([norm2(s.g, f) for s, f in zip(slabs, fs)])

    precond_op(slabs, bh, bs, to, transport, pc, not dagger)  # bhat = A^dag b
    bb = n2(bh)
    for x in xs:
        x.zero_()
    if bb == 0.0:
        return {"iterations": 0, "restarts": 0, "true_residual": 0.0, "converged": True}
    for s, r_, b_ in zip(slabs, r, bh):
        axpby(s.g, r_, 1.0, b_)
    r2 = n2(r)
    it = nrel = 0
    if sloppy_prec is not None:
        if int(sloppy_prec) != 4:
            raise ValueError("dd.cg: the sloppy fields are FP32 (TM_PREC_F32)")
        rs, ps, Aps, tes, tos, xsl = (_fields(slabs, 4) for _ in range(6))
        for s, a, b_ in zip(slabs, rs, r):
            axpby(s.g, a, 1.0, b_)  # FP32 copy of the FP64 residual
        for s, a, b_ in zip(slabs, ps, rs):
            axpby(s.g, a, 1.0, b_)
        for x in xsl:
            x.zero_()
        rr = n2(rs)
        maxr = math.sqrt(r2)
        converged = r2 <= tol2 * bb
        while not converged and it < maxiter:
            normal(Aps, ps, tes, tos)
            pAp = ar([dot(s.g, p_, a_) for s, p_, a_ in zip(slabs, ps, Aps)])
            alpha = rr / pAp
            for s, x, p_, r_, a_ in zip(slabs, xsl, ps, rs, Aps):
                axpby(s.g, x, 1.0, x, alpha, p_)
                axpby(s.g, r_, 1.0, r_, -alpha, a_)
            rnew = n2(rs)
            it += 1
            if not math.isfinite(rnew):
                raise L.TMError(L.TM_ERR_NAN, f"dd.cg: non-finite residual at iteration {it}")
            rn = math.sqrt(rnew)
            maxr = max(maxr, rn)
            if rn < delta * maxr or rnew <= tol2 * bb or it == maxiter:
                # reliable update: x += x_sloppy in FP64, true residual recomputed in FP64
                for s, x, d in zip(slabs, xs, xsl):
                    axpby(s.g, x, 1.0, d, 1.0, x)
                for x in xsl:
                    x.zero_()
                normal(Ap, xs, te, to)
                for s, r_, b_, a_ in zip(slabs, r, bh, Ap):
                    axpby(s.g, r_, 1.0, b_, -1.0, a_)
                r2 = n2(r)
                nrel += 1
                if r2 <= tol2 * bb:
                    converged = True
                    break
                for s, a, b_ in zip(slabs, rs, r):
                    axpby(s.g, a, 1.0, b_)
                rnew = n2(rs)
                maxr = math.sqrt(r2)
            beta = rnew / rr
            rr = rnew
            for s, p_, r_ in zip(slabs, ps, rs):
                axpby(s.g, p_, 1.0, r_, beta, p_)
        return {"iterations": it, "reliable_updates": nrel, "true_residual": math.sqrt(r2 / bb),
                "converged": r2 <= tol2 * bb}
    p = _fields(slabs)
    restarts = 0
    while r2 > tol2 * bb and it < maxiter and restarts < 5:
        for s, p_, r_ in zip(slabs, p, r):
            axpby(s.g, p_, 1.0, r_)
        rr = r2
        while rr > tol2 * bb and it < maxiter:
            normal(Ap, p, te, to)
            pAp = ar([dot(s.g, p_, a_) for s, p_, a_ in zip(slabs, p, Ap)])
            alpha = rr / pAp
            for s, x, p_, r_, a_ in zip(slabs, xs, p, r, Ap):
                axpby(s.g, x, 1.0, x, alpha, p_)
                axpby(s.g, r_, 1.0, r_, -alpha, a_)
            rnew = n2(r)
            it += 1
            if not math.isfinite(rnew):
                raise L.TMError(L.TM_ERR_NAN, f"dd.cg: non-finite residual at iteration {it}")
            if rnew <= tol2 * bb:
                rr = rnew
                break
            beta = rnew / rr
            rr = rnew
            for s, p_, r_ in zip(slabs, p, r):
                axpby(s.g, p_, 1.0, r_, beta, p_)
        normal(Ap, xs, te, to)  # true residual r = bhat - A^dag A x
        for s, r_, b_, a_ in zip(slabs, r, bh, Ap):
            axpby(s.g, r_, 1.0, b_, -1.0, a_)
        r2 = n2(r)
        restarts += 1
    return {"iterations": it, "restarts": restarts - 1, "true_residual": math.sqrt(r2 / bb),
            "converged": r2 <= tol2 * bb}

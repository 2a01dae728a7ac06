"""Domain decomposition in time (the multi-GPU parallelisation of sec. 2.1), emulated on one GPU:
the lattice cut into 1 ... Lt/2 time slabs, each in its own handle, faces exchanged by device
copies.  The decomposed operators give the same bits as the undecomposed ones (the faces carry the
values in the arithmetic precision) and match the oracle; the decomposed CG (one FP64 allreduce per
reduction) solves the system."""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {8: 1e-13, 4: 1e-6, 2: 5e-3}
CASES = [
    ("nd_4x4x2x8", (4, 4, 2, 8), 2, 0.1612, 0.135, 0.15),
    ("plus_6x2x4x8", (6, 2, 4, 8), 1, 0.1612, 0.004, 0.0),
    ("minus_2x4x4x12", (2, 4, 4, 12), -1, 0.16, 0.01, 0.0),
]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def nranks_of(L):
    Lt = L[3]
    return sorted({1, 2, Lt // 2} | ({3} if Lt % 6 == 0 else set()))


_cache = {}


def setup(case):
    import paper_1311_4462_gb300 as tmq
    if case[0] not in _cache:
        name, L, flavor, kappa, mu, eps = case
        p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
        po = orc.Params(L, kappa, mu, eps, flavor=flavor)
        U = inputs.gauge_field(L, 1700 + len(name))
        psi = inputs.spinor_field(L, p.nf, 2700 + len(name))
        chi = inputs.spinor_field(L, p.nf, 2800 + len(name))
        g = tmq.Gauge(p, torch.from_numpy(U))
        _cache[case[0]] = (p, po, U, psi, chi, g, {})
    return _cache[case[0]]


def slabs_of(case, R):
    from paper_1311_4462_gb300 import dd
    p, po, U, psi, chi, g, sl = setup(case)
    if R not in sl:
        sl[R] = dd.make_slabs(p, torch.from_numpy(U).to("cuda"), R)
    return sl[R]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [8, 4, 2])
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
def test_dd_precond_op_same_bits_as_one_slab(case, prec, pc, dagger):
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import dd
    p, po, U, psi, chi, g, _ = setup(case)
    tpsi = torch.from_numpy(psi).to("cuda")
    xe = tmq.pack(g, tpsi, 0, prec)
    out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
    tmq.precond_op(g, out, xe, tmp, pc, dagger)
    ref = tmq.unpack(g, out, 0)
    oref = orc.apply_M_pc(po, U, orc.project_parity(po, psi, 0), sym=bool(pc), dagger=dagger)
    for R in nranks_of(p.L):
        slabs = slabs_of(case, R)
        ins = dd.pack_slabs(slabs, dd.split_field(slabs, tpsi), 0, prec)
        outs, tmps = [s.field(prec) for s in slabs], [s.field(prec) for s in slabs]
        dd.precond_op(slabs, outs, ins, tmps, dd.LocalTransport(), pc, dagger)
        got = dd.unpack_slabs(slabs, outs, 0)
        assert torch.equal(got, ref), R
        assert rel(got.cpu().numpy(), oref) < TOL[prec]


@pytest.mark.parametrize("case", CASES[:2], ids=[c[0] for c in CASES[:2]])
@pytest.mark.parametrize("prec", [8, 4, 2])
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_dd_dslash_epilogues_and_regions(case, prec, dagger, out_parity):
    """Every epilogue (and the input prologue) of the decomposed hopping launch against tm_dslash;
    the interior-then-boundary split against one TM_DD_ALL launch."""
    import ctypes
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import _lib as Lb
    from paper_1311_4462_gb300 import dd
    p, po, U, psi, chi, g, _ = setup(case)
    tpsi, tchi = torch.from_numpy(psi).to("cuda"), torch.from_numpy(chi).to("cuda")
    ip = 1 - out_parity
    fin, fx = tmq.pack(g, tpsi, ip, prec), tmq.pack(g, tchi, out_parity, prec)
    R = 2
    slabs = slabs_of(case, R)
    ins = dd.pack_slabs(slabs, dd.split_field(slabs, tpsi), ip, prec)
    xs = dd.pack_slabs(slabs, dd.split_field(slabs, tchi), out_parity, prec)
    tr = dd.LocalTransport()
    fn = tmq.dslash_dagger if dagger else tmq.dslash
    for twist_in in (False, True):
        for epi in range(7):
            out = tmq.Field(g, prec)
            if twist_in:  # the prologue R^-1 on the input = tm_dslash of the twisted input
                tw = tmq.twist(g, tmq.Field(g, prec), fin, True, dagger)
                fn(g, out, tw, out_parity, epi, fx)
            else:
                fn(g, out, fin, out_parity, epi, fx)
            ref = tmq.unpack(g, out, out_parity)
            outs = [s.field(prec) for s in slabs]
            dd.dslash(slabs, outs, ins, out_parity, epi, xs, tr, dagger, twist_in=twist_in)
            got = dd.unpack_slabs(slabs, outs, out_parity)
            if twist_in:  # a separate twist pass rounds to the storage precision first
                assert rel(got.cpu().numpy(), ref.cpu().numpy()) < TOL[prec], epi
            else:
                assert torch.equal(got, ref), epi
    # the faces now hold ins (with the prologue); one TM_DD_ALL launch per slab = interior + boundary
    lib = Lb.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [s.field(prec) for s in slabs]
    dd.dslash(slabs, outs, ins, out_parity, tmq.TM_EPI_TWXPAY_ASYM, xs, tr, dagger, twist_in=True)
    outs_all = [s.field(prec) for s in slabs]
    for s, o, i, x in zip(slabs, outs_all, ins, xs):
        f = s.faces(prec)
        Lb.check(lib.tm_dd_dslash(s.g.h, o.ref(), i.ref(), out_parity, tmq.TM_EPI_TWXPAY_ASYM, x.ref(), int(dagger), 1,
                                  ctypes.c_void_p(f.recv_prev.data_ptr()), ctypes.c_void_p(f.recv_next.data_ptr()),
                                  Lb.TM_DD_ALL, st))
    assert torch.equal(dd.unpack_slabs(slabs, outs_all, out_parity), dd.unpack_slabs(slabs, outs, out_parity))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_dd_cg_full_solve(case):
    """prepare_rhs, CG on the normal equations with summed reductions, reconstruction: the full-system
    residual of the oracle, and the undecomposed solver's solution."""
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import dd
    p, po, U, psi, chi, g, _ = setup(case)
    tb = torch.from_numpy(chi).to("cuda")
    R = 2
    slabs = slabs_of(case, R)
    tr = dd.LocalTransport()
    parts = dd.split_field(slabs, tb)
    bes, bos = dd.pack_slabs(slabs, parts, 0), dd.pack_slabs(slabs, parts, 1)
    bps, xes, xos = ([s.field() for s in slabs] for _ in range(3))
    dd.prepare_rhs(slabs, bps, bes, bos, tr)
    st = dd.cg(slabs, xes, bps, tr, tol=1e-10)
    assert st["converged"] and st["true_residual"] <= 1e-10
    dd.reconstruct_odd(slabs, xos, bos, xes, tr)
    x = dd.unpack_slabs(slabs, xes, 0)
    dd.unpack_slabs(slabs, xos, 1, out=x)
    assert rel(orc.apply_M(po, U, x.cpu().numpy()), chi) < 1e-7
    be, bo = tmq.pack(g, tb, 0, 8), tmq.pack(g, tb, 1, 8)
    bp, xe = tmq.Field(g, 8), tmq.Field(g, 8)
    tmq.prepare_rhs(g, bp, be, bo, 0, False)
    assert torch.equal(tmq.unpack(g, bp, 0), dd.unpack_slabs(slabs, bps, 0))
    tmq.solve(g, xe, bp, solver="cg", tol=1e-10)
    assert rel(dd.unpack_slabs(slabs, xes, 0).cpu().numpy(), tmq.unpack(g, xe, 0).cpu().numpy()) < 1e-7
    # the decomposed reliable-update mixed CG (FP32 sloppy fields, FP64 updates), both PC forms
    for pc in (0, 1):
        bps2, xes2, xos2 = ([s.field() for s in slabs] for _ in range(3))
        dd.prepare_rhs(slabs, bps2, bes, bos, tr, pc)
        st = dd.cg(slabs, xes2, bps2, tr, pc=pc, tol=1e-10, sloppy_prec=4)
        assert st["converged"] and st["true_residual"] <= 1e-10 and st["reliable_updates"] >= 1
        dd.reconstruct_odd(slabs, xos2, bos, xes2, tr)  # both forms solve for the same psi_e (eq. 2.4)
        x2 = dd.unpack_slabs(slabs, xes2, 0)
        dd.unpack_slabs(slabs, xos2, 1, out=x2)
        assert rel(orc.apply_M(po, U, x2.cpu().numpy()), chi) < 1e-7


def test_dd_argument_errors():
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import _lib as Lb
    case = CASES[0]
    p, po, U, psi, chi, g, _ = setup(case)
    lib = Lb.load()
    slabs = slabs_of(case, 2)
    s = slabs[0]
    f = s.field(4)
    with pytest.raises(tmq.TMError):  # a slab refuses the undecomposed hopping calls
        tmq.precond_op(s.g, s.field(4), f, s.field(4), 0, False)
    with pytest.raises(tmq.TMError):
        tmq.dslash(s.g, s.field(4), f, 0)
    assert lib.tm_gauge_set_partition(s.g.h, 1, p.L[3]) == Lb.TM_ERR_ARG       # odd offset
    assert lib.tm_gauge_set_partition(s.g.h, p.L[3], p.L[3]) == Lb.TM_ERR_ARG  # beyond the lattice
    assert lib.tm_dd_dslash(g.h, f.ref(), s.field(4).ref(), 0, 0, None, 0, 0, None, None, 0, None) == Lb.TM_ERR_ARG
    assert lib.tm_dd_dslash(s.g.h, s.field(4).ref(), f.ref(), 0, 0, None, 0, 0, None, None, Lb.TM_DD_ALL,
                            None) == Lb.TM_ERR_ARG  # the boundary needs faces
    assert lib.tm_dd_dslash(s.g.h, s.field(4).ref(), f.ref(), 0, 0, None, 0, 0, None, None, 7, None) == Lb.TM_ERR_ARG


@pytest.mark.parametrize("recon", [18, 8])
@pytest.mark.parametrize("prec", [8, 4, 2])
def test_dd_other_link_formats(recon, prec):
    """18- and 8-real links: the face of the backward hop carries the sender's decoded link product."""
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import dd
    L = (4, 2, 4, 8)
    p = tmq.Params(L, 0.1612, 0.135, 0.15, flavor=tmq.TM_NDEG_DOUBLET, recon=recon)
    po = orc.Params(L, 0.1612, 0.135, 0.15, flavor=2)
    U = inputs.gauge_field(L, 1790)
    psi = inputs.spinor_field(L, 2, 2790)
    g = tmq.Gauge(p, torch.from_numpy(U))
    tpsi = torch.from_numpy(psi).to("cuda")
    xe = tmq.pack(g, tpsi, 0, prec)
    out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
    tr = dd.LocalTransport()
    for R in (2, 4):
        slabs = dd.make_slabs(p, torch.from_numpy(U).to("cuda"), R)
        ins = dd.pack_slabs(slabs, dd.split_field(slabs, tpsi), 0, prec)
        for pc, dag in ((0, False), (1, True)):
            tmq.precond_op(g, out, xe, tmp, pc, dag)
            outs, tmps = [s.field(prec) for s in slabs], [s.field(prec) for s in slabs]
            dd.precond_op(slabs, outs, ins, tmps, tr, pc, dag)
            got = dd.unpack_slabs(slabs, outs, 0)
            assert torch.equal(got, tmq.unpack(g, out, 0)), (R, pc, dag)
            ref = orc.apply_M_pc(po, U, orc.project_parity(po, psi, 0), sym=bool(pc), dagger=dag)
            assert rel(got.cpu().numpy(), ref) < TOL[prec]
        for s in slabs:
            s.close()
    g.close()

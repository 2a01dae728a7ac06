"""Clover-twisted-mass operators through the C ABI against the numpy oracle (oracle/clover.py).

Element-by-element comparison of unpacked outputs on the same seeded inputs: FP64 1e-13, FP32
1e-6, FP16 (spinors and clover blocks) 5e-3 per application; solvers by the full-system residual
recomputed by the oracle.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import clover as cl
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {8: 1e-13, 4: 1e-6, 2: 5e-3}
CSW = 1.6
# (name, L, flavor, kappa, mu, eps): ragged tails, L = 2 extents, both flavour signs, doublet
CASES = [
    ("plus_4x4x4x6", (4, 4, 4, 6), 1, 0.1612, 0.004, 0.0),
    ("minus_2x4x6x4", (2, 4, 6, 4), -1, 0.1612, 0.01, 0.0),
    ("nd_6x4x2x10", (6, 4, 2, 10), 2, 0.1612, 0.135, 0.15),
]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


_cache = {}


def setup(case, recon=12):
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = case
    key = (name, recon)
    if key not in _cache:
        p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=recon)
        po = orc.Params(L, kappa, mu, eps, flavor=flavor)
        U = inputs.gauge_field(L, 1900 + len(name))
        g = tmq.Gauge(p, torch.from_numpy(U))
        tmq.set_clover(g, CSW)
        psi = inputs.spinor_field(L, p.nf, 2900 + len(name))
        _cache[key] = (tmq, p, po, U, g, psi)
    return _cache[key]


def get(tmq, g, f, parity):
    return tmq.unpack(g, f, parity).cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [8, 4, 2])
@pytest.mark.parametrize("recon", [18, 12])
def test_preconditioned_operators(case, prec, recon):
    tmq, p, po, U, g, psi = setup(case, recon)
    xe = tmq.pack(g, torch.from_numpy(psi), 0, prec)
    pe = orc.project_parity(po, psi, 0)
    for sym in (0, 1):
        for dag in (False, True):
            out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
            tmq.precond_op(g, out, xe, tmp, sym, dag)
            ref = cl.apply_M_pc(po, U, CSW, pe, sym=bool(sym), dagger=dag)
            assert rel(get(tmq, g, out, 0), ref) < TOL[prec], (sym, dag)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [8, 4, 2])
def test_full_operator_rhs_and_reconstruction(case, prec):
    tmq, p, po, U, g, psi = setup(case)
    t = torch.from_numpy(psi)
    xe, xo = tmq.pack(g, t, 0, prec), tmq.pack(g, t, 1, prec)
    for dag in (False, True):
        oe, oo = tmq.Field(g, prec), tmq.Field(g, prec)
        tmq.mat(g, oe, oo, xe, xo, dag)
        got = get(tmq, g, oe, 0) + get(tmq, g, oo, 1)
        assert rel(got, cl.apply_M(po, U, CSW, psi, dagger=dag)) < TOL[prec], dag
        for sym in (0, 1):
            bp = tmq.Field(g, prec)
            tmq.prepare_rhs(g, bp, xe, xo, sym, dag)
            assert rel(get(tmq, g, bp, 0), cl.prepare_rhs(po, U, CSW, psi, bool(sym), dag)) < TOL[prec], (sym, dag)
        ro = tmq.Field(g, prec)
        tmq.reconstruct_odd(g, ro, xo, xe, dag)
        ref = cl.reconstruct_odd(po, U, CSW, orc.project_parity(po, psi, 0), psi, dag)
        assert rel(get(tmq, g, ro, 1), ref) < TOL[prec], dag


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [8, 4, 2])
def test_local_operator(case, prec):
    tmq, p, po, U, g, psi = setup(case)
    t = torch.from_numpy(psi)
    for parity in (0, 1):
        x = tmq.pack(g, t, parity, prec)
        px = orc.project_parity(po, psi, parity)
        for inverse in (False, True):
            for dag in (False, True):
                out = tmq.Field(g, prec)
                tmq.local_op(g, out, x, parity, inverse, dag)
                Lm = cl.local_matrix(po, U, CSW, inverse=inverse, dagger=dag)
                ref = orc.project_parity(po, cl.apply_local(po, Lm, px), parity)
                assert rel(get(tmq, g, out, parity), ref) < TOL[prec], (parity, inverse, dag)


def full_solve(tmq, g, b, pc, dagger, **kw):
    be, bo = tmq.pack(g, torch.from_numpy(b), 0, 8), tmq.pack(g, torch.from_numpy(b), 1, 8)
    bp = tmq.Field(g, 8)
    tmq.prepare_rhs(g, bp, be, bo, pc, dagger)
    xe = tmq.Field(g, 8)
    st = tmq.solve(g, xe, bp, pc=pc, dagger=dagger, **kw)
    if pc == 1 and dagger:  # right-preconditioned: the unknown is L_ee^dag psi_e
        t = tmq.Field(g, 8)
        tmq.local_op(g, t, xe, 0, inverse=True, dagger=True)
        xe = t
    xo = tmq.Field(g, 8)
    tmq.reconstruct_odd(g, xo, bo, xe, dagger)
    return tmq.unpack(g, xe, 0).cpu().numpy() + tmq.unpack(g, xo, 1).cpu().numpy(), st


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
def test_fp64_cg_solves_the_full_system(case, pc, dagger):
    tmq, p, po, U, g, b = setup(case)
    psi, st = full_solve(tmq, g, b, pc, dagger, solver="cg", tol=1e-12, maxiter=5000)
    assert st["status"] == 0 and st["true_residual"] <= 1e-12
    assert rel(cl.apply_M(po, U, CSW, psi, dagger=dagger), b) < 1e-8


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("sloppy", [4, 2], ids=["f32", "f16"])
def test_mixed_cg_reaches_fp64_tolerance(case, sloppy):
    tmq, p, po, U, g, b = setup(case)
    psi, st = full_solve(tmq, g, b, 0, False, solver="mixed", sloppy_prec=sloppy, tol=1e-10, maxiter=5000)
    assert st["status"] == 0 and st["true_residual"] <= 1e-10 and st["reliable_updates"] >= 1
    assert rel(cl.apply_M(po, U, CSW, psi), b) < 1e-6


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("minb", [1, 3, 4, 6])
def test_occupancy_forms(case, minb):
    tmq, p, po, U, g, psi = setup(case)
    saved = tmq.tune_export(g)
    tmq.tune_import(g, f"f64:c:{minb} f32:c:{minb} f16:c:{minb}")
    try:
        pe = orc.project_parity(po, psi, 0)
        for prec in (8, 4, 2):
            xe = tmq.pack(g, torch.from_numpy(psi), 0, prec)
            for sym in (0, 1):
                out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
                tmq.precond_op(g, out, xe, tmp, sym, False)
                assert rel(get(tmq, g, out, 0), cl.apply_M_pc(po, U, CSW, pe, sym=bool(sym))) < TOL[prec]
    finally:
        tmq.tune_import(g, saved)


def test_autotune_on_a_clover_handle():
    tmq, p, po, U, g, psi = setup(CASES[2])
    table = tmq.autotune(g)
    clov = [e for e in table.split() if e.split(":")[1] == "c"]
    assert len(clov) == 3
    xe = tmq.pack(g, torch.from_numpy(psi), 0, 4)
    out, tmp = tmq.Field(g, 4), tmq.Field(g, 4)
    tmq.precond_op(g, out, xe, tmp, 0, False)
    assert rel(get(tmq, g, out, 0), cl.apply_M_pc(po, U, CSW, orc.project_parity(po, psi, 0))) < TOL[4]


def test_removing_the_clover_term_restores_twisted_mass():
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = CASES[2]
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1950)
    psi = inputs.spinor_field(L, 2, 2950)
    g = tmq.Gauge(p, torch.from_numpy(U))
    xe = tmq.pack(g, torch.from_numpy(psi), 0, 8)
    pe = orc.project_parity(po, psi, 0)
    out, tmp = tmq.Field(g, 8), tmq.Field(g, 8)
    tmq.set_clover(g, 1.2)
    tmq.precond_op(g, out, xe, tmp, 0, False)
    assert rel(get(tmq, g, out, 0), cl.apply_M_pc(po, U, 1.2, pe)) < 1e-13
    tmq.set_clover(g, 0.0)
    tmq.precond_op(g, out, xe, tmp, 0, False)
    assert rel(get(tmq, g, out, 0), orc.apply_M_pc(po, U, pe)) < 1e-13
    g.close()


def test_unsupported_combinations_are_rejected():
    tmq, p, po, U, g, psi = setup(CASES[0])
    t = torch.from_numpy(psi)
    # DF64 fields
    xd = tmq.pack(g, t, 0, 16)
    with pytest.raises(tmq.TMError):
        tmq.precond_op(g, tmq.Field(g, 16), xd, tmq.Field(g, 16), 0, False)
    # multi-RHS fields
    x2 = tmq.pack(g, torch.stack([t, t]), 0, 4, nrhs=2)
    with pytest.raises(tmq.TMError):
        tmq.precond_op(g, tmq.Field(g, 4, 2), x2, tmq.Field(g, 4, 2), 0, False)
    # the constant-twist call and the force
    x = tmq.pack(g, t, 0, 8)
    with pytest.raises(tmq.TMError):
        tmq.twist(g, tmq.Field(g, 8), x)
    xo = tmq.pack(g, t, 1, 8)
    with pytest.raises(tmq.TMError):
        tmq.force(g, x, xo, x, xo)
    with pytest.raises(tmq.TMError):
        tmq.set_clover(g, float("nan"))
    # the handle still works after the rejected calls
    out, tmp = tmq.Field(g, 8), tmq.Field(g, 8)
    tmq.precond_op(g, out, x, tmp, 0, False)
    ref = cl.apply_M_pc(po, U, CSW, orc.project_parity(po, psi, 0))
    assert rel(get(tmq, g, out, 0), ref) < 1e-13

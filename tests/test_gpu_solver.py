"""CG solvers through the C ABI against the oracle (solutions) and against the full operator (residuals).

Several x satisfy a solver tolerance, so solver parity is stated as closeness to the oracle's
tightly converged solution within a condition-number margin, plus the full-system residual
|M psi - b| / |b| recomputed by the oracle in FP64.
"""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("deg_4^4", (4, 4, 4, 4), 1, 0.1612, 0.004, 0.0),
    ("nd_6x4x2x10", (6, 4, 2, 10), 2, 0.1612, 0.135, 0.15),
    ("minus_4x4x4x8", (4, 4, 4, 8), -1, 0.1612, 0.01, 0.0),
]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


_cache = {}


def setup(case):
    import paper_1311_4462_gb300 as tmq
    name = case[0]
    if name not in _cache:
        _, L, flavor, kappa, mu, eps = case
        p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
        po = orc.Params(L, kappa, mu, eps, flavor=flavor)
        U = inputs.gauge_field(L, 1100 + len(name))
        g = tmq.Gauge(p, torch.from_numpy(U))
        b = inputs.spinor_field(L, p.nf, 2200 + len(name))
        _cache[name] = (tmq, p, po, U, g, b)
    return _cache[name]


def full_solve(tmq, g, b, pc, dagger, **kw):
    be, bo = tmq.pack(g, torch.from_numpy(b), 0, 8), tmq.pack(g, torch.from_numpy(b), 1, 8)
    bp = tmq.Field(g, 8)
    tmq.prepare_rhs(g, bp, be, bo, pc, dagger)
    xe = tmq.Field(g, 8)
    st = tmq.solve(g, xe, bp, pc=pc, dagger=dagger, **kw)
    if pc == 1 and dagger:  # right-preconditioned: the unknown is R_ee^dag psi_e
        t = tmq.Field(g, 8)
        tmq.twist(g, t, xe, inverse=True, dagger=True)
        xe = t
    xo = tmq.Field(g, 8)
    tmq.reconstruct_odd(g, xo, bo, xe, dagger)
    psi = tmq.unpack(g, xe, 0).cpu().numpy() + tmq.unpack(g, xo, 1).cpu().numpy()
    return psi, st


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
def test_fp64_cg_full_system(case, pc, dagger):
    tmq, p, po, U, g, b = setup(case)
    psi, st = full_solve(tmq, g, b, pc, dagger, solver="cg", tol=1e-12, maxiter=5000)
    assert st["status"] == 0 and st["true_residual"] <= 1e-12
    # |b - A x| <= cond(A) * tol * |b| for a normal-equation residual tol; margin cond <= 1e4 here
    res = rel(orc.apply_M(po, U, psi, dagger=dagger), b)
    assert res < 1e-8, res


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_cg_matches_oracle_cg(case):
    tmq, p, po, U, g, b = setup(case)
    be = tmq.pack(g, torch.from_numpy(b), 0, 8)
    xe = tmq.Field(g, 8)
    st = tmq.solve(g, xe, be, solution=tmq.TM_SOLUTION_MATDAG_MAT, tol=1e-12, maxiter=5000)
    x_ref, it, res = orc.cg_normal(po, U, orc.project_parity(po, b, 0), tol=1e-12, maxiter=20000)
    got = tmq.unpack(g, xe, 0).cpu().numpy()
    assert rel(got, x_ref) < 1e-7
    # same Krylov method, same arithmetic: iteration counts agree closely
    assert abs(st["iterations"] - it) <= max(3, it // 20)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("sloppy", [4, 2], ids=["f32", "f16"])
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
def test_mixed_cg_reaches_fp64_tolerance(case, sloppy, pc):
    tmq, p, po, U, g, b = setup(case)
    psi, st = full_solve(tmq, g, b, pc, False, solver="mixed", sloppy_prec=sloppy, tol=1e-10, maxiter=5000)
    assert st["status"] == 0 and st["true_residual"] <= 1e-10 and st["reliable_updates"] >= 1
    psi64, _ = full_solve(tmq, g, b, pc, False, solver="cg", tol=1e-12, maxiter=5000)
    assert rel(psi, psi64) < 1e-5
    assert rel(orc.apply_M(po, U, psi), b) < 1e-6


def test_noconv_status_and_stats():
    tmq, p, po, U, g, b = setup(CASES[0])
    be = tmq.pack(g, torch.from_numpy(b), 0, 8)
    xe = tmq.Field(g, 8)
    st = tmq.solve(g, xe, be, tol=1e-12, maxiter=3, check=False)
    assert st["status"] == -3 and st["iterations"] == 3 and st["true_residual"] > 1e-12


def test_nan_source_is_reported():
    tmq, p, po, U, g, b = setup(CASES[0])
    bad = b.copy()
    bad[0, 0, 0, 0, 0, 0, 0] = np.nan
    be = tmq.pack(g, torch.from_numpy(bad), 0, 8)
    xe = tmq.Field(g, 8)
    st = tmq.solve(g, xe, be, tol=1e-10, check=False)
    assert st["status"] == -4


def test_zero_source_gives_zero_solution():
    tmq, p, po, U, g, b = setup(CASES[1])
    be = tmq.pack(g, torch.zeros(p.spinor_shape, dtype=torch.complex128), 0, 8)
    xe = tmq.pack(g, torch.from_numpy(b), 0, 8)
    st = tmq.solve(g, xe, be, tol=1e-10)
    assert st["status"] == 0 and st["iterations"] == 0
    assert np.abs(tmq.unpack(g, xe, 0).cpu().numpy()).max() == 0.0


def test_initial_guess_is_used():
    tmq, p, po, U, g, b = setup(CASES[1])
    be = tmq.pack(g, torch.from_numpy(b), 0, 8)
    xe = tmq.Field(g, 8)
    st1 = tmq.solve(g, xe, be, tol=1e-10)
    st2 = tmq.solve(g, xe, be, tol=1e-10, use_x0=True)
    assert st2["iterations"] <= 1 < st1["iterations"]


def test_solver_is_deterministic():
    tmq, p, po, U, g, b = setup(CASES[1])
    be = tmq.pack(g, torch.from_numpy(b), 0, 8)
    outs = []
    for _ in range(2):
        xe = tmq.Field(g, 8)
        tmq.solve(g, xe, be, solver="mixed", sloppy_prec=2, tol=1e-10)
        outs.append(xe.data.clone())
    assert torch.equal(outs[0], outs[1])


def test_workspace_too_small_is_reported():
    tmq, p, po, U, g, b = setup(CASES[0])
    be = tmq.pack(g, torch.from_numpy(b), 0, 8)
    xe = tmq.Field(g, 8)
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    sp = tmq.solver_params()
    import ctypes
    from paper_1311_4462_gb300 import _lib as L
    st = L.tm_solver_stats()
    status = L.load().tm_solve(g.h, xe.ref(), be.ref(), ctypes.byref(sp), ctypes.byref(st),
                               ctypes.c_void_p(ws.data_ptr()), 1024, None)
    assert status == L.TM_ERR_NOMEM


@pytest.mark.parametrize("prec", [8, 4, 2])
def test_norm_and_dot_reductions(prec):
    tmq, p, po, U, g, b = setup(CASES[1])
    c = inputs.spinor_field(p.L, p.nf, 2300)
    fb, fc = tmq.pack(g, torch.from_numpy(b), 0, prec), tmq.pack(g, torch.from_numpy(c), 0, prec)
    bb = tmq.unpack(g, fb, 0).cpu().numpy()
    cc = tmq.unpack(g, fc, 0).cpu().numpy()
    tol = 1e-14 if prec == 8 else 1e-6
    assert abs(tmq.norm2(g, fb) - np.vdot(bb, bb).real) / np.vdot(bb, bb).real < tol
    d = np.vdot(bb, cc).real
    assert abs(tmq.dot(g, fb, fc) - d) / (np.linalg.norm(bb) * np.linalg.norm(cc)) < tol


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("solver,sloppy", [("cg", 4), ("mixed", 4), ("mixed", 2)])
def test_df64_true_precision(case, solver, sloppy):
    """Solution accumulation and true residual in double-float: same solutions as the FP64 solver."""
    tmq, p, po, U, g, b = setup(case)
    for pc in (0, 1):
        psi, st = full_solve(tmq, g, b, pc, False, solver=solver, sloppy_prec=sloppy, tol=1e-10, maxiter=5000,
                             true_prec=tmq.TM_PREC_DF64)
        assert st["status"] == 0 and st["true_residual"] <= 1e-10
        psi64, _ = full_solve(tmq, g, b, pc, False, solver="cg", tol=1e-12, maxiter=5000)
        assert rel(psi, psi64) < 1e-6
        assert rel(orc.apply_M(po, U, psi), b) < 1e-6


def test_df64_cg_to_1e12():
    """A whole CG in DF64 reaches an FP64-level tolerance."""
    tmq, p, po, U, g, b = setup(CASES[1])
    psi, st = full_solve(tmq, g, b, 0, False, solver="cg", tol=1e-12, maxiter=5000, true_prec=tmq.TM_PREC_DF64)
    assert st["status"] == 0 and st["true_residual"] <= 1e-12
    assert rel(orc.apply_M(po, U, psi), b) < 1e-8


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
@pytest.mark.parametrize("sloppy", [4, 2], ids=["f32", "f16"])
def test_fused_pap_matches_the_separate_reduction(case, pc, sloppy):
    """<p, A^dag A p> and the residual update r -= alpha A^dag A p with |r|^2 computed in the
    hopping epilogues (staged launch forms; A^dag A p never stored) or by separate passes
    (register-capped form): both mixed solves converge to the same solution in about the same
    number of iterations."""
    tmq, p, po, U, g, b = setup(case)
    name = {4: "f32", 2: "f16"}[sloppy]
    saved = tmq.tune_export(g)
    sols, its = [], []
    for table in (f"{name}:0:{8 if p.nf == 2 else 9}:128", f"{name}:0:3:128"):
        tmq.tune_import(g, table)
        psi, st = full_solve(tmq, g, b, pc, False, solver="mixed", sloppy_prec=sloppy, tol=1e-10, maxiter=5000)
        assert st["true_residual"] <= 1e-10
        assert rel(orc.apply_M(po, U, psi), b) < 1e-7
        sols.append(psi)
        its.append(st["iterations"])
    tmq.tune_import(g, saved)
    assert rel(sols[0], sols[1]) < 1e-7
    assert abs(its[0] - its[1]) <= max(2, its[1] // 20), its


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("solver", ["cg", "mixed"])
def test_f64_full_links_solve(case, solver):
    """A handle whose FP64 links keep 18 reals (TM_GAUGE_F64_FULL_LINKS, used for the FP64 true
    residuals) solves to the same tolerance and the same solution as the recon-12 handle."""
    tmq, p, po, U, g, b = setup(case)
    gf = tmq.Gauge(p, torch.from_numpy(U), f64_full_links=True)
    try:
        tmq.tune_import(gf, tmq.tune_export(g))
        psi_f, st_f = full_solve(tmq, gf, b, 0, False, solver=solver, tol=1e-10, maxiter=5000)
        psi, st = full_solve(tmq, g, b, 0, False, solver=solver, tol=1e-10, maxiter=5000)
        assert st_f["status"] == 0 and st_f["true_residual"] <= 1e-10
        assert rel(orc.apply_M(po, U, psi_f), b) < 1e-7
        assert rel(psi_f, psi) < 1e-7
        assert abs(st_f["iterations"] - st["iterations"]) <= 2
    finally:
        gf.close()

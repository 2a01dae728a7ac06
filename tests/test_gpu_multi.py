"""Multi-RHS operator, batched solver and the stochastic loop estimator against the oracle."""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {8: 1e-13, 4: 1e-6, 2: 5e-3}
CASES = [
    ("nd_6x4x2x10", (6, 4, 2, 10), 2, 0.1612, 0.135, 0.15),
    ("plus_4x4x4x6", (4, 4, 4, 6), 1, 0.1612, 0.004, 0.0),
]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(case, nrhs, recon=12):
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = case
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=recon)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1500)
    g = tmq.Gauge(p, torch.from_numpy(U))
    src = np.stack([inputs.spinor_field(L, p.nf, 2600 + k) for k in range(nrhs)])
    return tmq, p, po, U, g, src


B3 = (13, 15, 33, 35)  # FP16 staged multi-RHS forms with three buffers


RPB_IDS = {2: "rpb2", 4: "rpb4", 8: "rpb8", 12: "staged2", 14: "staged4", 16: "paired", 32: "staged2g",
           34: "staged4g", 36: "pairedg", 13: "staged2b3", 15: "staged4b3", 33: "staged2gb3", 35: "staged4gb3"}


def prec_rpb(rpbs):
    """(precision, form) pairs: every form for every precision, the three-buffer forms for FP16 only."""
    return [pytest.param(p, r, id=f"{p}-{RPB_IDS[r]}") for p in (8, 4, 2) for r in rpbs if r not in B3 or p == 2]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,rpb", prec_rpb([2, 4, 8, 12, 14, 16, 32, 34, 36, 13, 15, 33, 35]))
def test_multi_rhs_operators_match_oracle(case, prec, rpb):
    # not a multiple of any block shape: the last group of every shape is ragged; the paired-source
    # form (one flavour, two sources through the doublet's kernels) needs an even count
    nr = 6 if rpb in (16, 36) else 5
    tmq, p, po, U, g, src = make(case, nr)
    tmq.tune_import(g, f"f16:m:{rpb}" if rpb in B3 else f"f64:m:{rpb} f32:m:{rpb} f16:m:{rpb}")
    t = torch.from_numpy(src)
    xe, xo = tmq.pack(g, t, 0, prec, nrhs=nr), tmq.pack(g, t, 1, prec, nrhs=nr)
    for pc in (0, 1):
        for dag in (False, True):
            out, tmp = tmq.Field(g, prec, nr), tmq.Field(g, prec, nr)
            tmq.precond_op(g, out, xe, tmp, pc, dag)
            got = tmq.unpack(g, out, 0).cpu().numpy()
            for r in range(nr):
                ref = orc.apply_M_pc(po, U, orc.project_parity(po, src[r], 0), sym=bool(pc), dagger=dag)
                assert rel(got[r], ref) < TOL[prec], (pc, dag, r)
    oe, oo = tmq.Field(g, prec, nr), tmq.Field(g, prec, nr)
    tmq.mat(g, oe, oo, xe, xo)
    got = tmq.unpack(g, oe, 0).cpu().numpy() + tmq.unpack(g, oo, 1).cpu().numpy()
    for r in range(nr):
        assert rel(got[r], orc.apply_M(po, U, src[r])) < TOL[prec]
    bp, xr = tmq.Field(g, prec, nr), tmq.Field(g, prec, nr)
    tmq.prepare_rhs(g, bp, xe, xo, 0, False)
    tmq.reconstruct_odd(g, xr, xo, xe, False)
    gp, gr = tmq.unpack(g, bp, 0).cpu().numpy(), tmq.unpack(g, xr, 1).cpu().numpy()
    for r in range(nr):
        assert rel(gp[r], orc.prepare_rhs(po, U, src[r])) < TOL[prec]
        assert rel(gr[r], orc.reconstruct_odd(po, U, orc.project_parity(po, src[r], 0), src[r])) < TOL[prec]
    g.close()


def test_precond_op_active_subset_and_bad_index():
    nr = 6
    tmq, p, po, U, g, src = make(CASES[0], nr)
    t = torch.from_numpy(src)
    xe = tmq.pack(g, t, 0, 4, nrhs=nr)
    out, tmp = tmq.Field(g, 4, nr), tmq.Field(g, 4, nr)
    out.data.fill_(7)  # sentinel bytes in every right-hand side
    before = out.data.clone()
    tmq.precond_op_active(g, out, xe, tmp, [4, 1, 99, 3])  # 99 is outside nrhs: skipped
    got = tmq.unpack(g, out, 0).cpu().numpy()
    per = out.data.numel() // nr
    for r in range(nr):
        if r in (4, 1, 3):
            ref = orc.apply_M_pc(po, U, orc.project_parity(po, src[r], 0))
            assert rel(got[r], ref) < TOL[4]
        else:
            assert torch.equal(out.data[r * per:(r + 1) * per], before[r * per:(r + 1) * per])
    g.close()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("solver,sloppy,tp", [("cg", 8, 8), ("mixed", 4, 8), ("mixed", 2, 8), ("mixed", 2, 16),
                                              ("cg", 8, 16)])
@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_solve_multi_matches_single_solves(case, solver, sloppy, tp, graph):
    nr = 4
    tmq, p, po, U, g, src = make(case, nr)
    src[2] = 0.0                  # a zero source converges at iteration 0
    src[3] = 3.0 * src[0]          # a scaled copy needs the same iterations as source 0
    t = torch.from_numpy(src)
    be, bo = tmq.pack(g, t, 0, 8, nrhs=nr), tmq.pack(g, t, 1, 8, nrhs=nr)
    bp = tmq.Field(g, 8, nr)
    tmq.prepare_rhs(g, bp, be, bo, 0, False)
    xe = tmq.Field(g, 8, nr)
    kw = dict(solver=solver, tol=1e-10, maxiter=5000, use_graph=graph, true_prec=tp)
    if solver == "mixed":
        kw["sloppy_prec"] = sloppy
    status, stats = tmq.solve_multi(g, xe, bp, **kw)
    assert status == 0
    assert stats[2]["iterations"] == 0
    assert abs(stats[3]["iterations"] - stats[0]["iterations"]) <= 1
    xo = tmq.Field(g, 8, nr)
    tmq.reconstruct_odd(g, xo, bo, xe, False)
    psi = tmq.unpack(g, xe, 0).cpu().numpy() + tmq.unpack(g, xo, 1).cpu().numpy()
    for r in (0, 1, 3):
        assert stats[r]["true_residual"] <= 1e-10
        assert rel(orc.apply_M(po, U, psi[r]), src[r]) < 1e-6
    assert np.abs(psi[2]).max() == 0.0
    # same solution as a single-source FP64 solve
    b1 = tmq.Field(g, 8)
    tmq.prepare_rhs(g, b1, tmq.pack(g, t[1], 0, 8), tmq.pack(g, t[1], 1, 8), 0, False)
    x1 = tmq.Field(g, 8)
    tmq.solve(g, x1, b1, tol=1e-12, maxiter=5000)
    assert rel(tmq.unpack(g, xe, 0).cpu().numpy()[1], tmq.unpack(g, x1, 0).cpu().numpy()) < 1e-6
    g.close()


@pytest.mark.parametrize("prec", [8, 16, 4, 2])
def test_g5dot(prec):
    nr = 3
    tmq, p, po, U, g, src = make(CASES[0], nr)
    other = np.stack([inputs.spinor_field(p.L, p.nf, 2700 + k) for k in range(nr)])
    fa, fb = tmq.pack(g, torch.from_numpy(src), 0, prec, nrhs=nr), tmq.pack(g, torch.from_numpy(other), 0, prec, nrhs=nr)
    a, b = tmq.unpack(g, fa, 0).cpu().numpy(), tmq.unpack(g, fb, 0).cpu().numpy()
    got = tmq.g5dot(g, fa, fb)
    g5 = np.array([1, 1, -1, -1])[:, None]
    for r in range(nr):
        ref = np.vdot(a[r], (b[r] * g5))
        assert abs(got[r] - ref) / (np.linalg.norm(a[r]) * np.linalg.norm(b[r])) < (1e-14 if prec in (8, 16) else 1e-6)
    g.close()


def test_loop_estimator_against_dense_trace():
    """Tr[gamma5 M^-1] from Z2 noise through the batched solver vs the exact dense trace (4^4)."""
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import loops
    L = (4, 4, 4, 4)
    p = tmq.Params(L, 0.1612, 0.004, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    po = orc.Params(L, 0.1612, 0.004, 0.0, flavor=1)
    U = inputs.gauge_field(L, 1600)
    g = tmq.Gauge(p, torch.from_numpy(U))
    n = int(np.prod(p.spinor_shape))
    M = np.stack([orc.apply_M(po, U, np.eye(n, dtype=complex)[j].reshape(p.spinor_shape)).reshape(n)
                  for j in range(n)], axis=1)
    Minv = np.linalg.inv(M)
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), n // 12)
    exact = np.sum(g5 * np.diag(Minv))
    res = loops.g5_trace(g, nsources=32, batch=8, seed0=3000, tol=1e-10, solver="mixed",
                         sloppy_prec=tmq.TM_PREC_F16)
    # per-source values are exact for each noise vector up to the solver tolerance
    for k, val in enumerate(res["per_source"][:8]):
        eta = inputs.z2_noise_counter(L, 1, 3000 + k).reshape(n)
        ref = np.vdot(eta, g5 * (Minv @ eta))
        assert abs(val - ref) / abs(ref) < 1e-6
    # the estimate is unbiased: within 4 standard errors of the exact trace
    assert abs(res["estimate"] - exact) < 4 * res["stderr"] + 1e-12
    g.close()


@pytest.mark.parametrize("prec", [8, 16, 4, 2])
def test_device_noise_matches_counter_definition(prec):
    import paper_1311_4462_gb300 as tmq
    nr = 3
    tmq_, p, po, U, g, src = make(CASES[0], 1)
    fe, fo = tmq.Field(g, prec, nr), tmq.Field(g, prec, nr)
    tmq.noise_z2(g, fe, 0, 41)
    tmq.noise_z2(g, fo, 1, 41)
    got = tmq.unpack(g, fe, 0).cpu().numpy() + tmq.unpack(g, fo, 1).cpu().numpy()
    for r in range(nr):
        ref = inputs.z2_noise_counter(p.L, p.nf, 41 + r)
        if prec == 8:
            assert np.array_equal(got[r], ref)  # bit-exact
        elif prec == 16:
            assert np.abs(got[r] - ref).max() < 1e-15
        else:
            assert np.abs(got[r] - ref).max() < 1e-3
    g.close()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,rpb", prec_rpb([4, 14, 16, 34, 36, 15, 35]))
def test_multi_rhs_gives_the_single_rhs_bits(case, prec, rpb):
    """Every multi-RHS form (register, staged, paired sources, either block order) performs the same
    operations per source as the single-RHS forms, so each source's output has the same bits."""
    nr = 6
    tmq, p, po, U, g, src = make(case, nr)
    name = {8: "f64", 4: "f32", 2: "f16"}[prec]
    tmq.tune_import(g, f"{name}:m:{rpb}")
    t = torch.from_numpy(src)
    xe = tmq.pack(g, t, 0, prec, nrhs=nr)
    for pc in (0, 1):
        for dag in (False, True):
            out, tmp = tmq.Field(g, prec, nr), tmq.Field(g, prec, nr)
            tmq.precond_op(g, out, xe, tmp, pc, dag)
            got = tmq.unpack(g, out, 0)
            for r in range(nr):
                x1 = tmq.pack(g, t[r], 0, prec)
                o1, t1 = tmq.Field(g, prec), tmq.Field(g, prec)
                tmq.precond_op(g, o1, x1, t1, pc, dag)
                assert torch.equal(got[r], tmq.unpack(g, o1, 0)), (pc, dag, r)
    g.close()

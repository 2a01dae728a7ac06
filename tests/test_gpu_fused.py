"""The fused preconditioned operator (both passes of M_pc in one persistent launch, tune entry
"<prec>:p:1") against the two-launch form (the same per-site arithmetic, so the same bits) and
against the oracle; no bounded wait may give up."""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {8: 1e-13, 4: 1e-6}
# one tile, two tiles, ragged tails, several time slices per tile and several tiles per slice
CASES = [
    ("nd_2^4", (2, 2, 2, 2), 2, 0.16, 0.135, 0.15),
    ("plus_4x4x4x6", (4, 4, 4, 6), 1, 0.1612, 0.004, 0.0),
    ("nd_6x4x2x10", (6, 4, 2, 10), 2, 0.1612, 0.135, 0.15),
    ("minus_8x6x4x10", (8, 6, 4, 10), -1, 0.1612, 0.004, 0.0),
    ("nd_8x8x8x16", (8, 8, 8, 16), 2, 0.1612, 0.135, 0.15),
    ("plus_16x8x8x12", (16, 8, 8, 12), 1, 0.1612, 0.004, 0.0),
]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [8, 4])
def test_fused_matches_two_launches_and_oracle(case, prec):
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = case
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1600 + len(name))
    psi = inputs.spinor_field(L, p.nf, 2600 + len(name))
    g = tmq.Gauge(p, torch.from_numpy(U))
    xe = tmq.pack(g, torch.from_numpy(psi), 0, prec)
    pe = orc.project_parity(po, psi, 0)
    name_p = {8: "f64", 4: "f32"}[prec]
    for pc, dag in ((0, False), (0, True), (1, False), (1, True)):
        outs = []
        for fused in (0, 1):
            tmq.tune_import(g, f"{name_p}:p:{fused}")
            out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
            for _ in range(3):  # repeated applications reuse the work list and the flags
                tmq.precond_op(g, out, xe, tmp, pc, dag)
            tmq.device_status(g)
            outs.append(out.data.clone())
        assert torch.equal(outs[0], outs[1]), (pc, dag)
        got = tmq.unpack(g, out, 0).cpu().numpy()
        assert rel(got, orc.apply_M_pc(po, U, pe, sym=bool(pc), dagger=dag)) < TOL[prec]
    g.close()


def test_fused_inside_the_solvers():
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = CASES[4]
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1650)
    b = inputs.spinor_field(L, 2, 2650)
    g = tmq.Gauge(p, torch.from_numpy(U))
    tmq.tune_import(g, "f64:p:1 f32:p:1")
    t = torch.from_numpy(b)
    be, bo = tmq.pack(g, t, 0, 8), tmq.pack(g, t, 1, 8)
    bp = tmq.Field(g, 8)
    tmq.prepare_rhs(g, bp, be, bo, 0, False)
    for solver in ("cg", "mixed"):
        xe, xo = tmq.Field(g, 8), tmq.Field(g, 8)
        st = tmq.solve(g, xe, bp, solver=solver, sloppy_prec=4, tol=1e-10, maxiter=5000)
        tmq.device_status(g)
        assert st["status"] == 0 and st["true_residual"] <= 1e-10
        tmq.reconstruct_odd(g, xo, bo, xe, False)
        psi = tmq.unpack(g, xe, 0).cpu().numpy() + tmq.unpack(g, xo, 1).cpu().numpy()
        assert rel(orc.apply_M(po, U, psi), b) < 1e-7
    g.close()


def test_fused_at_the_benchmark_size():
    import paper_1311_4462_gb300 as tmq
    L = (32, 32, 32, 64)
    p = tmq.Params(L, 0.1612, 0.135, 0.15, flavor=tmq.TM_NDEG_DOUBLET, recon=12)
    U = inputs.gauge_field(L, 1002)
    psi = inputs.spinor_field(L, 2, 2002)
    g = tmq.Gauge(p, torch.from_numpy(U))
    xe = tmq.pack(g, torch.from_numpy(psi), 0, 4)
    outs = []
    for fused in (0, 1):
        tmq.tune_import(g, f"f32:p:{fused}")
        out, tmp = tmq.Field(g, 4), tmq.Field(g, 4)
        tmq.precond_op(g, out, xe, tmp, 0, False)
        tmq.device_status(g)
        outs.append(out.data.clone())
    assert torch.equal(outs[0], outs[1])
    g.close()

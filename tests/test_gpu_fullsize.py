"""Parity at the benchmark's full lattice sizes, in the launch configuration bench.py times.

* 32^3x64 doublet (kappa 0.1612, mu-bar 0.135, eps-bar 0.15): M_asym through the autotuned
  handle (the bench's headline step) against the oracle on every even site, FP32 / FP16 / FP64.
* 16^3x32 one flavour (kappa 0.1612, mu 0.004): FP64 CG to 1e-10 + odd reconstruction, the full
  system residual recomputed by the oracle.
* 32^3x64 one flavour: four sources through one multi-RHS operator launch, each against the oracle.
* 24^3x48 one flavour: the link force against the oracle's.
Each oracle application at these sizes takes a few seconds on the host cores.
"""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def nd_full():
    import paper_1311_4462_gb300 as tmq
    L = (32, 32, 32, 64)
    p = tmq.Params(L, 0.1612, 0.135, 0.15, flavor=tmq.TM_NDEG_DOUBLET, recon=12)
    po = orc.Params(L, 0.1612, 0.135, 0.15, flavor=2)
    U = inputs.gauge_field(L, 1002)
    psi = inputs.spinor_field(L, 2, 2002)
    g = tmq.Gauge(p, torch.from_numpy(U))
    tmq.autotune(g)
    ref = orc.apply_M_pc(po, U, orc.project_parity(po, psi, 0))
    yield tmq, g, psi, ref
    g.close()


@pytest.mark.parametrize("prec,tol", [(4, 1e-6), (2, 5e-3), (8, 1e-13)], ids=["f32", "f16", "f64"])
def test_headline_step_32x32x32x64_doublet(nd_full, prec, tol):
    tmq, g, psi, ref = nd_full
    xe = tmq.pack(g, torch.from_numpy(psi), 0, prec)
    tmp, out = tmq.Field(g, prec), tmq.Field(g, prec)
    # the two launches of the bench's step
    tmq.dslash(g, tmp, xe, 1, tmq.TM_EPI_TWINV)
    tmq.dslash(g, out, tmp, 0, tmq.TM_EPI_TWXPAY_ASYM, xe)
    got = tmq.unpack(g, out, 0).cpu().numpy()
    assert rel(got, ref) < tol
    # and tm_precond_op gives the same bits
    out2 = tmq.Field(g, prec)
    tmq.precond_op(g, out2, xe, tmp, tmq.TM_PC_ASYM, False)
    assert torch.equal(out.data, out2.data)


def test_fp64_solve_16x16x16x32_full_system_residual():
    import paper_1311_4462_gb300 as tmq
    L = (16, 16, 16, 32)
    p = tmq.Params(L, 0.1612, 0.004, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    po = orc.Params(L, 0.1612, 0.004, 0.0, flavor=1)
    U = inputs.gauge_field(L, 1001)
    b = inputs.spinor_field(L, 1, 2001)
    g = tmq.Gauge(p, torch.from_numpy(U))
    tb = torch.from_numpy(b)
    be, bo = tmq.pack(g, tb, 0, 8), tmq.pack(g, tb, 1, 8)
    bp = tmq.Field(g, 8)
    tmq.prepare_rhs(g, bp, be, bo, 0, False)
    xe, xo = tmq.Field(g, 8), tmq.Field(g, 8)
    st = tmq.solve(g, xe, bp, tol=1e-10, solver="cg")
    assert st["true_residual"] <= 1e-10
    tmq.reconstruct_odd(g, xo, bo, xe, False)
    psi = tmq.unpack(g, xe, 0).cpu().numpy() + tmq.unpack(g, xo, 1).cpu().numpy()
    assert rel(orc.apply_M(po, U, psi), b) < 1e-7
    g.close()


def test_multi_rhs_32x32x32x64_one_flavour():
    import paper_1311_4462_gb300 as tmq
    L = (32, 32, 32, 64)
    p = tmq.Params(L, 0.1612, 0.004, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    po = orc.Params(L, 0.1612, 0.004, 0.0, flavor=1)
    U = inputs.gauge_field(L, 1004)
    g = tmq.Gauge(p, torch.from_numpy(U))
    nr = 4
    fe = tmq.Field(g, 4, nr)
    tmq.noise_z2(g, fe, 0, 3000)
    out, tmp = tmq.Field(g, 4, nr), tmq.Field(g, 4, nr)
    tmq.precond_op(g, out, fe, tmp, 0, False)
    got = tmq.unpack(g, out, 0).cpu().numpy()
    for r in (0, 3):  # two of the four sources (each oracle call is a full-lattice application)
        eta = orc.project_parity(po, inputs.z2_noise_counter(L, 1, 3000 + r), 0)
        assert rel(got[r], orc.apply_M_pc(po, U, eta)) < 1e-6
    g.close()


def test_force_24x24x24x48():
    import paper_1311_4462_gb300 as tmq
    L = (24, 24, 24, 48)
    p = tmq.Params(L, 0.1612, 0.004, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    po = orc.Params(L, 0.1612, 0.004, 0.0, flavor=1)
    U = inputs.gauge_field(L, 1003)
    psi, gv = inputs.spinor_field(L, 1, 2003), inputs.spinor_field(L, 1, 2103)
    g = tmq.Gauge(p, torch.from_numpy(U))
    tp, tg = torch.from_numpy(psi), torch.from_numpy(gv)
    for prec, tol in ((8, 1e-13), (4, 2e-6)):
        F = tmq.force(g, tmq.pack(g, tp, 0, prec), tmq.pack(g, tp, 1, prec), tmq.pack(g, tg, 0, prec),
                      tmq.pack(g, tg, 1, prec), coef=1.0, project=True).cpu().numpy()
        if prec == 8:
            ref = orc.force(po, U, psi, gv, coef=1.0, project=True)
        assert rel(F, ref) < tol
    g.close()

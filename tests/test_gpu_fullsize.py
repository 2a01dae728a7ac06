"""Parity at the benchmark's full lattice sizes, in the launch configuration bench.py times.

* 32^3x64 doublet (kappa 0.1612, mu-bar 0.135, eps-bar 0.15): M_asym through the autotuned
  handle (the bench's headline step) against the oracle on every even site, FP32 / FP16 / FP64.
* 16^3x32 one flavour (kappa 0.1612, mu 0.004): FP64 CG to 1e-10 + odd reconstruction, the full
  system residual recomputed by the oracle.
* 32^3x64 one flavour: four sources through one multi-RHS operator launch, each against the oracle.
* 24^3x48 one flavour: the link force against the oracle's.
* 32^3x64 clover-twisted mass (both doublets): M_pc on 12 sampled sites against the one-site-at-a-time
  clover oracle.
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


@pytest.mark.parametrize("nf", [1, 2], ids=["one_flavour", "doublet"])
def test_clover_32x32x32x64_sampled_sites(nf):
    """TM-clover M_pc at the benchmark's lattice and launch configuration (autotuned handle, c_sw
    1.6), against the one-site-at-a-time clover oracle on 12 sampled even sites (including both
    time-boundary slices)."""
    import paper_1311_4462_gb300 as tmq
    from oracle import clover as cl
    L = (32, 32, 32, 64)
    mu, eps, flavor = (0.135, 0.15, 2) if nf == 2 else (0.004, 0.0, 1)
    p = tmq.Params(L, 0.1612, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, 0.1612, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1002)
    psi = inputs.spinor_field(L, nf, 2002)
    g = tmq.Gauge(p, torch.from_numpy(U))
    tmq.set_clover(g, 1.6)
    tmq.autotune(g)
    rng = np.random.default_rng(77)
    sites = []
    while len(sites) < 12:
        x, y, z = (int(v) for v in rng.integers(0, 32, size=3))
        t = [0, 63][len(sites)] if len(sites) < 2 else int(rng.integers(0, 64))
        if (x + y + z + t) % 2 == 0:
            sites.append((x, y, z, t))
    for sym in (False, True):
        ref = cl.apply_M_pc_at(po, U, 1.6, psi, sites, sym=sym)
        for prec, tol in ((4, 1e-6), (2, 5e-3), (8, 1e-13)):
            if sym and prec != 4:
                continue
            xe = tmq.pack(g, torch.from_numpy(psi), 0, prec)
            out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
            tmq.precond_op(g, out, xe, tmp, int(sym), False)
            got = tmq.unpack(g, out, 0).cpu().numpy()
            got = np.stack([got[t, z, y, x] for (x, y, z, t) in sites])
            assert rel(got, ref) < tol, (sym, prec, rel(got, ref))
    g.close()

"""Link force and autograd functions through the C ABI, against the oracle and finite differences."""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("deg_doublet_4^4", (4, 4, 4, 4), 2, 0.1612, 0.004, 0.0),
    ("nd_6x4x2x10", (6, 4, 2, 10), 2, 0.1612, 0.135, 0.15),
    ("plus_2x4x6x8", (2, 4, 6, 8), 1, 0.1612, 0.004, 0.0),
]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def su3_exp(H, h):
    w, V = np.linalg.eigh(H)
    return (V * np.exp(1j * h * w)[..., None, :]) @ np.conj(np.swapaxes(V, -1, -2))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [8, 4])
@pytest.mark.parametrize("recon", [18, 12, 8])
@pytest.mark.parametrize("project", [False, True])
def test_force_kernel_matches_oracle(case, prec, recon, project):
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = case
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=recon)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1300)
    psi, gv = inputs.spinor_field(L, p.nf, 2400), inputs.spinor_field(L, p.nf, 2401)
    g = tmq.Gauge(p, torch.from_numpy(U))
    tp, tg = torch.from_numpy(psi), torch.from_numpy(gv)
    F = tmq.force(g, tmq.pack(g, tp, 0, prec), tmq.pack(g, tp, 1, prec), tmq.pack(g, tg, 0, prec),
                  tmq.pack(g, tg, 1, prec), coef=0.7, project=project).cpu().numpy()
    ref = orc.force(po, U, psi, gv, coef=0.7, project=project)
    assert rel(F, ref) < (1e-13 if prec == 8 else 2e-6)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64], ids=["f64", "f32"])
def test_tmapply_autograd(dtype):
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300.autograd import TMApply
    name, L, flavor, kappa, mu, eps = CASES[1]
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1301)
    psi, gy = inputs.spinor_field(L, p.nf, 2402), inputs.spinor_field(L, p.nf, 2403)
    tU = torch.from_numpy(U).to("cuda").to(dtype).requires_grad_(True)
    tpsi = torch.from_numpy(psi).to("cuda").to(dtype).requires_grad_(True)
    y = TMApply.apply(tU, tpsi, p)
    tol = 1e-13 if dtype == torch.complex128 else 2e-6
    Ucast = tU.detach().cpu().numpy().astype(np.complex128)
    pcast = tpsi.detach().cpu().numpy().astype(np.complex128)
    assert rel(y.detach().cpu().numpy(), orc.apply_M(po, Ucast, pcast)) < tol
    y.backward(torch.from_numpy(gy).to("cuda").to(dtype))
    assert rel(tpsi.grad.cpu().numpy(), orc.apply_M(po, Ucast, gy, dagger=True)) < tol
    assert rel(tU.grad.cpu().numpy(), orc.force(po, Ucast, pcast, gy, coef=1.0, project=True)) < tol * 5


def test_tmapply_gradient_finite_differences():
    """d/dh Re<g, M(e^{ihw}U) psi> and d/dh Re<g, M(U)(psi + h v)> match <grad, direction>."""
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300.autograd import TMApply
    name, L, flavor, kappa, mu, eps = CASES[0]
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=18)
    U = inputs.gauge_field(L, 1302)
    psi, gy = inputs.spinor_field(L, p.nf, 2404), inputs.spinor_field(L, p.nf, 2405)
    tU = torch.from_numpy(U).to("cuda").requires_grad_(True)
    tpsi = torch.from_numpy(psi).to("cuda").requires_grad_(True)
    tg = torch.from_numpy(gy).to("cuda")
    loss = torch.vdot(tg.reshape(-1), TMApply.apply(tU, tpsi, p).reshape(-1)).real
    loss.backward()
    w = inputs.su3_algebra_direction(U.shape[:-2], 5100)
    h = 1e-6

    def Lval(UU, pp):
        y = TMApply.apply(torch.from_numpy(UU).to("cuda"), torch.from_numpy(pp).to("cuda"), p)
        return torch.vdot(tg.reshape(-1), y.reshape(-1)).real.item()

    fd = (Lval(su3_exp(w, h) @ U, psi) - Lval(su3_exp(w, -h) @ U, psi)) / (2 * h)
    an = np.sum(np.conj(tU.grad.cpu().numpy()) * (1j * w @ U)).real
    assert abs(fd - an) / abs(fd) < 1e-6
    v = inputs.spinor_field(L, p.nf, 2406)
    fd = (Lval(U, psi + h * v) - Lval(U, psi - h * v)) / (2 * h)
    an = np.sum(np.conj(tpsi.grad.cpu().numpy()) * v).real
    assert abs(fd - an) / abs(fd) < 1e-6


def test_pseudofermion_force_vs_oracle():
    """S and its gradients against the oracle's own even-odd CG solves and force formula.

    (Finite differences of S itself are pinned on the CPU with dense solves; with iterative solves
    S(U +- h w) is only smooth to the solver tolerance, so it is not differenced here.)"""
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300.autograd import PseudofermionAction
    name, L, flavor, kappa, mu, eps = CASES[1]
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1303)
    phi = inputs.spinor_field(L, p.nf, 2407)
    tU = torch.from_numpy(U).to("cuda").requires_grad_(True)
    tphi = torch.from_numpy(phi).to("cuda").requires_grad_(True)
    S = PseudofermionAction.apply(tU, tphi, p, 1e-11)
    S.backward()

    def osolve(b, dagger):
        bp = orc.prepare_rhs(po, U, b, dagger=dagger)
        y = orc.apply_M_pc(po, U, bp, dagger=not dagger)
        xe, _, _ = orc.cg_normal(po, U, y, dagger=dagger, tol=1e-12, maxiter=50000)
        return xe + orc.reconstruct_odd(po, U, xe, b, dagger=dagger)
    Y = osolve(phi, True)
    X = osolve(Y, False)
    assert abs(S.item() - np.vdot(phi, X).real) / abs(S.item()) < 1e-8
    F_ref = orc.force(po, U, X, Y, coef=-2.0, project=True)
    assert rel(tU.grad.cpu().numpy(), F_ref) < 1e-6
    assert rel(tphi.grad.cpu().numpy(), 2 * X) < 1e-6


def test_autograd_reuses_the_handle_while_U_is_unchanged():
    """Repeated calls with the same, unmodified U share one gauge handle (the links are packed once);
    an in-place change of U makes a new one.  The upstream gradient scales the results."""
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import autograd as tag
    from paper_1311_4462_gb300.autograd import PseudofermionAction, TMApply
    name, L, flavor, kappa, mu, eps = CASES[1]
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    U = inputs.gauge_field(L, 1304)
    psi, phi = inputs.spinor_field(L, p.nf, 2408), inputs.spinor_field(L, p.nf, 2409)
    tU = torch.from_numpy(U).to("cuda").requires_grad_(True)
    tpsi = torch.from_numpy(psi).to("cuda")
    y1 = TMApply.apply(tU, tpsi, p)
    g1 = tag.gauge_for(tU, p, (tmq.TM_PREC_F64,))
    y2 = TMApply.apply(tU, tpsi, p)
    assert tag.gauge_for(tU, p, (tmq.TM_PREC_F64,)) is g1
    assert torch.equal(y1, y2)
    tphi = torch.from_numpy(phi).to("cuda").requires_grad_(True)
    S = PseudofermionAction.apply(tU, tphi, p, 1e-11)
    assert tag.gauge_for(tU, p, (tmq.TM_PREC_F64,)) is g1  # FP64 CG: the same FP64-only handle
    (0.5 * S).backward()
    gU_half, gphi_half = tU.grad.clone(), tphi.grad.clone()
    tU.grad, tphi.grad = None, None
    S = PseudofermionAction.apply(tU, tphi, p, 1e-11)
    S.backward()
    assert torch.allclose(2 * gU_half, tU.grad, rtol=1e-12, atol=0)
    assert torch.allclose(2 * gphi_half, tphi.grad, rtol=1e-12, atol=0)
    with torch.no_grad():
        tU.mul_(1.0)  # an in-place change bumps U's version: the cached links are stale
    assert tag.gauge_for(tU, p, (tmq.TM_PREC_F64,)) is not g1
    tag.clear_cache()


def test_handle_with_a_subset_of_link_precisions():
    """tm_gauge_create_ex packs only the masked storage forms; calls on the others are refused."""
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = CASES[1]
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1305)
    psi = inputs.spinor_field(L, p.nf, 2410)
    g = tmq.Gauge(p, torch.from_numpy(U), precs=(tmq.TM_PREC_F32,))
    xe = tmq.pack(g, torch.from_numpy(psi), 0, 4)
    out, tmp = tmq.Field(g, 4), tmq.Field(g, 4)
    tmq.precond_op(g, out, xe, tmp, 0, False)
    assert rel(tmq.unpack(g, out, 0).cpu().numpy(), orc.apply_M_pc(po, U, orc.project_parity(po, psi, 0))) < 1e-6
    x64 = tmq.pack(g, torch.from_numpy(psi), 0, 8)
    with pytest.raises(tmq.TMError) as e:
        tmq.precond_op(g, tmq.Field(g, 8), x64, tmq.Field(g, 8), 0, False)
    assert "no links" in str(e.value)
    with pytest.raises(tmq.TMError):
        tmq.set_clover(g, 1.0)  # the clover field is built from the FP64 links
    tmq.autotune(g)  # tunes the packed precision only
    g.close()


@pytest.mark.parametrize("recon", [12, 8])
def test_force_and_clover_with_full_fp64_links(recon):
    """TM_GAUGE_F64_FULL_LINKS: the FP64 force reads the 18-real FP64 links (the bits of an 18-real
    handle), the FP32 force the handle's recon, and the clover term builds from the FP64 links."""
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = CASES[1]
    U = inputs.gauge_field(L, 1306)
    psi, gv = inputs.spinor_field(L, 2, 2411), inputs.spinor_field(L, 2, 2412)
    tp, tg = torch.from_numpy(psi), torch.from_numpy(gv)
    hs = {"flag": tmq.Gauge(tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=recon), torch.from_numpy(U),
                            f64_full_links=True),
          "plain": tmq.Gauge(tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=recon), torch.from_numpy(U)),
          "r18": tmq.Gauge(tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=18), torch.from_numpy(U))}
    F = {}
    for k, g in hs.items():
        for prec in (8, 4):
            F[k, prec] = tmq.force(g, tmq.pack(g, tp, 0, prec), tmq.pack(g, tp, 1, prec), tmq.pack(g, tg, 0, prec),
                                   tmq.pack(g, tg, 1, prec), coef=0.7, project=True).cpu().numpy()
    assert np.array_equal(F["flag", 8], F["r18", 8])
    assert np.array_equal(F["flag", 4], F["plain", 4])
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    assert rel(F["flag", 8], orc.force(po, U, psi, gv, coef=0.7, project=True)) < 1e-13
    g = hs["flag"]
    tmq.set_clover(g, 1.6)
    x = tmq.pack(g, tp, 0, 8)
    out, tmp = tmq.Field(g, 8), tmq.Field(g, 8)
    tmq.precond_op(g, out, x, tmp, 0, False)
    ref = hs["r18"]
    tmq.set_clover(ref, 1.6)
    x18 = tmq.pack(ref, tp, 0, 8)
    out18, tmp18 = tmq.Field(ref, 8), tmq.Field(ref, 8)
    tmq.precond_op(ref, out18, x18, tmp18, 0, False)
    assert torch.equal(out.data, out18.data)
    for h in hs.values():
        h.close()

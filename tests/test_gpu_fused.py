"""The fused preconditioned operator (both passes of M_pc in one persistent launch, tune entry
"<prec>:p:1") against the two-launch form (the same per-site arithmetic, so the same bits) and
against the oracle; no bounded wait may give up on the handle's own work list.  A work list that
leaves out first-pass work makes the waits give up at their time limit: the failure is reported
(TM_ERR_TIMEOUT), never a hang, and the handle works normally afterwards."""
import ctypes
import time

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


def _without_first_pass_group(lib, L, group):
    Lc = (ctypes.c_int * 4)(*L)
    n = lib.tm_fused_work_list(Lc, 152, None, 0)
    buf = (ctypes.c_int * n)()
    assert lib.tm_fused_work_list(Lc, 152, buf, n) == n
    items = [v for v in buf if v != (group << 1)]
    assert len(items) == n - 1
    return (ctypes.c_int * len(items))(*items), len(items)


@pytest.mark.parametrize("prec", [8, 4])
def test_bounded_wait_gives_up_and_reports_timeout(prec):
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import _lib as Lb
    lib = Lb.load()
    L = (8, 8, 8, 8)  # 2048 even sites: 16 tiles of 128 sites = 4 work groups
    p = tmq.Params(L, 0.1612, 0.135, 0.15, flavor=tmq.TM_NDEG_DOUBLET, recon=12)
    U = inputs.gauge_field(L, 1660)
    psi = inputs.spinor_field(L, 2, 2660)
    g = tmq.Gauge(p, torch.from_numpy(U))
    name_p = {8: "f64", 4: "f32"}[prec]
    xe = tmq.pack(g, torch.from_numpy(psi), 0, prec)
    tmq.tune_import(g, f"{name_p}:p:0")
    ref, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
    tmq.precond_op(g, ref, xe, tmp, 0, False)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    items, n = _without_first_pass_group(lib, L, 1)
    assert lib.tm_fused_set_work_list(g.h, items, n, 200_000_000, stream) == Lb.TM_OK, Lb.last_error()
    tmq.tune_import(g, f"{name_p}:p:1")
    out = tmq.Field(g, prec)
    torch.cuda.synchronize()
    t0 = time.time()
    tmq.precond_op(g, out, xe, tmp, 0, False)  # second-pass sites next to group 1 wait for it
    with pytest.raises(tmq.TMError) as e:
        tmq.device_status(g)
    elapsed = time.time() - t0
    assert e.value.status == Lb.TM_ERR_TIMEOUT
    assert elapsed < 5.0, elapsed  # one 0.2 s limit, not one per waiting site
    tmq.device_status(g)  # the word was cleared by the read
    # a solve through the broken list reports the timeout instead of a result
    be, bo = tmq.pack(g, torch.from_numpy(psi), 0, 8), tmq.pack(g, torch.from_numpy(psi), 1, 8)
    bp, xs = tmq.Field(g, 8), tmq.Field(g, 8)
    tmq.prepare_rhs(g, bp, be, bo, 0, False)
    tmq.tune_import(g, "f64:p:1 f32:p:1")
    st = tmq.solve(g, xs, bp, solver="cg", tol=1e-10, maxiter=2, check=False)
    assert st["status"] == Lb.TM_ERR_TIMEOUT
    tmq.device_status(g)
    # the handle's own list restored: the fused operator gives the two-launch bits again
    assert lib.tm_fused_set_work_list(g.h, None, 0, 1_000_000_000, stream) == Lb.TM_OK
    tmq.tune_import(g, f"{name_p}:p:1")
    tmq.precond_op(g, out, xe, tmp, 0, False)
    tmq.device_status(g)
    assert torch.equal(out.data, ref.data)
    # entries naming no group, and lists longer than the handle's, are refused on the host
    bad = (ctypes.c_int * 1)(99 << 1)
    assert lib.tm_fused_set_work_list(g.h, bad, 1, 1_000_000_000, stream) == Lb.TM_ERR_ARG
    assert lib.tm_fused_set_work_list(g.h, items, 10 ** 6, 1_000_000_000, stream) == Lb.TM_ERR_ARG
    g.close()

"""Edge cases of the library: the largest right-hand-side count, one past it, zero fields, and the
smallest lattice, each against the oracle or the documented error."""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = (2, 2, 2, 4)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def handle(flavor=1, mu=0.004, eps=0.0):
    import paper_1311_4462_gb300 as tmq
    p = tmq.Params(L, 0.1612, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, 0.1612, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, 1800)
    return tmq, p, po, U, tmq.Gauge(p, torch.from_numpy(U))


@pytest.mark.parametrize("prec,tol", [(8, 1e-13), (4, 1e-6), (2, 5e-3)])
def test_64_right_hand_sides_in_one_launch(prec, tol):
    tmq, p, po, U, g = handle()
    nr = 64
    fe = tmq.Field(g, prec, nr)
    tmq.noise_z2(g, fe, 0, 5000)
    out, tmp = tmq.Field(g, prec, nr), tmq.Field(g, prec, nr)
    tmq.precond_op(g, out, fe, tmp, 0, False)
    got = tmq.unpack(g, out, 0).cpu().numpy()
    for r in (0, 31, 63):
        eta = orc.project_parity(po, inputs.z2_noise_counter(L, 1, 5000 + r), 0)
        assert rel(got[r], orc.apply_M_pc(po, U, eta)) < tol
    g.close()


def test_65_right_hand_sides_are_refused():
    tmq, p, po, U, g = handle()
    f = tmq.Field(g, 4, 65)
    out, tmp = tmq.Field(g, 4, 65), tmq.Field(g, 4, 65)
    with pytest.raises(tmq.TMError):
        tmq.precond_op(g, out, f, tmp, 0, False)
    b, x = tmq.Field(g, 8, 65), tmq.Field(g, 8, 65)
    with pytest.raises(tmq.TMError):
        tmq.solve_multi(g, x, b, tol=1e-8)
    g.close()


def test_zero_fields():
    tmq, p, po, U, g = handle(flavor=2, mu=0.135, eps=0.15)
    z = tmq.pack(g, torch.zeros(p.spinor_shape, dtype=torch.complex128), 0, 2)
    assert tmq.norm2(g, z) == 0.0
    out, tmp = tmq.Field(g, 2), tmq.Field(g, 2)
    tmq.precond_op(g, out, z, tmp, 1, True)
    assert tmq.norm2(g, out) == 0.0  # FP16 with a zero site norm stays exactly zero
    g.close()


def test_multi_rhs_solve_with_64_sources_and_one_zero_source():
    tmq, p, po, U, g = handle()
    nr = 64
    src = np.stack([inputs.z2_noise_counter(L, 1, 6000 + r) for r in range(nr)])
    src[5] = 0.0
    t = torch.from_numpy(src)
    be = tmq.pack(g, t, 0, 8, nrhs=nr)
    xe = tmq.Field(g, 8, nr)
    st, stats = tmq.solve_multi(g, xe, be, solver="mixed", sloppy_prec=4, tol=1e-10, maxiter=2000)
    assert st == 0
    assert stats[5]["iterations"] == 0
    got = tmq.unpack(g, xe, 0).cpu().numpy()
    assert np.abs(got[5]).max() == 0.0
    for r in (0, 63):
        y = orc.project_parity(po, src[r], 0)
        Ay = orc.apply_M_pc(po, U, y, dagger=True)
        x, _, _ = orc.cg_normal(po, U, Ay, tol=1e-13)
        # several x meet the tolerance; within the condition-number margin of this small system
        assert rel(got[r], x) < 1e-7
    g.close()

"""Pins for the clover-twisted-mass oracle (oracle/clover.py), independent of the CUDA path.

* c_sw = 0 reduces every operator to the C oracle's twisted-mass one.
* Free field: F = 0, so the clover term vanishes for any c_sw.
* Abelian fields U_mu(x) = exp(i theta_mu(x)) 1: each leaf equals the plaquette at its corner,
  so F_{mu nu}(x) = (i/4) sum over the four corners of sin(plaquette angle), a scalar formula;
  a constant field strength gives the closed form T = kappa c_sw sin(phi) sigma_{mu nu}.
* Gauge covariance of F and of M under a random SU(3) transformation.
* T is hermitian and commutes with gamma5; gamma5(tau1)-hermiticity of M; <x, M y> = <M^dag x, y>.
* Schur: the even-odd solve plus reconstruction solves the full system (dense LU on 2^4).
"""
import numpy as np
import pytest

import oracle as orc
from oracle import clover as cl
from paper_1311_4462_gb300 import inputs

L4 = (4, 4, 4, 4)
CASES = [("plus", 1, 0.16, 0.01, 0.0), ("minus", -1, 0.16, 0.01, 0.0), ("nd", 2, 0.1612, 0.135, 0.15)]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def params(case, L=L4):
    _, flavor, kappa, mu, eps = case
    return orc.Params(L, kappa, mu, eps, flavor=flavor)


def coords(L):
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return x, y, z, t


def abelian_links(L, theta):
    """U_mu(x) = exp(i theta[mu](x)) times the 3x3 identity."""
    return np.exp(1j * theta)[..., None, None] * np.eye(3)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_csw_zero_is_the_twisted_mass_operator(case):
    p = params(case)
    U = inputs.gauge_field(L4, 1700)
    psi = inputs.spinor_field(L4, p.nf, 2700)
    assert rel(cl.apply_M(p, U, 0.0, psi), orc.apply_M(p, U, psi)) < 1e-14
    assert rel(cl.apply_M(p, U, 0.0, psi, dagger=True), orc.apply_M(p, U, psi, dagger=True)) < 1e-14
    pe = orc.project_parity(p, psi, 0)
    for sym in (False, True):
        for dag in (False, True):
            assert rel(cl.apply_M_pc(p, U, 0.0, pe, sym, dag), orc.apply_M_pc(p, U, pe, sym, dag)) < 1e-14
            assert rel(cl.prepare_rhs(p, U, 0.0, psi, sym, dag), orc.prepare_rhs(p, U, psi, sym, dag)) < 1e-14
        assert rel(cl.reconstruct_odd(p, U, 0.0, pe, psi, sym), orc.reconstruct_odd(p, U, pe, psi, sym)) < 1e-14


def test_free_field_has_no_clover_term():
    p = params(CASES[2])
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4,) + L4[::-1] + (3, 3)).copy()
    assert np.abs(cl.field_strength(U)).max() == 0.0
    psi = inputs.spinor_field(L4, 2, 2701)
    assert rel(cl.apply_M(p, U, 1.7, psi), orc.apply_M(p, U, psi)) < 1e-15


def test_abelian_random_angles_match_the_corner_plaquette_formula():
    L = (4, 6, 4, 8)
    rng = np.random.default_rng(5)
    theta = rng.uniform(-np.pi, np.pi, size=(4,) + L[::-1])
    F = cl.field_strength(abelian_links(L, theta))

    def sh(a, mu, s):
        return np.roll(a, -s, axis={0: 3, 1: 2, 2: 1, 3: 0}[mu])

    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                assert np.abs(F[mu, nu]).max() == 0.0
                continue
            # plaquette angle with lower corner y, traversed mu first
            ang = theta[mu] + sh(theta[nu], mu, 1) - sh(theta[mu], nu, 1) - theta[nu]
            s = (np.sin(ang) + np.sin(sh(ang, mu, -1)) + np.sin(sh(sh(ang, mu, -1), nu, -1))
                 + np.sin(sh(ang, nu, -1)))
            expect = (0.25j * s)[..., None, None] * np.eye(3)
            assert np.abs(F[mu, nu] - expect).max() < 1e-14, (mu, nu)


@pytest.mark.parametrize("plane", [(0, 1), (2, 3), (1, 3)])
def test_constant_field_strength_closed_form(plane):
    mu, nu = plane
    L = (4, 6, 4, 8)
    ext = L  # extent of direction k is L[k]
    k = 1
    phi = 2 * np.pi * k / ext[nu]
    xs = coords(L)
    theta = np.zeros((4,) + L[::-1])
    theta[mu] = phi * xs[nu]  # U_mu(x) = exp(i phi x_nu): every plaquette of the plane has angle -phi
    U = abelian_links(L, theta)
    F = cl.field_strength(U)
    for a in range(4):
        for b in range(4):
            want = 0.0
            if (a, b) == (mu, nu):
                want = -1j * np.sin(phi)
            elif (a, b) == (nu, mu):
                want = 1j * np.sin(phi)
            assert np.abs(F[a, b] - want * np.eye(3)).max() < 1e-14
    p = params(CASES[0], L)
    csw = 1.3
    psi = inputs.spinor_field(L, 1, 2702)
    diff = cl.apply_M(p, U, csw, psi) - orc.apply_M(p, U, psi)
    # sigma_{mu nu} = (i/2)[g_mu, g_nu] = i g_mu g_nu for mu != nu (the gammas anticommute)
    sig = 1j * orc.gamma(mu) @ orc.gamma(nu)
    expect = p.kappa * csw * np.sin(phi) * np.einsum("st,...fta->...fsa", sig, psi)
    assert rel(diff, expect) < 1e-13


def test_sigma_is_hermitian_and_commutes_with_gamma5():
    g5 = orc.gamma(4)
    for mu in range(4):
        for nu in range(4):
            s = cl.sigma(mu, nu)
            assert np.abs(s - s.conj().T).max() < 1e-15
            assert np.abs(s @ g5 - g5 @ s).max() < 1e-15
            assert np.abs(s + cl.sigma(nu, mu)).max() < 1e-15


def test_clover_term_hermitian_block_diagonal_in_chirality():
    p = params(CASES[0])
    U = inputs.gauge_field(L4, 1701)
    T = cl.clover_term(p, U, 1.1)
    assert np.abs(T - np.conj(np.swapaxes(T, -1, -2))).max() < 1e-14
    G5 = np.kron(orc.gamma(4), np.eye(3))
    assert np.abs(T @ G5 - G5 @ T).max() < 1e-14
    assert np.abs(T).max() > 1e-2  # a rough field gives a clover term of order kappa c_sw


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gauge_covariance(case):
    p = params(case)
    U = inputs.gauge_field(L4, 1702)
    psi = inputs.spinor_field(L4, p.nf, 2703)
    Om = inputs.gauge_transform(L4, 1703)  # one random SU(3) matrix per site
    Up = np.stack([Om @ U[mu] @ cl.dag(cl.shift(Om, mu, 1)) for mu in range(4)])
    psip = np.einsum("...ab,...fsb->...fsa", Om, psi)
    F, Fp = cl.field_strength(U), cl.field_strength(Up)
    assert np.abs(Fp - Om @ F @ cl.dag(Om)).max() < 1e-13
    lhs = cl.apply_M(p, Up, 1.2, psip)
    rhs = np.einsum("...ab,...fsb->...fsa", Om, cl.apply_M(p, U, 1.2, psi))
    assert rel(lhs, rhs) < 1e-13


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_adjoints(case):
    p = params(case)
    U = inputs.gauge_field(L4, 1704)
    x = inputs.spinor_field(L4, p.nf, 2704)
    y = inputs.spinor_field(L4, p.nf, 2705)
    csw = 1.4
    lhs = np.vdot(x, cl.apply_M(p, U, csw, y))
    rhs = np.vdot(cl.apply_M(p, U, csw, x, dagger=True), y)
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(x) * np.linalg.norm(cl.apply_M(p, U, csw, y))
    xe, ye = orc.project_parity(p, x, 0), orc.project_parity(p, y, 0)
    for sym in (False, True):
        My = cl.apply_M_pc(p, U, csw, ye, sym)
        lhs = np.vdot(xe, My)
        rhs = np.vdot(cl.apply_M_pc(p, U, csw, xe, sym, dagger=True), ye)
        assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(xe) * np.linalg.norm(My)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gamma5_hermiticity(case):
    p = params(case)
    U = inputs.gauge_field(L4, 1705)
    psi = inputs.spinor_field(L4, p.nf, 2706)
    csw = 0.9
    g5 = orc.gamma(4)

    def G5(v):
        return np.einsum("st,...fta->...fsa", g5, v)

    if p.nf == 2:
        # M^dag = gamma5 tau1 M gamma5 tau1
        def S(v):
            return G5(v[..., ::-1, :, :])
        assert rel(cl.apply_M(p, U, csw, psi, dagger=True), S(cl.apply_M(p, U, csw, S(psi)))) < 1e-14
    else:
        # M(mu)^dag = gamma5 M(-mu) gamma5
        pm = orc.Params(p.L, p.kappa, -p.mu, 0.0, flavor=p.flavor)
        assert rel(cl.apply_M(p, U, csw, psi, dagger=True), G5(cl.apply_M(pm, U, csw, G5(psi)))) < 1e-14


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_even_odd_solve_solves_the_full_system(case):
    L = (2, 2, 2, 2)
    p = params(case, L)
    U = inputs.gauge_field(L, 1706)
    b = inputs.spinor_field(L, p.nf, 2707)
    csw = 1.5
    n = b.size
    # dense full operator, column by column
    M = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        M[:, j] = cl.apply_M(p, U, csw, e.reshape(b.shape)).ravel()
    psi = np.linalg.solve(M, b.ravel()).reshape(b.shape)
    for sym in (False, True):
        bp = cl.prepare_rhs(p, U, csw, b, sym)
        # dense solve of the even system
        even = orc.parity_mask(p, 0)[..., None, None, None] * np.ones(b.shape, bool)
        idx = np.flatnonzero(even.ravel())
        A = np.empty((idx.size, idx.size), dtype=np.complex128)
        for j, k in enumerate(idx):
            e = np.zeros(n, dtype=np.complex128)
            e[k] = 1.0
            A[:, j] = cl.apply_M_pc(p, U, csw, e.reshape(b.shape), sym).ravel()[idx]
        xe = np.zeros(n, dtype=np.complex128)
        xe[idx] = np.linalg.solve(A, bp.ravel()[idx])
        xe = xe.reshape(b.shape)
        assert rel(xe, orc.project_parity(p, psi, 0)) < 1e-12
        xo = cl.reconstruct_odd(p, U, csw, xe, b)
        assert rel(xe + xo, psi) < 1e-12


def test_cg_reaches_the_dense_solution():
    L = (2, 2, 2, 4)
    p = params(CASES[2], L)
    U = inputs.gauge_field(L, 1707)
    b = inputs.spinor_field(L, 2, 2708)
    csw = 1.1
    bp = cl.prepare_rhs(p, U, csw, b)
    y = cl.apply_M_pc(p, U, csw, bp, dagger=True)
    x, it, res = cl.cg_normal(p, U, csw, y, tol=1e-12)
    assert res < 1e-11 and it > 0
    psi = x + cl.reconstruct_odd(p, U, csw, x, b)
    assert rel(cl.apply_M(p, U, csw, psi), b) < 1e-9


@pytest.mark.parametrize("case", [CASES[0], CASES[2]], ids=["plus", "nd"])
def test_patch_oracle_matches_the_whole_lattice_oracle(case):
    """The one-site-at-a-time oracle used at full lattice sizes agrees with the whole-lattice one,
    including sites next to the antiperiodic time boundary and the periodic wraps."""
    L = (8, 10, 8, 12)
    p = params(case, L)
    U = inputs.gauge_field(L, 1710)
    psi = inputs.spinor_field(L, p.nf, 2710)
    pe = orc.project_parity(p, psi, 0)
    sites = [(0, 0, 0, 0), (7, 9, 0, 0), (1, 3, 2, 10), (6, 2, 4, 6), (3, 9, 7, 11), (2, 2, 2, 0), (7, 1, 1, 11)]
    for sym, dag in ((False, False), (True, False), (False, True), (True, True)):
        full = cl.apply_M_pc(p, U, 1.3, pe, sym=sym, dagger=dag)
        got = cl.apply_M_pc_at(p, U, 1.3, psi, sites, sym=sym, dagger=dag)
        want = np.stack([full[t, z, y, x] for (x, y, z, t) in sites])
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max(), (sym, dag)

"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the mathematics.

None of these re-types the oracle's loops: each compares it with an independent
route to the same number (momentum-space closed form, dense block algebra and LU
solves, a symmetry of the operator, finite differences of a scalar function).
A dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

# DeGrand-Rossi gamma matrices (gamma_1..gamma_4 <-> x, y, z, t), typed from the basis definition.
G = [
    np.array([[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]]),
    np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=complex),
    np.array([[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]]),
    np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=complex),
]
G5 = np.diag([1, 1, -1, -1]).astype(complex)
TAU1 = np.array([[0, 1], [1, 0]], dtype=complex)
TAU3 = np.diag([1, -1]).astype(complex)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ----------------------------------------------------------------------------- gamma algebra
def test_gamma_tables_match_basis_and_clifford():
    for mu in range(4):
        assert np.array_equal(orc.gamma(mu), G[mu])
        assert np.allclose(G[mu], G[mu].conj().T)
        for nu in range(4):
            anti = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.allclose(anti, 2 * (mu == nu) * np.eye(4))
    assert np.allclose(orc.gamma(4), G5)
    assert np.allclose(G[0] @ G[1] @ G[2] @ G[3], G5)


# ----------------------------------------------------------------------------- twist R
@pytest.mark.parametrize("flavor,mu,eps", [(2, 0.135, 0.15), (2, 0.004, 0.0), (1, 0.01, 0.0), (-1, 0.01, 0.0)])
def test_twist_matrix_and_inverse_closed_form(flavor, mu, eps):
    p = orc.Params((2, 2, 2, 2), kappa=0.1612, mu=mu, eps=eps, flavor=flavor)
    a, b = 2 * p.kappa * p.mu, 2 * p.kappa * p.eps
    if p.nf == 2:
        X = 1j * a * np.kron(TAU3, G5) + b * np.kron(TAU1, np.eye(4))
        det = 1 + a * a - b * b
    else:
        X = 1j * a * flavor * G5
        det = 1 + a * a
    R = np.eye(4 * p.nf) + X
    assert np.allclose(orc.twist_matrix(p), R, atol=1e-15)
    # X^2 = (b^2 - a^2) 1, so R^-1 = (1 - X) / (1 + a^2 - b^2)
    assert np.allclose(X @ X, (det - 1) * -np.eye(4 * p.nf), atol=1e-15)
    Rinv = orc.twist_matrix(p, inverse=True)
    assert np.allclose(Rinv, (np.eye(4 * p.nf) - X) / det, atol=1e-15)
    assert np.allclose(Rinv @ R, np.eye(4 * p.nf), atol=1e-15)
    assert np.allclose(orc.twist_matrix(p, dagger=True), R.conj().T, atol=1e-15)
    assert np.allclose(orc.twist_matrix(p, inverse=True, dagger=True), np.linalg.inv(R).conj().T, atol=1e-15)


def test_twist_singular_is_reported():
    # 1 + a^2 - b^2 = 0 with a = 0: b = 1, i.e. eps = 1 / (2 kappa)
    p = orc.Params((2, 2, 2, 2), kappa=0.125, mu=0.0, eps=4.0, flavor=2)
    with pytest.raises(ZeroDivisionError):
        orc.twist_matrix(p, inverse=True)


# ----------------------------------------------------------------------------- free field
def _plane_wave(L, p_mom, u):
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    ph = np.exp(1j * (p_mom[0] * x + p_mom[1] * y + p_mom[2] * z + p_mom[3] * t))
    return ph[..., None, None, None] * u[None, None, None, None]


@pytest.mark.parametrize("flavor,mu,eps,tbc", [(2, 0.135, 0.15, True), (1, 0.01, 0.0, True), (-1, 0.02, 0.0, False),
                                               (2, 0.004, 0.0, True)])
@pytest.mark.parametrize("dagger", [False, True])
def test_free_field_plane_wave_closed_form(flavor, mu, eps, tbc, dagger):
    """U = 1: M e^{ipx}u = [1 - 2k sum cos p + 2ik sum gamma sin p + 2ik mu g5 tau3 + 2k eps tau1] e^{ipx}u."""
    L = (4, 6, 2, 8)
    p = orc.Params(L, kappa=0.16, mu=mu, eps=eps, flavor=flavor, t_antiperiodic=tbc)
    U = np.zeros(p.gauge_shape, dtype=complex)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    g = inputs.rng(7)
    nf = p.nf
    for n in [(0, 0, 0, 0), (1, 2, 1, 3), (3, 5, 1, 7), (2, 1, 0, 4)]:
        pm = [2 * np.pi * n[i] / L[i] for i in range(3)]
        pm.append((2 * np.pi * n[3] + (np.pi if tbc else 0.0)) / L[3])
        u = g.standard_normal((nf, 4, 3)) + 1j * g.standard_normal((nf, 4, 3))
        psi = _plane_wave(L, pm, u)
        k = p.kappa
        sgn = -1.0 if dagger else 1.0
        Ms = (1 - 2 * k * sum(np.cos(q) for q in pm)) * np.eye(4) + sgn * 2j * k * sum(
            G[m] * np.sin(pm[m]) for m in range(4))
        if nf == 2:
            Mfull = np.kron(np.eye(2), Ms) + sgn * 2j * k * mu * np.kron(TAU3, G5) + 2 * k * eps * np.kron(TAU1, np.eye(4))
        else:
            Mfull = Ms + sgn * 2j * k * mu * flavor * G5
        ue = np.einsum("ij,jc->ic", Mfull, u.reshape(4 * nf, 3)).reshape(nf, 4, 3)
        expect = _plane_wave(L, pm, ue)
        got = orc.apply_M(p, U, psi, dagger=dagger)
        assert rel(got, expect) < 1e-13, n


# ----------------------------------------------------------------------------- dense brute force
def _dense(fn, shape):
    n = int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1.0
        cols.append(fn(e.reshape(shape)).reshape(n))
    return np.stack(cols, axis=1)


@pytest.fixture(scope="module")
def dense_nd():
    L = (2, 2, 2, 4)
    p = orc.Params(L, kappa=0.16, mu=0.135, eps=0.15, flavor=2)
    U = inputs.gauge_field(L, 1001)
    M = _dense(lambda v: orc.apply_M(p, U, v), p.spinor_shape)
    Md = _dense(lambda v: orc.apply_M(p, U, v, dagger=True), p.spinor_shape)
    return p, U, M, Md


def test_dense_adjoint_and_gamma5_tau1_hermiticity(dense_nd):
    p, U, M, Md = dense_nd
    assert rel(Md, M.conj().T) < 1e-15
    V = int(np.prod(p.L))
    g5t1 = np.kron(np.eye(V), np.kron(np.kron(TAU1, G5), np.eye(3)))
    assert rel(g5t1 @ M @ g5t1, M.conj().T) < 1e-15


def test_single_flavour_gamma5_hermiticity_and_doublet_split():
    L = (2, 2, 4, 2)
    U = inputs.gauge_field(L, 1002)
    pp = orc.Params(L, kappa=0.16, mu=0.01, flavor=1)
    pm = orc.Params(L, kappa=0.16, mu=0.01, flavor=-1)
    Mp = _dense(lambda v: orc.apply_M(pp, U, v), pp.spinor_shape)
    Mm = _dense(lambda v: orc.apply_M(pm, U, v), pm.spinor_shape)
    V = int(np.prod(L))
    g5 = np.kron(np.eye(V), np.kron(G5, np.eye(3)))
    assert rel(g5 @ Mp @ g5, Mm.conj().T) < 1e-15
    # the degenerate doublet (eps = 0) is diag(M(+mu), M(-mu)) in flavour
    pd = orc.Params(L, kappa=0.16, mu=0.01, eps=0.0, flavor=2)
    psi = inputs.spinor_field(L, 2, 2001)
    out = orc.apply_M(pd, U, psi)
    assert rel(out[..., 0:1, :, :], orc.apply_M(pp, U, psi[..., 0:1, :, :])) < 1e-15
    assert rel(out[..., 1:2, :, :], orc.apply_M(pm, U, psi[..., 1:2, :, :])) < 1e-15


def test_wilson_limit_is_gamma5_hermitian():
    L = (2, 4, 2, 2)
    p = orc.Params(L, kappa=0.13, mu=0.0, eps=0.0, flavor=1)
    U = inputs.gauge_field(L, 1003)
    M = _dense(lambda v: orc.apply_M(p, U, v), p.spinor_shape)
    V = int(np.prod(L))
    g5 = np.kron(np.eye(V), np.kron(G5, np.eye(3)))
    assert rel(g5 @ M @ g5, M.conj().T) < 1e-15
    assert rel(M, M.conj().T) > 1e-3  # not hermitian itself


def _eo_index(p, parity):
    m = orc.parity_mask(p, parity)
    idx = np.arange(int(np.prod(p.spinor_shape))).reshape(p.spinor_shape)
    return idx[m].reshape(-1)


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_complement_matches_dense_blocks(dense_nd, sym, dagger):
    """eq. 2.2 / 2.3 LHS == Schur complement of the dense M (R_ee^-1 times it for sym)."""
    p, U, M, Md = dense_nd
    e, o = _eo_index(p, 0), _eo_index(p, 1)
    A = Md if dagger else M
    S = A[np.ix_(e, e)] - A[np.ix_(e, o)] @ np.linalg.solve(A[np.ix_(o, o)], A[np.ix_(o, e)])
    if sym:
        Ree = A[np.ix_(e, e)]  # the even-even block of M is R_ee itself
        S = np.linalg.solve(Ree, S) if not dagger else S @ np.linalg.inv(Ree)
    n = M.shape[0]
    Spc = _dense(lambda v: orc.apply_M_pc(p, U, v, sym=sym, dagger=dagger), p.spinor_shape)
    assert rel(Spc[np.ix_(e, e)], S) < 1e-14
    # nothing leaks to odd sites
    assert np.abs(Spc[o, :]).max() == 0.0
    del n


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("dagger", [False, True])
def test_eo_solve_matches_dense_lu(dense_nd, sym, dagger):
    """prepare_rhs -> CG on the normal equations -> reconstruct_odd reproduces the dense solution of M psi = b."""
    p, U, M, Md = dense_nd
    b = inputs.spinor_field(p.L, 2, 2002)
    A = Md if dagger else M
    exact = np.linalg.solve(A, b.reshape(-1)).reshape(p.spinor_shape)
    bp = orc.prepare_rhs(p, U, b, sym=sym, dagger=dagger)
    y = orc.apply_M_pc(p, U, bp, sym=sym, dagger=not dagger)  # A^dag b'
    xe, it, res = orc.cg_normal(p, U, y, sym=sym, dagger=dagger, tol=1e-13, maxiter=5000)
    assert res < 1e-12 and it > 0
    if sym and dagger:  # right-preconditioned: the unknown is R_ee^dag psi_e
        xe = orc.twist(p, xe, inverse=True, dagger=True)
    xo = orc.reconstruct_odd(p, U, xe, b, dagger=dagger)
    psi = xe + xo
    assert rel(psi, exact) < 1e-10
    assert rel(orc.apply_M(p, U, psi, dagger=dagger), b) < 1e-10


def test_cg_normal_matches_dense_normal_solve(dense_nd):
    p, U, M, Md = dense_nd
    e = _eo_index(p, 0)
    y = orc.project_parity(p, inputs.spinor_field(p.L, 2, 2003), 0)
    S = _dense(lambda v: orc.apply_M_pc(p, U, v), p.spinor_shape)[np.ix_(e, e)]
    exact = np.linalg.solve(S.conj().T @ S, y.reshape(-1)[e])
    x, it, res = orc.cg_normal(p, U, y, tol=1e-13, maxiter=5000)
    assert rel(x.reshape(-1)[e], exact) < 1e-10


# ----------------------------------------------------------------------------- gauge covariance
@pytest.mark.parametrize("L,flavor", [((4, 4, 4, 4), 2), ((2, 4, 6, 8), 1), ((6, 2, 4, 4), -1)])
def test_gauge_covariance(L, flavor):
    p = orc.Params(L, kappa=0.16, mu=0.135, eps=0.15 if flavor == 2 else 0.0, flavor=flavor)
    U = inputs.gauge_field(L, 1004)
    psi = inputs.spinor_field(L, p.nf, 2004)
    Om = inputs.gauge_transform(L, 4004)  # [Lt, Lz, Ly, Lx, 3, 3]
    Up = np.empty_like(U)
    for mu in range(4):
        shift = 3 - mu  # array axis of direction mu in [Lt, Lz, Ly, Lx]
        Om_fwd = np.roll(Om, -1, axis=shift)  # Omega(x + mu)
        Up[mu] = Om @ U[mu] @ np.conj(np.swapaxes(Om_fwd, -1, -2))
    rot = lambda v: np.einsum("tzyxab,tzyxfsb->tzyxfsa", Om, v)
    lhs = orc.apply_M(p, Up, rot(psi))
    rhs = rot(orc.apply_M(p, U, psi))
    assert rel(lhs, rhs) < 1e-14
    # a perturbation that is not a gauge transformation must break it
    assert rel(orc.apply_M(p, Up, psi), orc.apply_M(p, U, psi)) > 1e-3


def test_adjoint_identity_random_vectors():
    L = (4, 4, 4, 4)
    p = orc.Params(L, kappa=0.16, mu=0.01, eps=0.0, flavor=2)
    U = inputs.gauge_field(L, 1000)
    x, y = inputs.spinor_field(L, 2, 2005), inputs.spinor_field(L, 2, 2006)
    # scale: |x| |M y|, the size of the terms whose sum the inner product is
    My = orc.apply_M(p, U, y)
    lhs = np.vdot(x, My)
    rhs = np.vdot(orc.apply_M(p, U, x, dagger=True), y)
    assert abs(lhs - rhs) / (np.linalg.norm(x) * np.linalg.norm(My)) < 1e-15
    for sym in (False, True):
        xe, ye = orc.project_parity(p, x, 0), orc.project_parity(p, y, 0)
        My = orc.apply_M_pc(p, U, ye, sym=sym)
        lhs = np.vdot(xe, My)
        rhs = np.vdot(orc.apply_M_pc(p, U, xe, sym=sym, dagger=True), ye)
        assert abs(lhs - rhs) / (np.linalg.norm(xe) * np.linalg.norm(My)) < 1e-15


def test_full_system_residual_after_reconstruct_4x4():
    L = (4, 4, 4, 4)
    p = orc.Params(L, kappa=0.16, mu=0.135, eps=0.15, flavor=2)
    U = inputs.gauge_field(L, 1000)
    b = inputs.spinor_field(L, 2, 2007)
    xs = []
    for sym in (False, True):
        bp = orc.prepare_rhs(p, U, b, sym=sym)
        y = orc.apply_M_pc(p, U, bp, sym=sym, dagger=True)
        xe, it, res = orc.cg_normal(p, U, y, sym=sym, tol=1e-12, maxiter=5000)
        psi = xe + orc.reconstruct_odd(p, U, xe, b)
        assert rel(orc.apply_M(p, U, psi), b) < 1e-10
        xs.append(xe)
    assert rel(xs[0], xs[1]) < 1e-9  # asym and sym PC solve for the same psi_e


# ----------------------------------------------------------------------------- force
def _su3_exp(H, h):
    w, V = np.linalg.eigh(H)
    return (V * np.exp(1j * h * w)[..., None, :]) @ np.conj(np.swapaxes(V, -1, -2))


def test_force_link_gradient_finite_differences():
    """d/dh Re<g, M(e^{ih w} U) psi> at h = 0 == Re sum tr(G^dag i w U), by central differences."""
    L = (4, 4, 4, 4)
    p = orc.Params(L, kappa=0.16, mu=0.01, eps=0.0, flavor=2)
    U = inputs.gauge_field(L, 1000)
    psi, g = inputs.spinor_field(L, 2, 2008), inputs.spinor_field(L, 2, 2009)
    Graw = orc.force(p, U, psi, g, project=False)
    Gp = orc.force(p, U, psi, g, project=True)
    # projected gradient lies in the tangent space: Gp U^dag anti-hermitian and traceless
    Z = Gp @ np.conj(np.swapaxes(U, -1, -2))
    assert np.abs(Z + np.conj(np.swapaxes(Z, -1, -2))).max() < 1e-12
    assert np.abs(np.trace(Z, axis1=-2, axis2=-1)).max() < 1e-12
    Lf = lambda UU: np.vdot(g, orc.apply_M(p, UU, psi)).real
    h = 1e-6
    for seed in range(3):
        w = inputs.su3_algebra_direction(U.shape[:-2], 5000 + seed)
        fd = (Lf(_su3_exp(w, h) @ U) - Lf(_su3_exp(w, -h) @ U)) / (2 * h)
        dU = 1j * w @ U
        an_raw = np.sum(np.conj(Graw) * dU).real
        an_proj = np.sum(np.conj(Gp) * dU).real
        assert abs(fd - an_raw) / abs(fd) < 1e-7
        assert abs(fd - an_proj) / abs(fd) < 1e-7
    # single-link directions, including a link across the antiperiodic time boundary
    for (mu, t, z, y, x) in [(3, 3, 1, 2, 0), (0, 0, 0, 0, 3), (2, 2, 3, 0, 1), (3, 0, 0, 0, 0)]:
        w = np.zeros(U.shape, dtype=complex)
        w[mu, t, z, y, x] = inputs.su3_algebra_direction((), 6000 + mu + t)
        fd = (Lf(_su3_exp(w, h) @ U) - Lf(_su3_exp(w, -h) @ U)) / (2 * h)
        an = np.sum(np.conj(Gp) * (1j * w @ U)).real
        assert abs(fd - an) < 1e-7 * max(1.0, abs(fd))


def test_pseudofermion_force_finite_differences():
    """S = phi^dag (M^dag M)^-1 phi: dS/dU from the link gradient with psi = X, g = -2 Y, X = (M^dag M)^-1 phi, Y = M X."""
    L = (2, 2, 2, 4)
    p = orc.Params(L, kappa=0.16, mu=0.135, eps=0.15, flavor=2)
    U = inputs.gauge_field(L, 1005)
    phi = inputs.spinor_field(L, 2, 2010)
    n = int(np.prod(p.spinor_shape))

    def S(UU):
        M = _dense(lambda v: orc.apply_M(p, UU, v), p.spinor_shape)
        return np.vdot(phi.reshape(n), np.linalg.solve(M.conj().T @ M, phi.reshape(n))).real

    M = _dense(lambda v: orc.apply_M(p, U, v), p.spinor_shape)
    X = np.linalg.solve(M.conj().T @ M, phi.reshape(n)).reshape(p.spinor_shape)
    Y = orc.apply_M(p, U, X)
    F = orc.force(p, U, X, Y, coef=-2.0, project=True)
    h = 1e-6
    for seed in range(2):
        w = inputs.su3_algebra_direction(U.shape[:-2], 7000 + seed)
        fd = (S(_su3_exp(w, h) @ U) - S(_su3_exp(w, -h) @ U)) / (2 * h)
        an = np.sum(np.conj(F) * (1j * w @ U)).real
        assert abs(fd - an) / abs(fd) < 1e-6

"""Plain FP64 CPU oracle for the twisted-mass operator with a clover (Sheikholeslami-Wohlert) term.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by ``tests/`` and by the
CPU-baseline leg of ``bench.py``; never by the product path.  It shares no code with the CUDA
path; the hopping term and the twist are the C oracle's (``oracle.hop``, ``oracle.twist_matrix``).

The paper names the combination of clover improvement with twisted mass as its next step
(Conclusion).  The clover term is the standard one, written here in the kappa normalisation of
eq. 2.1 (M = 2 kappa (D_W + m)):

  M = A + 2 i kappa mu gamma5 tau3 (+ 2 kappa eps tau1) - kappa H,      A = 1 + T,
  T(x) = i kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),      sigma_{mu nu} = (i/2)[g_mu, g_nu],
  F_{mu nu}(x) = (Q_{mu nu}(x) - Q_{mu nu}(x)^dag) / 8,
  Q_{mu nu}(x) = the sum of the four plaquettes of the mu-nu plane that start and end at x,
                 all traversed in the same sense (mu first, then nu).

T is hermitian and commutes with gamma5, so the local operator L = A + (R - 1) (R the twist of
eq. 2.1) is block diagonal in chirality; the oracle nevertheless assembles and inverts the whole
(flavour x spin x colour) matrix of every site with numpy, without using that structure.
Even-odd operators follow eq. 2.2-2.4 with R replaced by L:
  M_asym = L_ee - kappa^2 H_eo L_oo^-1 H_oe,   M_sym = 1 - kappa^2 L_ee^-1 H_eo L_oo^-1 H_oe.

Arrays: spinor complex128 [Lt, Lz, Ly, Lx, nf, 4, 3]; gauge complex128 [4, Lt, Lz, Ly, Lx, 3, 3]
(mu = 0..3 <-> x, y, z, t); the gauge field is periodic in every direction (the antiperiodic
time boundary belongs to the fermion hop only).
"""
from __future__ import annotations

import numpy as np

from . import Params, gamma, hop, parity_mask, twist_matrix

# lattice axis of each direction in [Lt, Lz, Ly, Lx] site arrays
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def shift(A, mu: int, s: int):
    """B(x) = A(x + s mu^) for an array whose first four axes are [Lt, Lz, Ly, Lx] (periodic)."""
    return np.roll(A, -s, axis=_AXIS[mu])


def dag(A):
    return np.conj(np.swapaxes(A, -1, -2))


def field_strength(U):
    """F[mu, nu] (complex [4, 4, Lt, Lz, Ly, Lx, 3, 3]) from the clover leaves; F[nu, mu] = -F[mu, nu]."""
    U = np.asarray(U, dtype=np.complex128)
    F = np.zeros((4, 4) + U.shape[1:], dtype=np.complex128)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Um, Un = U[mu], U[nu]
            # leaf at corner x:             x -> x+mu -> x+mu+nu -> x+nu -> x
            q = Um @ shift(Un, mu, 1) @ dag(shift(Um, nu, 1)) @ dag(Un)
            # leaf at corner x-mu:          x -> x+nu -> x-mu+nu -> x-mu -> x
            q = q + Un @ dag(shift(shift(Um, mu, -1), nu, 1)) @ dag(shift(Un, mu, -1)) @ shift(Um, mu, -1)
            # leaf at corner x-mu-nu:       x -> x-mu -> x-mu-nu -> x-nu -> x
            q = q + (dag(shift(Um, mu, -1)) @ dag(shift(shift(Un, mu, -1), nu, -1))
                     @ shift(shift(Um, mu, -1), nu, -1) @ shift(Un, nu, -1))
            # leaf at corner x-nu:          x -> x-nu -> x-nu+mu -> x+mu -> x
            q = q + dag(shift(Un, nu, -1)) @ shift(Um, nu, -1) @ shift(shift(Un, nu, -1), mu, 1) @ dag(Um)
            F[mu, nu] = (q - dag(q)) / 8.0
            F[nu, mu] = -F[mu, nu]
    return F


def sigma(mu: int, nu: int) -> np.ndarray:
    g = [gamma(k) for k in range(4)]
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def clover_term(p: Params, U, csw: float):
    """T(x) = i kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x), complex [Lt, Lz, Ly, Lx, 12, 12]
    with row / column index 3 s + c (spin s, colour c)."""
    F = field_strength(U)
    site = F.shape[2:6]
    T = np.zeros(site + (4, 3, 4, 3), dtype=np.complex128)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            T += np.einsum("st,...ab->...satb", sigma(mu, nu), F[mu, nu])
    return (1j * p.kappa * csw * T).reshape(site + (12, 12))


def local_matrix(p: Params, U, csw: float, inverse=False, dagger=False):
    """L(x) = 1 + T(x) + (R - 1) as a (flavour, spin, colour) matrix per site,
    complex [Lt, Lz, Ly, Lx, 12 nf, 12 nf]; optionally its adjoint and / or inverse."""
    T = clover_term(p, U, csw)
    nf = p.nf
    R = twist_matrix(p)                              # (4 nf) x (4 nf) in (flavour, spin)
    L = np.kron(R, np.eye(3))[None, None, None, None]  # (flavour, spin, colour) order
    L = L + np.einsum("fg,...ij->...figj", np.eye(nf), T).reshape(T.shape[:4] + (12 * nf, 12 * nf))
    if dagger:
        L = dag(L)
    if inverse:
        L = np.linalg.inv(L)
    return L


def apply_local(p: Params, L, psi):
    psi = np.asarray(psi, dtype=np.complex128)
    v = psi.reshape(psi.shape[:4] + (12 * p.nf,))
    return np.einsum("...ij,...j->...i", L, v).reshape(psi.shape)


def apply_M(p: Params, U, csw: float, psi, dagger=False):
    """Full operator M psi = L psi - kappa H psi (M^dag: L^dag psi - kappa H^dag psi)."""
    return apply_local(p, local_matrix(p, U, csw, dagger=dagger), psi) - p.kappa * hop(p, U, psi, dagger)


def _proj(p: Params, v, parity: int):
    return np.where(parity_mask(p, parity)[..., None, None, None], v, 0)


def apply_M_pc(p: Params, U, csw: float, psi, sym=False, dagger=False):
    """Even-odd Schur complement on the even sites (psi restricted to even sites)."""
    k2 = p.kappa * p.kappa
    ve = _proj(p, psi, 0)
    Li = local_matrix(p, U, csw, inverse=True, dagger=dagger)
    if sym and dagger:
        # M_sym^dag = 1 - kappa^2 H^dag_eo L_oo^-dag H^dag_oe L_ee^-dag
        t = _proj(p, hop(p, U, apply_local(p, Li, ve), True), 1)
        t = _proj(p, hop(p, U, apply_local(p, Li, t), True), 0)
        return ve - k2 * t
    t = _proj(p, hop(p, U, ve, dagger), 1)
    t = _proj(p, hop(p, U, apply_local(p, Li, t), dagger), 0)
    if sym:
        return ve - k2 * _proj(p, apply_local(p, Li, t), 0)
    L = local_matrix(p, U, csw, dagger=dagger)
    return _proj(p, apply_local(p, L, ve), 0) - k2 * t


def prepare_rhs(p: Params, U, csw: float, b, sym=False, dagger=False):
    """b'_e = b_e + kappa H_eo L_oo^-1 b_o (daggered with dagger); the symmetric, non-adjoint
    system takes L_ee^-1 b'_e (its adjoint is right-preconditioned, so b'_e is kept)."""
    Li = local_matrix(p, U, csw, inverse=True, dagger=dagger)
    t = _proj(p, hop(p, U, apply_local(p, Li, _proj(p, b, 1)), dagger), 0)
    bp = _proj(p, b, 0) + p.kappa * t
    if sym and not dagger:
        bp = _proj(p, apply_local(p, Li, bp), 0)
    return bp


def reconstruct_odd(p: Params, U, csw: float, psi_e, b, dagger=False):
    """psi_o = L_oo^-1 (b_o + kappa H_oe psi_e) (daggered with dagger)."""
    Li = local_matrix(p, U, csw, inverse=True, dagger=dagger)
    t = _proj(p, b, 1) + p.kappa * _proj(p, hop(p, U, _proj(p, psi_e, 0), dagger), 1)
    return _proj(p, apply_local(p, Li, t), 1)


def cg_normal(p: Params, U, csw: float, y, sym=False, dagger=False, tol=1e-12, maxiter=10000):
    """Plain CG on A^dag A x = y with A = M_pc (or M_pc^dag); returns (x, iterations, true residual)."""
    def A(v, d):
        return apply_M_pc(p, U, csw, v, sym=sym, dagger=d)

    def AA(v):
        return A(A(v, dagger), not dagger)

    y = _proj(p, y, 0)
    x = np.zeros_like(y)
    r = y.copy()
    q = r.copy()
    rr = np.vdot(r, r).real
    yy = np.vdot(y, y).real
    it = 0
    while it < maxiter and rr > tol * tol * yy:
        Aq = AA(q)
        alpha = rr / np.vdot(q, Aq).real
        x = x + alpha * q
        r = r - alpha * Aq
        rr_new = np.vdot(r, r).real
        q = r + (rr_new / rr) * q
        rr = rr_new
        it += 1
    res = np.linalg.norm(y - AA(x)) / np.linalg.norm(y)
    return x, it, float(res)


def apply_M_pc_at(p: Params, U, csw: float, psi, sites, sym=False, dagger=False, R=4):
    """(M_pc psi)(x) at the given even sites x = (x, y, z, t), one by one, for lattices too large
    for the whole-lattice oracle.  Each output depends only on psi within two hops and on links
    within three hops of x, so it is the output at the centre of the whole-lattice oracle applied
    to a 2R^4 patch (R = 4: coordinates x-4 ... x+3, periodic copy of the lattice around x).  The
    patch is periodic in every direction: the antiperiodic time boundary of the lattice is carried
    by negating U_t on its last time slice (every plaquette contains those links in pairs, so F is
    unchanged, and each hop across the boundary picks up the -1).  Returns complex
    [len(sites), nf, 4, 3]."""
    Lx, Ly, Lz, Lt = p.L
    n = 2 * R
    assert min(p.L) >= n, "the lattice must be at least as large as the patch"
    Ug = np.array(U, dtype=np.complex128, copy=True)
    if p.t_antiperiodic:
        Ug[3, Lt - 1] *= -1.0
    pp = Params((n, n, n, n), p.kappa, p.mu, p.eps, flavor=p.flavor, t_antiperiodic=False)
    out = []
    for (x, y, z, t) in sites:
        assert (x + y + z + t) % 2 == 0, "even sites only"
        it = (np.arange(n) + t - R) % Lt
        iz = (np.arange(n) + z - R) % Lz
        iy = (np.arange(n) + y - R) % Ly
        ix = (np.arange(n) + x - R) % Lx
        sl = np.ix_(it, iz, iy, ix)
        Up = np.stack([Ug[mu][sl] for mu in range(4)])
        ps = np.asarray(psi)[sl]
        r = apply_M_pc(pp, Up, csw, _proj(pp, ps, 0), sym=sym, dagger=dagger)
        out.append(r[R, R, R, R])
    return np.stack(out)

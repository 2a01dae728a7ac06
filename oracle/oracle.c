/*
 * oracle.c -- plain FP64 CPU oracle for the Wilson twisted-mass operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The CUDA product path never
 * calls it, and the two share no code, tables or headers.
 *
 * Everything here is the plain definition of the operators, written out as
 * loops over sites, directions, flavours, spins and colours with full 4x4
 * gamma matrices and explicit 3x3 link products.  There is no even-odd
 * index arithmetic: even-odd blocks are realised on full-lattice vectors by
 * zeroing the sites of the other parity, and the hopping term maps
 * even-supported vectors to odd-supported ones by construction.
 *
 * Conventions (the kappa normalisation of the twisted-mass operator):
 *   M psi(x) = R psi(x) - kappa * (H psi)(x)
 *   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                     + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)
 *   R = 1 + 2 i kappa mu gamma5 tau3 + 2 kappa eps tau1           (eq. 2.1)
 *   Gamma matrices in the DeGrand-Rossi chiral basis, gamma5 = g1 g2 g3 g4.
 *   Periodic in x, y, z; the hops across t = Lt-1 <-> 0 carry a factor -1
 *   when the time boundary is antiperiodic.
 *
 * Memory layout (shared with the tests only through plain numpy arrays):
 *   site s = x + Lx*(y + Ly*(z + Lz*t));
 *   spinor element (s, f, spin, colour) at ((s*nf + f)*4 + spin)*3 + colour;
 *   link element (mu, s, row, col) at ((mu*V + s)*3 + row)*3 + col.
 *
 * Functions whose parity against the paper is pinned by the CPU tests:
 *   orc_hop, orc_twist, orc_M            -- free-field closed form, dense
 *                                           brute force, gauge covariance,
 *                                           gamma5-tau1 hermiticity, adjoint
 *   orc_M_pc, orc_prepare_rhs,
 *   orc_reconstruct_odd                  -- Schur identity vs dense solve,
 *                                           full-system residual (eq. 2.2-2.4)
 *   orc_cg_normal                        -- dense LU solve
 *   orc_force                            -- central finite differences
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int L[4];      /* Lx, Ly, Lz, Lt */
    int nf;        /* 1 (single flavour) or 2 (doublet) */
    int fsign;     /* tau3 eigenvalue of the single flavour: +1 or -1 */
    int tbc;       /* 1: antiperiodic in t, 0: periodic */
    double kappa, mu, eps;
} orc_params;

/* ---- gamma matrices, DeGrand-Rossi basis; index 0..3 <-> x, y, z, t ---- */
static const cplx GAMMA[4][4][4] = {
    {{0, 0, 0, I}, {0, 0, I, 0}, {0, -I, 0, 0}, {-I, 0, 0, 0}},
    {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    {{0, 0, I, 0}, {0, 0, 0, -I}, {-I, 0, 0, 0}, {0, I, 0, 0}},
    {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
};

static void matmul4(const cplx a[4][4], const cplx b[4][4], cplx c[4][4])
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

/* gamma5 = gamma1 gamma2 gamma3 gamma4 */
static void gamma5(cplx g5[4][4])
{
    cplx t1[4][4], t2[4][4];
    matmul4(GAMMA[0], GAMMA[1], t1);
    matmul4(t1, GAMMA[2], t2);
    matmul4(t2, GAMMA[3], g5);
}

void orc_gamma(int mu, double *out_re_im)
{
    /* mu = 0..3 -> gamma_{mu+1}; mu = 4 -> gamma5.  Output 4x4 complex, row-major. */
    cplx g[4][4];
    if (mu == 4) gamma5(g);
    else memcpy(g, GAMMA[mu], sizeof(g));
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            out_re_im[2 * (4 * i + j)] = creal(g[i][j]);
            out_re_im[2 * (4 * i + j) + 1] = cimag(g[i][j]);
        }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static long volume(const orc_params *p)
{
    return (long)p->L[0] * p->L[1] * p->L[2] * p->L[3];
}

static long site_of(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

static void coords_of(const int L[4], long s, int c[4])
{
    c[0] = (int)(s % L[0]); s /= L[0];
    c[1] = (int)(s % L[1]); s /= L[1];
    c[2] = (int)(s % L[2]); s /= L[2];
    c[3] = (int)s;
}

/*
 * out = H in   (dagger = 0)   or   out = H^dag in   (dagger = 1).
 * H^dag has the two spin projectors exchanged: (1 + gamma_mu) with the
 * forward link and (1 - gamma_mu) with the backward link.
 */
void orc_hop(const orc_params *p, const cplx *U, const cplx *in, cplx *out, int dagger)
{
    const long V = volume(p);
    const int nf = p->nf;
    const double sg = dagger ? -1.0 : 1.0;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int c[4];
        coords_of(p->L, s, c);
        cplx acc[2][4][3];
        memset(acc, 0, sizeof(acc));
        for (int mu = 0; mu < 4; mu++) {
            for (int dir = 0; dir < 2; dir++) { /* 0: forward hop, 1: backward hop */
                int cn[4] = {c[0], c[1], c[2], c[3]};
                double phase = 1.0;
                if (dir == 0) {
                    cn[mu] = c[mu] + 1;
                    if (cn[mu] == p->L[mu]) {
                        cn[mu] = 0;
                        if (mu == 3 && p->tbc) phase = -1.0;
                    }
                } else {
                    cn[mu] = c[mu] - 1;
                    if (cn[mu] < 0) {
                        cn[mu] = p->L[mu] - 1;
                        if (mu == 3 && p->tbc) phase = -1.0;
                    }
                }
                const long sn = site_of(p->L, cn);
                /* link: U_mu(x) forward, U_mu(x-mu)^dag backward */
                cplx link[3][3];
                const long ls = (dir == 0) ? s : sn;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        cplx u = U[(((long)mu * V + ls) * 3 + a) * 3 + b];
                        if (dir == 0) link[a][b] = u;
                        else link[b][a] = conj(u);
                    }
                /* projector 1 - sg*gamma (forward) or 1 + sg*gamma (backward) */
                const double ps = (dir == 0) ? -sg : sg;
                cplx proj[4][4];
                for (int i = 0; i < 4; i++)
                    for (int j = 0; j < 4; j++)
                        proj[i][j] = (i == j ? 1.0 : 0.0) + ps * GAMMA[mu][i][j];
                for (int f = 0; f < nf; f++) {
                    const cplx *v = in + (sn * nf + f) * 12;
                    cplx uv[4][3];
                    for (int sp = 0; sp < 4; sp++)
                        for (int a = 0; a < 3; a++) {
                            cplx t = 0;
                            for (int b = 0; b < 3; b++) t += link[a][b] * v[sp * 3 + b];
                            uv[sp][a] = t;
                        }
                    for (int i = 0; i < 4; i++)
                        for (int a = 0; a < 3; a++) {
                            cplx t = 0;
                            for (int j = 0; j < 4; j++) t += proj[i][j] * uv[j][a];
                            acc[f][i][a] += phase * t;
                        }
                }
            }
        }
        for (int f = 0; f < nf; f++)
            for (int i = 0; i < 4; i++)
                for (int a = 0; a < 3; a++) out[((s * nf + f) * 4 + i) * 3 + a] = acc[f][i][a];
    }
}

/* Gauss-Jordan inverse of an n x n complex matrix with partial pivoting. */
static int invert(int n, const cplx *a_in, cplx *inv)
{
    cplx a[8][16];
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            a[i][j] = (j < n) ? a_in[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (cabs(a[r][col]) > cabs(a[piv][col])) piv = r;
        if (cabs(a[piv][col]) == 0.0) return -1;
        if (piv != col)
            for (int j = 0; j < 2 * n; j++) {
                cplx t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t;
            }
        const cplx d = a[col][col];
        for (int j = 0; j < 2 * n; j++) a[col][j] /= d;
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            const cplx f = a[r][col];
            for (int j = 0; j < 2 * n; j++) a[r][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) inv[i * n + j] = a[i][n + j];
    return 0;
}

/*
 * The local twist on the (flavour, spin) index, D = 4*nf:
 *   R = 1 + i (2 kappa mu) gamma5 tau3 + (2 kappa eps) tau1   (doublet)
 *   R = 1 + i (2 kappa mu) fsign gamma5                       (one flavour)
 * mode bit 0: inverse, bit 1: hermitian conjugate (applied after the inverse).
 */
int orc_twist_matrix(const orc_params *p, int mode, double *out_re_im)
{
    const int nf = p->nf, D = 4 * nf;
    cplx g5[4][4];
    gamma5(g5);
    const double a = 2.0 * p->kappa * p->mu, b = 2.0 * p->kappa * p->eps;
    const double tau3[2][2] = {{1, 0}, {0, -1}}, tau1[2][2] = {{0, 1}, {1, 0}};
    cplx R[64], T[64];
    for (int f = 0; f < nf; f++)
        for (int s = 0; s < 4; s++)
            for (int f2 = 0; f2 < nf; f2++)
                for (int s2 = 0; s2 < 4; s2++) {
                    cplx v = (f == f2 && s == s2) ? 1.0 : 0.0;
                    if (nf == 2) {
                        v += I * a * g5[s][s2] * tau3[f][f2];
                        if (s == s2) v += b * tau1[f][f2];
                    } else {
                        v += I * a * (double)p->fsign * g5[s][s2];
                    }
                    R[(f * 4 + s) * D + f2 * 4 + s2] = v;
                }
    if (mode & 1) {
        if (invert(D, R, T)) return -1;
    } else {
        memcpy(T, R, sizeof(cplx) * D * D);
    }
    if (mode & 2) {
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++) R[i * D + j] = conj(T[j * D + i]);
        memcpy(T, R, sizeof(cplx) * D * D);
    }
    if (out_re_im)
        for (int i = 0; i < D * D; i++) {
            out_re_im[2 * i] = creal(T[i]);
            out_re_im[2 * i + 1] = cimag(T[i]);
        }
    return 0;
}

/* out = T in with T the twist matrix of orc_twist_matrix(mode); in-place allowed. */
int orc_twist(const orc_params *p, const cplx *in, cplx *out, int mode)
{
    const int nf = p->nf, D = 4 * nf;
    double m[2 * 64];
    if (orc_twist_matrix(p, mode, m)) return -1;
    cplx T[64];
    for (int i = 0; i < D * D; i++) T[i] = m[2 * i] + I * m[2 * i + 1];
    const long V = volume(p);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        cplx v[8][3], w[8][3];
        for (int k = 0; k < D; k++)
            for (int a = 0; a < 3; a++) v[k][a] = in[(s * D + k) * 3 + a];
        for (int k = 0; k < D; k++)
            for (int a = 0; a < 3; a++) {
                cplx t = 0;
                for (int k2 = 0; k2 < D; k2++) t += T[k * D + k2] * v[k2][a];
                w[k][a] = t;
            }
        for (int k = 0; k < D; k++)
            for (int a = 0; a < 3; a++) out[(s * D + k) * 3 + a] = w[k][a];
    }
    return 0;
}

/* Zero every site whose parity (x+y+z+t) mod 2 differs from `parity`. */
void orc_parity_project(const orc_params *p, cplx *v, int parity)
{
    const long V = volume(p);
    const int n = 12 * p->nf;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int c[4];
        coords_of(p->L, s, c);
        if (((c[0] + c[1] + c[2] + c[3]) & 1) != parity)
            for (int k = 0; k < n; k++) v[s * n + k] = 0;
    }
}

static cplx *vec_alloc(const orc_params *p)
{
    return (cplx *)calloc((size_t)volume(p) * 12 * p->nf, sizeof(cplx));
}

static long vec_len(const orc_params *p) { return volume(p) * 12 * p->nf; }

/* out = M in, or M^dag in:  M = R - kappa H,  M^dag = R^dag - kappa H^dag  (eq. 2.1) */
int orc_M(const orc_params *p, const cplx *U, const cplx *in, cplx *out, int dagger)
{
    cplx *h = vec_alloc(p);
    if (!h) return -1;
    orc_hop(p, U, in, h, dagger);
    int rc = orc_twist(p, in, out, dagger ? 2 : 0);
    const long n = vec_len(p);
    for (long i = 0; i < n; i++) out[i] -= p->kappa * h[i];
    free(h);
    return rc;
}

/*
 * Even-even Schur complements (eq. 2.2 and 2.3, with the paper's D_eo read
 * as the bare hopping block H_eo):
 *   asym:  M_asym  = R_ee - kappa^2 H_eo R_oo^-1 H_oe
 *          M_asym^dag = R_ee^dag - kappa^2 H^dag_eo R_oo^-dag H^dag_oe
 *   sym:   M_sym   = 1 - kappa^2 R_ee^-1 H_eo R_oo^-1 H_oe
 *          M_sym^dag  = 1 - kappa^2 H^dag_eo R_oo^-dag H^dag_oe R_ee^-dag
 * `in` is a full-lattice vector; only its even sites are used, and the
 * result is supported on even sites.
 */
int orc_M_pc(const orc_params *p, const cplx *U, const cplx *in, cplx *out, int sym, int dagger)
{
    const long n = vec_len(p);
    cplx *ve = vec_alloc(p), *t1 = vec_alloc(p), *t2 = vec_alloc(p);
    if (!ve || !t1 || !t2) { free(ve); free(t1); free(t2); return -1; }
    memcpy(ve, in, sizeof(cplx) * n);
    orc_parity_project(p, ve, 0);
    const int tw = dagger ? 2 : 0, twinv = dagger ? 3 : 1;
    int rc = 0;
    if (sym && dagger) {
        rc |= orc_twist(p, ve, t2, twinv);          /* R_ee^-dag v        */
        orc_hop(p, U, t2, t1, 1);                   /* H^dag_oe           */
        orc_parity_project(p, t1, 1);
        rc |= orc_twist(p, t1, t1, twinv);          /* R_oo^-dag          */
        orc_hop(p, U, t1, t2, 1);                   /* H^dag_eo           */
        orc_parity_project(p, t2, 0);
        for (long i = 0; i < n; i++) out[i] = ve[i] - p->kappa * p->kappa * t2[i];
    } else {
        orc_hop(p, U, ve, t1, dagger);              /* H_oe v             */
        orc_parity_project(p, t1, 1);
        rc |= orc_twist(p, t1, t1, twinv);          /* R_oo^-1            */
        orc_hop(p, U, t1, t2, dagger);              /* H_eo               */
        orc_parity_project(p, t2, 0);
        if (sym) {
            rc |= orc_twist(p, t2, t2, twinv);      /* R_ee^-1            */
            for (long i = 0; i < n; i++) out[i] = ve[i] - p->kappa * p->kappa * t2[i];
        } else {
            rc |= orc_twist(p, ve, t1, tw);         /* R_ee v             */
            for (long i = 0; i < n; i++) out[i] = t1[i] - p->kappa * p->kappa * t2[i];
        }
    }
    orc_parity_project(p, out, 0);
    free(ve); free(t1); free(t2);
    return rc;
}

/*
 * Right-hand side of the even system obtained by eliminating the odd sites
 * from M psi = b (or M^dag psi = b with dagger = 1):
 *   asym:  b'_e = b_e + kappa H_eo R_oo^-1 b_o           M_asym psi_e = b'_e
 *   sym:   b'_e = R_ee^-1 (b_e + kappa H_eo R_oo^-1 b_o)  M_sym psi_e = b'_e
 * With dagger = 1 every factor is daggered.  For sym the daggered system is
 * preconditioned from the right, because M_sym^dag = M_asym^dag R_ee^-dag:
 *   b'_e = b_e + kappa H^dag_eo R_oo^-dag b_o,  M_sym^dag y = b'_e,
 *   psi_e = R_ee^-dag y.
 */
int orc_prepare_rhs(const orc_params *p, const cplx *U, const cplx *b, cplx *bprime, int sym, int dagger)
{
    const long n = vec_len(p);
    cplx *bo = vec_alloc(p), *t = vec_alloc(p);
    if (!bo || !t) { free(bo); free(t); return -1; }
    const int twinv = dagger ? 3 : 1;
    memcpy(bo, b, sizeof(cplx) * n);
    orc_parity_project(p, bo, 1);
    int rc = orc_twist(p, bo, bo, twinv);
    orc_hop(p, U, bo, t, dagger);
    orc_parity_project(p, t, 0);
    memcpy(bprime, b, sizeof(cplx) * n);
    orc_parity_project(p, bprime, 0);
    for (long i = 0; i < n; i++) bprime[i] += p->kappa * t[i];
    if (sym && !dagger) rc |= orc_twist(p, bprime, bprime, twinv);
    free(bo); free(t);
    return rc;
}

/*
 * Odd-site solution from the even one (block elimination of M psi = b):
 *   psi_o = R_oo^-1 (b_o + kappa H_oe psi_e)      (daggered when dagger = 1)
 * Output is a full-lattice vector supported on odd sites.
 */
int orc_reconstruct_odd(const orc_params *p, const cplx *U, const cplx *psi_e, const cplx *b, cplx *psi_o,
                        int dagger)
{
    const long n = vec_len(p);
    cplx *ve = vec_alloc(p), *t = vec_alloc(p);
    if (!ve || !t) { free(ve); free(t); return -1; }
    memcpy(ve, psi_e, sizeof(cplx) * n);
    orc_parity_project(p, ve, 0);
    orc_hop(p, U, ve, t, dagger);
    memcpy(psi_o, b, sizeof(cplx) * n);
    orc_parity_project(p, psi_o, 1);
    for (long i = 0; i < n; i++) psi_o[i] += p->kappa * t[i];
    int rc = orc_twist(p, psi_o, psi_o, dagger ? 3 : 1);
    orc_parity_project(p, psi_o, 1);
    free(ve); free(t);
    return rc;
}

static double rdot(long n, const cplx *a, const cplx *b)
{
    double s = 0;
    for (long i = 0; i < n; i++) s += creal(conj(a[i]) * b[i]);
    return s;
}

/*
 * Conjugate gradient on the normal equations A^dag A x = y for the even
 * operator A = M_pc (dagger = 0) or A = M_pc^dag (dagger = 1).  x holds the
 * initial guess on entry.  Stops when the recursively updated residual falls
 * below tol * |y|; *true_res receives |y - A^dag A x| / |y| recomputed at
 * the end.  Returns the iteration count, or -1 on allocation failure.
 */
int orc_cg_normal(const orc_params *p, const cplx *U, int sym, int dagger, const cplx *y, cplx *x, double tol,
                  int maxiter, double *true_res)
{
    const long n = vec_len(p);
    cplx *r = vec_alloc(p), *pp = vec_alloc(p), *t = vec_alloc(p), *ap = vec_alloc(p);
    if (!r || !pp || !t || !ap) { free(r); free(pp); free(t); free(ap); return -1; }
    orc_M_pc(p, U, x, t, sym, dagger);
    orc_M_pc(p, U, t, ap, sym, !dagger);
    for (long i = 0; i < n; i++) r[i] = y[i] - ap[i];
    orc_parity_project(p, r, 0);
    memcpy(pp, r, sizeof(cplx) * n);
    const double yy = rdot(n, y, y);
    double rr = rdot(n, r, r);
    int it = 0;
    while (it < maxiter && rr > tol * tol * yy) {
        orc_M_pc(p, U, pp, t, sym, dagger);
        orc_M_pc(p, U, t, ap, sym, !dagger);
        const double alpha = rr / rdot(n, pp, ap);
        for (long i = 0; i < n; i++) {
            x[i] += alpha * pp[i];
            r[i] -= alpha * ap[i];
        }
        const double rr_new = rdot(n, r, r);
        const double beta = rr_new / rr;
        for (long i = 0; i < n; i++) pp[i] = r[i] + beta * pp[i];
        rr = rr_new;
        it++;
    }
    orc_M_pc(p, U, x, t, sym, dagger);
    orc_M_pc(p, U, t, ap, sym, !dagger);
    for (long i = 0; i < n; i++) r[i] = y[i] - ap[i];
    orc_parity_project(p, r, 0);
    if (true_res) *true_res = sqrt(rdot(n, r, r) / yy);
    free(r); free(pp); free(t); free(ap);
    return it;
}

/*
 * Link gradient of L(U) = Re < g, M(U) psi >  (inner product conjugate-linear
 * in its first argument), as the complex matrix G_mu(x) with
 *   dL = Re sum_{ij} conj(G_ij) dU_ij
 * for an unconstrained variation dU of U_mu(x).  From eq. 2.1 only the two
 * hopping terms that contain U_mu(x) contribute:
 *   G_mu(x) = -kappa * bc * [ sum_s ((1 - gamma_mu) g(x))_s  psi(x+mu)_s^dag
 *                           + sum_s psi(x)_s ((1 + gamma_mu) g(x+mu))_s^dag ]
 * summed over flavours, with bc = -1 on the links that cross the
 * antiperiodic time boundary.  The result is multiplied by `coef`.
 * project = 1 replaces G by its component in the tangent space of SU(3) at U,
 *   P(G) = TA(G U^dag) U,  TA(Z) = (Z - Z^dag)/2 - tr(Z - Z^dag)/6.
 */
void orc_force(const orc_params *p, const cplx *U, const cplx *psi, const cplx *g, double coef, cplx *G,
               int project)
{
    const long V = volume(p);
    const int nf = p->nf;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int c[4];
        coords_of(p->L, s, c);
        for (int mu = 0; mu < 4; mu++) {
            int cn[4] = {c[0], c[1], c[2], c[3]};
            double bc = 1.0;
            cn[mu] = c[mu] + 1;
            if (cn[mu] == p->L[mu]) {
                cn[mu] = 0;
                if (mu == 3 && p->tbc) bc = -1.0;
            }
            const long sn = site_of(p->L, cn);
            cplx m[3][3];
            memset(m, 0, sizeof(m));
            for (int f = 0; f < nf; f++) {
                const cplx *gx = g + (s * nf + f) * 12, *gy = g + (sn * nf + f) * 12;
                const cplx *px = psi + (s * nf + f) * 12, *py = psi + (sn * nf + f) * 12;
                cplx w1[4][3], w2[4][3];
                for (int i = 0; i < 4; i++)
                    for (int a = 0; a < 3; a++) {
                        cplx t1 = gx[i * 3 + a], t2 = gy[i * 3 + a];
                        for (int j = 0; j < 4; j++) {
                            t1 -= GAMMA[mu][i][j] * gx[j * 3 + a];
                            t2 += GAMMA[mu][i][j] * gy[j * 3 + a];
                        }
                        w1[i][a] = t1;
                        w2[i][a] = t2;
                    }
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        cplx t = 0;
                        for (int i = 0; i < 4; i++)
                            t += w1[i][a] * conj(py[i * 3 + b]) + px[i * 3 + a] * conj(w2[i][b]);
                        m[a][b] += t;
                    }
            }
            const double scale = -p->kappa * bc * coef;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) m[a][b] *= scale;
            const cplx *u = U + ((long)mu * V + s) * 9;
            if (project) {
                cplx z[3][3], ta[3][3];
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        cplx t = 0;
                        for (int k = 0; k < 3; k++) t += m[a][k] * conj(u[b * 3 + k]);
                        z[a][b] = t;
                    }
                cplx tr = 0;
                for (int a = 0; a < 3; a++) tr += z[a][a] - conj(z[a][a]);
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++)
                        ta[a][b] = 0.5 * (z[a][b] - conj(z[b][a])) - (a == b ? tr / 6.0 : 0.0);
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        cplx t = 0;
                        for (int k = 0; k < 3; k++) t += ta[a][k] * u[k * 3 + b];
                        m[a][b] = t;
                    }
            }
            cplx *out = G + ((long)mu * V + s) * 9;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) out[a * 3 + b] = m[a][b];
        }
    }
}

// tm_clover.cu -- the clover field of a handle (built once on the device from its FP64 links)
// and the local clover-twisted-mass operator L = C + X applied as a pass of its own.
//
// F_{mu nu}(x) = (Q - Q^dag) / 8 with Q the four plaquettes of the mu-nu plane that start and
// end at x, all traversed mu first; C = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu},
// sigma_{mu nu} = (i/2)[g_mu, g_nu] (DeGrand-Rossi basis, the one the hopping kernel's
// projectors encode).  C is stored per gamma5 block together with D^-1 = (C^2 - X^2)^-1, the
// factor of L^-1 = (C - X) D^-1 (tm_clover.cuh).
#include <math.h>
#include <string.h>

#include "tm_clover.cuh"
#include "tm_internal.h"

namespace tmk {

struct CloverBuildArgs {
    const void *links;  // the handle's FP64 links, [mu][parity][chunk][Vh]
    int Vh, X1h, Lx, Ly, Lz, Lt;
    double w[6][2][2][2][2];  // i kappa c_sw sigma_{mu nu}[2g+s][2g+s'] as (re, im): [plane][g][s][s']
    double x2;                // X^2, a number
    void *out64, *out32, *out16;
    float *norm16;
    int *err;  // set to 1 when a D block is numerically singular
};

__device__ __forceinline__ void m3_mul(const Link<double> &a, const Link<double> &b, Link<double> &c)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            C<double> s = cmul(a.u[i][0], b.u[0][j]);
            s = cadd(s, cmul(a.u[i][1], b.u[1][j]));
            c.u[i][j] = cadd(s, cmul(a.u[i][2], b.u[2][j]));
        }
}
// c = a b^dag
__device__ __forceinline__ void m3_mul_dag(const Link<double> &a, const Link<double> &b, Link<double> &c)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            C<double> s = cmul(a.u[i][0], cconj(b.u[j][0]));
            s = cadd(s, cmul(a.u[i][1], cconj(b.u[j][1])));
            c.u[i][j] = cadd(s, cmul(a.u[i][2], cconj(b.u[j][2])));
        }
}
// c = a^dag b
__device__ __forceinline__ void m3_dag_mul(const Link<double> &a, const Link<double> &b, Link<double> &c)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            C<double> s = cmulc(a.u[0][i], b.u[0][j]);
            s = cadd(s, cmulc(a.u[1][i], b.u[1][j]));
            c.u[i][j] = cadd(s, cmulc(a.u[2][i], b.u[2][j]));
        }
}

template <int RECON>
__device__ __forceinline__ void fetch_link(const CloverBuildArgs &a, int mu, int x, int y, int z, int t,
                                           Link<double> &U)
{
    x = (x % a.Lx + a.Lx) % a.Lx;
    y = (y % a.Ly + a.Ly) % a.Ly;
    z = (z % a.Lz + a.Lz) % a.Lz;
    t = (t % a.Lt + a.Lt) % a.Lt;
    const long lex = x + (long)a.Lx * (y + (long)a.Ly * (z + (long)a.Lz * t));
    const int par = (x + y + z + t) & 1;
    using LL = LinkLayout<P64, RECON>;
    const typename LL::chunk *G = reinterpret_cast<const typename LL::chunk *>(a.links);
    LinkLoader<P64, RECON>::load(G + (size_t)(mu * 2 + par) * LL::N * a.Vh, (int)(lex >> 1), a.Vh, U);
}

// Gauss-Jordan inverse of a 6x6 complex matrix with partial pivoting; false when a pivot is
// below tiny (relative to the largest entry of the matrix)
__device__ bool invert6(C<double> m[6][6], C<double> inv[6][6])
{
    double amax = 0.0;
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            amax = fmax(amax, fabs(m[i][j].r) + fabs(m[i][j].i));
            inv[i][j] = {i == j ? 1.0 : 0.0, 0.0};
        }
    for (int c = 0; c < 6; c++) {
        int piv = c;
        double best = -1.0;
        for (int r = c; r < 6; r++) {
            const double v = m[r][c].r * m[r][c].r + m[r][c].i * m[r][c].i;
            if (v > best) { best = v; piv = r; }
        }
        if (!(sqrt(best) > 1e-13 * amax)) return false;
        if (piv != c)
            for (int j = 0; j < 6; j++) {
                C<double> t = m[c][j]; m[c][j] = m[piv][j]; m[piv][j] = t;
                t = inv[c][j]; inv[c][j] = inv[piv][j]; inv[piv][j] = t;
            }
        const C<double> p = m[c][c];
        const double d = p.r * p.r + p.i * p.i;
        const C<double> pi = {p.r / d, -p.i / d};
        for (int j = 0; j < 6; j++) {
            m[c][j] = cmul(pi, m[c][j]);
            inv[c][j] = cmul(pi, inv[c][j]);
        }
        for (int r = 0; r < 6; r++) {
            if (r == c) continue;
            const C<double> f = m[r][c];
            for (int j = 0; j < 6; j++) {
                m[r][j] = csub(m[r][j], cmul(f, m[c][j]));
                inv[r][j] = csub(inv[r][j], cmul(f, inv[c][j]));
            }
        }
    }
    return true;
}

// pack a hermitian 6x6 matrix (its hermitian part) into 36 reals
__device__ __forceinline__ void pack_herm(const C<double> m[6][6], double h[36])
{
    for (int i = 0; i < 6; i++) h[i] = m[i][i].r;
    int k = 6;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            h[k] = 0.5 * (m[i][j].r + m[j][i].r);
            h[k + 1] = 0.5 * (m[i][j].i - m[j][i].i);
            k += 2;
        }
}

__device__ void store_block(const CloverBuildArgs &a, int parity, int blk, int cb, const double h[36])
{
    {
        double2 *p = reinterpret_cast<double2 *>(a.out64) + ((size_t)parity * 4 * 18 + (size_t)blk * 18) * a.Vh + cb;
        for (int k = 0; k < 18; k++) p[(size_t)k * a.Vh] = make_double2(h[2 * k], h[2 * k + 1]);
    }
    {
        float4 *p = reinterpret_cast<float4 *>(a.out32) + ((size_t)parity * 4 * 9 + (size_t)blk * 9) * a.Vh + cb;
        for (int k = 0; k < 9; k++)
            p[(size_t)k * a.Vh] = make_float4((float)h[4 * k], (float)h[4 * k + 1], (float)h[4 * k + 2], (float)h[4 * k + 3]);
    }
    {
        double m = 0.0;
        for (int k = 0; k < 36; k++) m = fmax(m, fabs(h[k]));
        const double inv = m > 0.0 ? 1.0 / m : 0.0;
        float t[40];
        for (int k = 0; k < 40; k++) t[k] = k < 36 ? (float)(h[k] * inv) : 0.f;
        uint4 *p = reinterpret_cast<uint4 *>(a.out16) + ((size_t)parity * 4 * 5 + (size_t)blk * 5) * a.Vh + cb;
        for (int k = 0; k < 5; k++) {
            uint4 c;
            c.x = f2h(t[8 * k + 0], t[8 * k + 1]);
            c.y = f2h(t[8 * k + 2], t[8 * k + 3]);
            c.z = f2h(t[8 * k + 4], t[8 * k + 5]);
            c.w = f2h(t[8 * k + 6], t[8 * k + 7]);
            p[(size_t)k * a.Vh] = c;
        }
        a.norm16[((size_t)parity * 4 + blk) * a.Vh + cb] = (float)m;
    }
}

// one thread per site of either parity (id < Vh: even, else odd)
template <int RECON>
__global__ void __launch_bounds__(128) k_clover_build(const __grid_constant__ CloverBuildArgs a)
{
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= 2L * a.Vh) return;
    const int parity = id >= a.Vh ? 1 : 0;
    const int cb = (int)(id - (long)parity * a.Vh);
    int r = cb;
    const int xh = r % a.X1h;
    r /= a.X1h;
    const int y = r % a.Ly;
    r /= a.Ly;
    const int z = r % a.Lz;
    const int t = r / a.Lz;
    const int x = 2 * xh + ((parity + y + z + t) & 1);
    const int X[4] = {x, y, z, t};

    C<double> Cb[2][6][6];
    for (int g = 0; g < 2; g++)
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) Cb[g][i][j] = {i == j ? 1.0 : 0.0, 0.0};

    int plane = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, plane++) {
            int e[4] = {0, 0, 0, 0}, f[4] = {0, 0, 0, 0};
            e[mu] = 1;
            f[nu] = 1;
            Link<double> A, B, P, Q;
            // leaf at corner x: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
            fetch_link<RECON>(a, mu, X[0], X[1], X[2], X[3], A);
            fetch_link<RECON>(a, nu, X[0] + e[0], X[1] + e[1], X[2] + e[2], X[3] + e[3], B);
            m3_mul(A, B, P);
            fetch_link<RECON>(a, mu, X[0] + f[0], X[1] + f[1], X[2] + f[2], X[3] + f[3], B);
            m3_mul_dag(P, B, Q);
            fetch_link<RECON>(a, nu, X[0], X[1], X[2], X[3], B);
            m3_mul_dag(Q, B, P);
            Link<double> S = P;
            // leaf at corner x-mu: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
            fetch_link<RECON>(a, nu, X[0], X[1], X[2], X[3], A);
            fetch_link<RECON>(a, mu, X[0] - e[0] + f[0], X[1] - e[1] + f[1], X[2] - e[2] + f[2], X[3] - e[3] + f[3], B);
            m3_mul_dag(A, B, P);
            fetch_link<RECON>(a, nu, X[0] - e[0], X[1] - e[1], X[2] - e[2], X[3] - e[3], B);
            m3_mul_dag(P, B, Q);
            fetch_link<RECON>(a, mu, X[0] - e[0], X[1] - e[1], X[2] - e[2], X[3] - e[3], B);
            m3_mul(Q, B, P);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) S.u[i][j] = cadd(S.u[i][j], P.u[i][j]);
            // leaf at corner x-mu-nu: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
            fetch_link<RECON>(a, nu, X[0] - e[0] - f[0], X[1] - e[1] - f[1], X[2] - e[2] - f[2], X[3] - e[3] - f[3], A);
            fetch_link<RECON>(a, mu, X[0] - e[0], X[1] - e[1], X[2] - e[2], X[3] - e[3], B);
            m3_mul(A, B, Q);  // (U_mu(x-mu)^dag U_nu(x-mu-nu)^dag) = (U_nu(x-mu-nu) U_mu(x-mu))^dag
            fetch_link<RECON>(a, mu, X[0] - e[0] - f[0], X[1] - e[1] - f[1], X[2] - e[2] - f[2], X[3] - e[3] - f[3], B);
            m3_dag_mul(Q, B, P);
            fetch_link<RECON>(a, nu, X[0] - f[0], X[1] - f[1], X[2] - f[2], X[3] - f[3], B);
            m3_mul(P, B, Q);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) S.u[i][j] = cadd(S.u[i][j], Q.u[i][j]);
            // leaf at corner x-nu: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
            fetch_link<RECON>(a, nu, X[0] - f[0], X[1] - f[1], X[2] - f[2], X[3] - f[3], A);
            fetch_link<RECON>(a, mu, X[0] - f[0], X[1] - f[1], X[2] - f[2], X[3] - f[3], B);
            m3_dag_mul(A, B, P);
            fetch_link<RECON>(a, nu, X[0] - f[0] + e[0], X[1] - f[1] + e[1], X[2] - f[2] + e[2], X[3] - f[3] + e[3], B);
            m3_mul(P, B, Q);
            fetch_link<RECON>(a, mu, X[0], X[1], X[2], X[3], B);
            m3_mul_dag(Q, B, P);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) S.u[i][j] = cadd(S.u[i][j], P.u[i][j]);
            // F = (Q - Q^dag) / 8, accumulated into both gamma5 blocks of C
            for (int g = 0; g < 2; g++)
                for (int s = 0; s < 2; s++)
                    for (int sp = 0; sp < 2; sp++) {
                        const C<double> w = {a.w[plane][g][s][sp][0], a.w[plane][g][s][sp][1]};
                        if (w.r == 0.0 && w.i == 0.0) continue;
                        for (int c = 0; c < 3; c++)
                            for (int d = 0; d < 3; d++) {
                                const C<double> Fcd = {0.125 * (S.u[c][d].r - S.u[d][c].r),
                                                       0.125 * (S.u[c][d].i + S.u[d][c].i)};
                                Cb[g][3 * s + c][3 * sp + d] = cadd(Cb[g][3 * s + c][3 * sp + d], cmul(w, Fcd));
                            }
                    }
        }

    for (int g = 0; g < 2; g++) {
        double h[36];
        pack_herm(Cb[g], h);
        store_block(a, parity, g, cb, h);
        // D = C^2 - X^2 and its inverse
        C<double> D[6][6], Di[6][6];
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) {
                C<double> s = {i == j ? -a.x2 : 0.0, 0.0};
                for (int k = 0; k < 6; k++) s = cadd(s, cmul(Cb[g][i][k], Cb[g][k][j]));
                D[i][j] = s;
            }
        if (!invert6(D, Di)) {
            atomicExch(a.err, 1);
            for (int i = 0; i < 6; i++)
                for (int j = 0; j < 6; j++) Di[i][j] = {0.0, 0.0};
        }
        pack_herm(Di, h);
        store_block(a, parity, 2 + g, cb, h);
    }
}

// out = L in (INV = false) or L^-1 in on the sites of `parity`, any nrhs = 1 parity field
template <int PREC, int NF, bool INV>
__global__ void __launch_bounds__(128) k_clover_apply(void *out, float *out_norm, const void *in, const float *in_norm,
                                                      const void *clov, const float *cnorm, int parity, int Vh,
                                                      const __grid_constant__ Twist<typename Traits<PREC>::real> X)
{
    using T = typename Traits<PREC>::real;
    using SC = typename Traits<PREC>::schunk;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= Vh) return;
    const size_t fstride = (size_t)Traits<PREC>::SCHUNKS * Vh;
    T v[NF][24];
    const SC *I = reinterpret_cast<const SC *>(in);
#pragma unroll
    for (int f = 0; f < NF; f++) load_spinor<PREC>(I + f * fstride, in_norm ? in_norm + (size_t)f * Vh : nullptr, cb, Vh, v[f]);
    apply_clover<PREC, NF, INV>(clov, cnorm, parity, cb, Vh, X, v);
    SC *O = reinterpret_cast<SC *>(out);
#pragma unroll
    for (int f = 0; f < NF; f++) store_spinor<PREC>(O + f * fstride, out_norm ? out_norm + (size_t)f * Vh : nullptr, cb, Vh, v[f]);
}

// ------------------------------------------------------------------------------------------ host
// DeGrand-Rossi gamma matrices, index 0..3 <-> x, y, z, t, as (re, im)
static const double DR_GAMMA[4][4][4][2] = {
    {{{0, 0}, {0, 0}, {0, 0}, {0, 1}}, {{0, 0}, {0, 0}, {0, 1}, {0, 0}}, {{0, 0}, {0, -1}, {0, 0}, {0, 0}},
     {{0, -1}, {0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 0}, {-1, 0}}, {{0, 0}, {0, 0}, {1, 0}, {0, 0}}, {{0, 0}, {1, 0}, {0, 0}, {0, 0}},
     {{-1, 0}, {0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 1}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {0, -1}}, {{0, -1}, {0, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {0, 1}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {1, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {1, 0}}, {{1, 0}, {0, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {1, 0}, {0, 0}, {0, 0}}},
};

// i kappa c_sw sigma_{mu nu} restricted to the gamma5 blocks; false if sigma mixed the blocks
static bool clover_weights(double kc, double w[6][2][2][2][2])
{
    int plane = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, plane++) {
            double sr[4][4], si[4][4];
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) {
                    double cr = 0, ci = 0;  // [g_mu, g_nu]_ij
                    for (int k = 0; k < 4; k++) {
                        const double *a = DR_GAMMA[mu][i][k], *b = DR_GAMMA[nu][k][j];
                        const double *c = DR_GAMMA[nu][i][k], *d = DR_GAMMA[mu][k][j];
                        cr += (a[0] * b[0] - a[1] * b[1]) - (c[0] * d[0] - c[1] * d[1]);
                        ci += (a[0] * b[1] + a[1] * b[0]) - (c[0] * d[1] + c[1] * d[0]);
                    }
                    // sigma = (i/2) [g_mu, g_nu]
                    sr[i][j] = -0.5 * ci;
                    si[i][j] = 0.5 * cr;
                }
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++)
                    if ((i >> 1) != (j >> 1) && (sr[i][j] != 0.0 || si[i][j] != 0.0)) return false;
            for (int g = 0; g < 2; g++)
                for (int s = 0; s < 2; s++)
                    for (int sp = 0; sp < 2; sp++) {
                        // i kappa c_sw sigma
                        w[plane][g][s][sp][0] = -kc * si[2 * g + s][2 * g + sp];
                        w[plane][g][s][sp][1] = kc * sr[2 * g + s][2 * g + sp];
                    }
        }
    return true;
}

size_t clover_bytes(int pidx, long Vh)
{
    // per parity: 4 blocks x 36 reals
    switch (pidx) {
    case 0: return (size_t)2 * 4 * 18 * 16 * Vh;
    case 1: return (size_t)2 * 4 * 9 * 16 * Vh;
    case 2: return (size_t)2 * 4 * 5 * 16 * Vh;
    default: return 0;
    }
}

void clover_free(tm_gauge *g)
{
    for (int i = 0; i < 3; i++) {
        if (g->clov[i]) cudaFree(g->clov[i]);
        g->clov[i] = nullptr;
    }
    if (g->clov_norm) cudaFree(g->clov_norm);
    g->clov_norm = nullptr;
    g->csw = 0.0;
}

tm_status clover_build(tm_gauge *g, double csw, cudaStream_t s)
{
    CloverBuildArgs a;
    memset(&a, 0, sizeof(a));
    if (!clover_weights(g->p.kappa * csw, a.w)) {
        set_error("clover: sigma_{mu nu} is not block diagonal in the gamma5 basis");
        return TM_ERR_ARG;
    }
    const double ta = 2.0 * g->p.kappa * g->p.mu, tb = 2.0 * g->p.kappa * g->p.epsilon;
    a.x2 = (g->nf == 2) ? (tb * tb - ta * ta) : -ta * ta;
    if (!g->links[0]) {
        set_error("clover: the clover field is built from the FP64 links, which this handle did not pack");
        return TM_ERR_ARG;
    }
    a.links = g->links[0];
    a.Vh = g->Vh;
    a.X1h = g->X1h;
    a.Lx = g->p.L[0];
    a.Ly = g->p.L[1];
    a.Lz = g->p.L[2];
    a.Lt = g->p.L[3];
    void *buf[3] = {nullptr, nullptr, nullptr};
    float *nrm = nullptr;
    int *err = nullptr;
    tm_status st = TM_OK;
    for (int i = 0; i < 3 && st == TM_OK; i++)
        if (cudaMalloc(&buf[i], clover_bytes(i, g->Vh)) != cudaSuccess) st = TM_ERR_NOMEM;
    if (st == TM_OK && cudaMalloc(&nrm, sizeof(float) * 8 * (size_t)g->Vh) != cudaSuccess) st = TM_ERR_NOMEM;
    if (st == TM_OK && cudaMalloc(&err, sizeof(int)) != cudaSuccess) st = TM_ERR_NOMEM;
    if (st != TM_OK) {
        cudaGetLastError();
        set_error("clover: device allocation failed");
    }
    if (st == TM_OK) st = cuda_check(cudaMemsetAsync(err, 0, sizeof(int), s), "clover memset");
    if (st == TM_OK) {
        a.out64 = buf[0];
        a.out32 = buf[1];
        a.out16 = buf[2];
        a.norm16 = nrm;
        a.err = err;
        const long n = 2L * g->Vh;
        const unsigned grid = (unsigned)((n + 127) / 128);
        switch (link_recon(g, 0)) {  // the clover term is built from the FP64 links
        case 18: k_clover_build<18><<<grid, 128, 0, s>>>(a); break;
        case 12: k_clover_build<12><<<grid, 128, 0, s>>>(a); break;
        default: k_clover_build<8><<<grid, 128, 0, s>>>(a); break;
        }
        st = cuda_check(cudaGetLastError(), "clover build launch");
    }
    int herr = 0;
    if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s), "clover flag");
    if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "clover build");
    if (st == TM_OK && herr) {
        set_error("clover: C^2 - X^2 is singular at some site (c_sw too large for this field)");
        st = TM_ERR_ARG;
    }
    if (err) cudaFree(err);
    if (st != TM_OK) {
        for (int i = 0; i < 3; i++)
            if (buf[i]) cudaFree(buf[i]);
        if (nrm) cudaFree(nrm);
        return st;
    }
    clover_free(g);
    for (int i = 0; i < 3; i++) g->clov[i] = buf[i];
    g->clov_norm = nrm;
    g->csw = csw;
    return TM_OK;
}

template <int PREC>
static cudaError_t apply_impl(const tm_gauge *g, const tm_field *out, const tm_field *in, int parity, bool inverse,
                              const Twist<typename Traits<PREC>::real> &X, cudaStream_t s)
{
    const int pidx = PREC == P64 ? 0 : (PREC == P32 ? 1 : 2);
    const unsigned grid = (unsigned)((g->Vh + 127) / 128);
    const void *cl = g->clov[pidx];
    const float *cn = g->clov_norm;
#define TM_CA(NF, INV) \
    k_clover_apply<PREC, NF, INV><<<grid, 128, 0, s>>>(out->data, out->norm, in->data, in->norm, cl, cn, parity, g->Vh, X)
    if (g->nf == 1) {
        if (inverse) TM_CA(1, true); else TM_CA(1, false);
    } else {
        if (inverse) TM_CA(2, true); else TM_CA(2, false);
    }
#undef TM_CA
    return cudaGetLastError();
}

cudaError_t launch_clover_apply(const tm_gauge *g, const tm_field *out, const tm_field *in, int parity, bool inverse,
                                const Twist<double> &X, cudaStream_t s)
{
    switch (in->prec) {
    case TM_PREC_F64: return apply_impl<P64>(g, out, in, parity, inverse, X, s);
    case TM_PREC_F32:
    case TM_PREC_F16: {
        Twist<float> f;
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++)
                for (int k = 0; k < 2; k++) f.m[i][j][k] = {(float)X.m[i][j][k].r, (float)X.m[i][j][k].i};
        return in->prec == TM_PREC_F32 ? apply_impl<P32>(g, out, in, parity, inverse, f, s)
                                        : apply_impl<P16>(g, out, in, parity, inverse, f, s);
    }
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tmk

// tm_force.cu -- link gradient of the twisted-mass operator (eq. 2.1) for differentiation.
//
// For L = Re <g, M(U) psi> (inner product conjugate-linear in g) only the two hopping terms
// holding U_mu(x) depend on it: the forward hop at x and the backward hop at x + mu.  With
// dL = Re sum_ij conj(G_ij) dU_ij the gradient is
//   G_mu(x) = -kappa * bc * sum_f [ sum_s ((1 - g_mu) g(x))_s  psi(x+mu)_s^dag
//                                  + sum_s psi(x)_s ((1 + g_mu) g(x+mu))_s^dag ]
// (bc = -1 on links across the antiperiodic time boundary), times a caller coefficient.
// The twist R does not depend on U.  project = 1 returns the component in the tangent space
// of SU(3) at U: P(G) = TA(G U^dag) U with TA(Z) = (Z - Z^dag)/2 - tr(Z - Z^dag)/6.
// One thread per site computes its four links; the colour outer products of spin-projected
// half-spinors are summed over the two projected spin rows and the flavours in registers and the
// 3x3 results are written in the canonical gauge layout.
#include "tm_blas.cuh"
#include "tm_core.cuh"
#include "tm_internal.h"

namespace tmk {

struct ForceArgs {
    const void *psi[2];
    const float *psi_norm[2];
    const void *gv[2];
    const float *gv_norm[2];
    const void *gauge;
    void *out;
    int Vh, X1h, Lx, Ly, Lz, Lt, nf, tbc, project;
    double coef;  // -kappa * caller coefficient
};

// Both projectors are twice rank-2 hermitian projectors whose lower spin rows are a unitary image
// of the upper ones, so a spin sum of an outer product with (1 -+ g_mu) collapses to the two
// upper rows:  sum_s ((1 - g) a)_s b_s^dag = sum_{s=0,1} ((1 - g) a)_s ((1 - g) b)_s^dag  (and the
// same with 1 + g).  The upper rows of (1 + sp g_mu) v are those of the hopping kernel's projection:
//   mu = x: (v0 + sp i v3, v1 + sp i v2)    mu = y: (v0 - sp v3, v1 + sp v2)
//   mu = z: (v0 + sp i v2, v1 - sp i v3)    mu = t: (v0 + sp v2, v1 + sp v3)
template <int MU, typename T>
__device__ __forceinline__ void project_upper(const C<T> v[4][3], T sp, C<T> h[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const C<T> p0 = v[0][c], p1 = v[1][c], p2 = v[2][c], p3 = v[3][c];
        if (MU == 0) {
            h[0][c] = {p0.r - sp * p3.i, p0.i + sp * p3.r};
            h[1][c] = {p1.r - sp * p2.i, p1.i + sp * p2.r};
        } else if (MU == 1) {
            h[0][c] = {p0.r - sp * p3.r, p0.i - sp * p3.i};
            h[1][c] = {p1.r + sp * p2.r, p1.i + sp * p2.i};
        } else if (MU == 2) {
            h[0][c] = {p0.r - sp * p2.i, p0.i + sp * p2.r};
            h[1][c] = {p1.r + sp * p3.i, p1.i - sp * p3.r};
        } else {
            h[0][c] = {p0.r + sp * p2.r, p0.i + sp * p2.i};
            h[1][c] = {p1.r + sp * p3.r, p1.i + sp * p3.i};
        }
    }
}

template <int PREC, typename T>
__device__ __forceinline__ void load_sp(const void *base, const float *norm, int f, int cb, int Vh, C<T> v[4][3])
{
    using SC = typename Traits<PREC>::schunk;
    using R = typename Traits<PREC>::real;
    R r[24];
    const SC *p = reinterpret_cast<const SC *>(base) + (long)f * Traits<PREC>::SCHUNKS * Vh;
    load_spinor<PREC>(p, norm ? norm + (long)f * Vh : nullptr, cb, Vh, r);
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) v[s][c] = {(T)r[2 * (3 * s + c)], (T)r[2 * (3 * s + c) + 1]};
}

// Complex multiply-adds as chains of fused multiply-adds.  binary32 pairs the real and imaginary
// parts in one packed f32x2 FMA per step (the same rounding as the two scalar FMAs of that step),
// so a complex multiply-add is two instructions instead of four.
// s += a conj(b):  s.r += a.i b.i, s.i -= a.r b.i, then s.r += a.r b.r, s.i += a.i b.r
template <typename T>
__device__ __forceinline__ void cmacc(C<T> &s, C<T> a, C<T> b)
{
    s.r = fma(a.r, b.r, fma(a.i, b.i, s.r));
    s.i = fma(a.i, b.r, fma(-a.r, b.i, s.i));
}
__device__ __forceinline__ void cmacc(C<float> &s, C<float> a, C<float> b)
{
    float2 t = __ffma2_rn(make_float2(a.i, -a.r), make_float2(b.i, b.i), make_float2(s.r, s.i));
    t = __ffma2_rn(make_float2(a.r, a.i), make_float2(b.r, b.r), t);
    s = {t.x, t.y};
}
// s += a b:  s.r -= a.i b.i, s.i += a.r b.i, then s.r += a.r b.r, s.i += a.i b.r
template <typename T>
__device__ __forceinline__ void cmac(C<T> &s, C<T> a, C<T> b)
{
    s.r = fma(a.r, b.r, fma(-a.i, b.i, s.r));
    s.i = fma(a.i, b.r, fma(a.r, b.i, s.i));
}
__device__ __forceinline__ void cmac(C<float> &s, C<float> a, C<float> b)
{
    float2 t = __ffma2_rn(make_float2(-a.i, a.r), make_float2(b.i, b.i), make_float2(s.r, s.i));
    t = __ffma2_rn(make_float2(a.r, a.i), make_float2(b.r, b.r), t);
    s = {t.x, t.y};
}

// m += sum_{s=0,1} a_s b_s^dag (colour outer products of two projected half-spinors)
template <typename T>
__device__ __forceinline__ void outer_add(const C<T> a[2][3], const C<T> b[2][3], C<T> m[3][3])
{
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) cmacc(m[i][j], a[s][i], b[s][j]);  // a_i conj(b_j)
}

// neighbour x + mu of site (x, y, z, t) with checkerboard index cb, and the boundary sign
template <int MU, typename T>
__device__ __forceinline__ int force_neighbour(const ForceArgs &a, int cb, int x, int y, int z, int t, T &bc)
{
    bc = T(1);
    if (MU == 0) return (cb - (x >> 1)) + (((x == a.Lx - 1) ? 0 : x + 1) >> 1);
    if (MU == 1) return (y == a.Ly - 1) ? cb - (a.Ly - 1) * a.X1h : cb + a.X1h;
    if (MU == 2) return (z == a.Lz - 1) ? cb - (a.Lz - 1) * a.X1h * a.Ly : cb + a.X1h * a.Ly;
    const int s = a.X1h * a.Ly * a.Lz;
    if (t == a.Lt - 1 && a.tbc) bc = T(-1);
    return (t == a.Lt - 1) ? cb - (a.Lt - 1) * s : cb + s;
}

// The gradient of U_mu(x): g(x), psi(x+mu), psi(x), g(x+mu) (loadv(k, f, v), k = 0..3) projected
// to half-spinors and the two outer products summed, scaled by coef * bc, and (project) taken to
// the tangent space at U (loadu(U)).
template <int MU, int NF, typename T, typename LV, typename LU>
__device__ __forceinline__ void gradient_core(const ForceArgs &a, T bc, LV loadv, LU loadu, C<T> m[3][3])
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) m[i][j] = {T(0), T(0)};
#pragma unroll
    for (int f = 0; f < NF; f++) {
        C<T> v[4][3], ha[2][3], hb[2][3];
        // sum_s ((1 - g) g(x))_s psi(x+mu)_s^dag
        loadv(0, f, v);
        project_upper<MU>(v, T(-1), ha);
        loadv(1, f, v);
        project_upper<MU>(v, T(-1), hb);
        outer_add(ha, hb, m);
        // sum_s psi(x)_s ((1 + g) g(x+mu))_s^dag
        loadv(2, f, v);
        project_upper<MU>(v, T(1), ha);
        loadv(3, f, v);
        project_upper<MU>(v, T(1), hb);
        outer_add(ha, hb, m);
    }
    const T sc = (T)a.coef * bc;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) m[i][j] = cscale(sc, m[i][j]);
    if (a.project) {
        Link<T> U;
        loadu(U);
        C<T> zz[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                C<T> s = {T(0), T(0)};
#pragma unroll
                for (int k = 0; k < 3; k++) cmacc(s, m[i][k], U.u[j][k]);  // (m U^dag)_ij
                zz[i][j] = s;
            }
        // TA(Z) = (Z - Z^dag)/2 - i Im tr(Z)/3 (the trace of (Z - Z^dag)/2 is i Im tr Z)
        const T imtr = (zz[0][0].i + zz[1][1].i + zz[2][2].i) / T(3);
        C<T> ta[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                ta[i][j] = {T(0.5) * (zz[i][j].r - zz[j][i].r), T(0.5) * (zz[i][j].i + zz[j][i].i)};
                if (i == j) ta[i][j].i -= imtr;
            }
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                C<T> s = {T(0), T(0)};
#pragma unroll
                for (int k = 0; k < 3; k++) cmac(s, ta[i][k], U.u[k][j]);  // (TA U)_ij
                m[i][j] = s;
            }
    }
}

// The gradient of U_mu(x) with its operands read from global memory.
template <int PREC, int RECON, int NF, int MU, typename T>
__device__ __forceinline__ void link_gradient(const ForceArgs &a, int par, int cb, int x, int y, int z, int t,
                                              C<T> m[3][3])
{
    T bc;
    const int nb = force_neighbour<MU>(a, cb, x, y, z, t, bc);
    auto loadv = [&](int k, int f, C<T> v[4][3]) {
        const int fp = (k == 0 || k == 2) ? par : 1 - par, site = (k == 0 || k == 2) ? cb : nb;
        if (k == 0 || k == 3) load_sp<PREC>(a.gv[fp], a.gv_norm[fp], f, site, a.Vh, v);
        else load_sp<PREC>(a.psi[fp], a.psi_norm[fp], f, site, a.Vh, v);
    };
    auto loadu = [&](Link<T> &U) {
        using LL = LinkLayout<PREC, RECON>;
        const typename LL::chunk *G = reinterpret_cast<const typename LL::chunk *>(a.gauge);
        LinkLoader<PREC, RECON>::load(G + (size_t)(MU * 2 + par) * LL::N * a.Vh, cb, a.Vh, U);
    };
    gradient_core<MU, NF, T>(a, bc, loadv, loadu, m);
}

// Ask L1 for the operands of direction MU that do not come from this site: the neighbour's psi
// and g (every flavour, every chunk) and the link.  Issued one direction ahead, so their DRAM
// latency overlaps the arithmetic of the current direction without holding registers.
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
template <int PREC, int RECON, int NF, int MU>
__device__ __forceinline__ void prefetch_dir(const ForceArgs &a, int par, int cb, int x, int y, int z, int t)
{
    using SC = typename Traits<PREC>::schunk;
    using LL = LinkLayout<PREC, RECON>;
    typename Traits<PREC>::real bc;
    const int nb = force_neighbour<MU>(a, cb, x, y, z, t, bc);
    const SC *ps = reinterpret_cast<const SC *>(a.psi[1 - par]), *gs = reinterpret_cast<const SC *>(a.gv[1 - par]);
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
        for (int k = 0; k < Traits<PREC>::SCHUNKS; k++) {
            const size_t off = ((size_t)f * Traits<PREC>::SCHUNKS + k) * a.Vh + nb;
            prefetch_l1(ps + off);
            prefetch_l1(gs + off);
        }
    const typename LL::chunk *G = reinterpret_cast<const typename LL::chunk *>(a.gauge) + (size_t)(MU * 2 + par) * LL::N * a.Vh;
#pragma unroll
    for (int k = 0; k < LL::N; k++) prefetch_l1(G + (size_t)k * a.Vh + cb);
}

// One thread per site x (both parities, lexicographic order, so a warp covers a contiguous run
// of the canonical output) computes its four links in turn, re-reading psi(x), g(x) from L1;
// each link's 3x3 gradient goes through the warp's part of a shared-memory tile so that the warp
// writes its contiguous run of the canonical layout with 16-byte stores (warp-level syncs only: no
// block barrier holds the other warps).  (Measured alternatives, slower at 24^3x48 in FP32: one
// warp per direction and 32 sites, 143 us; every operand of a warp's links copied into shared
// memory by cp.async first, 181-254 us; the same form as here with block barriers, 133 us.)
// the warp's run of sites for direction MU: stage in shared memory, then 16-byte stores
template <int MU, typename CT, typename T>
__device__ __forceinline__ void store_links(const ForceArgs &a, long V, bool valid, const C<T> m[3][3], CT *tile)
{
    const int lane = threadIdx.x & 31;
    const long w0 = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);  // the warp's first site
    CT *wt = tile + (threadIdx.x & ~31) * 9;
    if (valid) {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                CT v;
                v.x = m[i][j].r;
                v.y = m[i][j].i;
                wt[lane * 9 + 3 * i + j] = v;
            }
    }
    __syncwarp();
    const long nsite = (V - w0) < 32 ? (V - w0) : 32;
    if (nsite > 0) {
        // 9 complex per site: a multiple of 16 bytes per 2 sites, and the warp's run starts at an
        // even site (w0 is a multiple of 32), so its output starts 16-byte aligned
        const long nvec = nsite * 9 * (long)sizeof(CT) / 16;
        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<CT *>(a.out) + ((long)MU * V + w0) * 9);
        const uint4 *src = reinterpret_cast<const uint4 *>(wt);
        for (long k = lane; k < nvec; k += 32) dst[k] = src[k];
        // an odd number of complex64 sites leaves 8 bytes: written element-wise
        if (sizeof(CT) == 8 && (nsite * 9) % 2 == 1 && lane == 0)
            reinterpret_cast<CT *>(a.out)[((long)MU * V + w0) * 9 + nsite * 9 - 1] = wt[nsite * 9 - 1];
    }
    __syncwarp();  // the tile is rewritten by the next direction
}

template <int PREC, int RECON, int NF, typename CT>
__global__ void __launch_bounds__(128, (PREC == P64 ? 2 : 5)) k_force(const __grid_constant__ ForceArgs a)
{
    using T = typename Traits<PREC>::real;
    __shared__ __align__(16) CT tile[128 * 9];
    const long V = 2L * a.Vh;
    const long lex0 = (long)blockIdx.x * blockDim.x;
    const long lex = lex0 + threadIdx.x;
    const bool valid = lex < V;  // every thread takes part in its warp's syncs
    int x = 0, y = 0, z = 0, t = 0, par = 0, cb = 0;
    if (valid) {
        long r = lex;
        x = (int)(r % a.Lx);
        r /= a.Lx;
        y = (int)(r % a.Ly);
        r /= a.Ly;
        z = (int)(r % a.Lz);
        t = (int)(r / a.Lz);
        par = (x + y + z + t) & 1;
        cb = (int)(lex >> 1);
    }
    C<T> m[3][3];
    if (valid) {
        prefetch_dir<PREC, RECON, NF, 1>(a, par, cb, x, y, z, t);
        link_gradient<PREC, RECON, NF, 0>(a, par, cb, x, y, z, t, m);
    }
    store_links<0>(a, V, valid, m, tile);
    if (valid) {
        prefetch_dir<PREC, RECON, NF, 2>(a, par, cb, x, y, z, t);
        link_gradient<PREC, RECON, NF, 1>(a, par, cb, x, y, z, t, m);
    }
    store_links<1>(a, V, valid, m, tile);
    if (valid) {
        prefetch_dir<PREC, RECON, NF, 3>(a, par, cb, x, y, z, t);
        link_gradient<PREC, RECON, NF, 2>(a, par, cb, x, y, z, t, m);
    }
    store_links<2>(a, V, valid, m, tile);
    if (valid) link_gradient<PREC, RECON, NF, 3>(a, par, cb, x, y, z, t, m);
    store_links<3>(a, V, valid, m, tile);
}

}  // namespace tmk

using namespace tmk;

extern "C" tm_status tm_force(const tm_gauge *g, void *F_canon, int canon_type, const tm_field *psi_e,
                              const tm_field *psi_o, const tm_field *g_e, const tm_field *g_o, double coef,
                              int project, void *stream)
{
    TM_NVTX("tm_force");
    if (!g || !F_canon || !psi_e || !psi_o || !g_e || !g_o) { set_error("tm_force: null argument"); return TM_ERR_ARG; }
    if (g->csw != 0.0) {
        set_error("tm_force: the link derivative of the clover term is not implemented");
        return TM_ERR_ARG;
    }
    if (g->dd) { set_error("tm_force: the handle holds one time slab of a decomposed lattice"); return TM_ERR_ARG; }
    const tm_field *fs[4] = {psi_e, psi_o, g_e, g_o};
    for (auto f : fs) {
        if (!f->data || f->prec != psi_e->prec || f->nrhs != 1 || (f->prec == TM_PREC_F16 && !f->norm)) {
            set_error("tm_force: fields must be single-RHS and share one precision");
            return TM_ERR_ARG;
        }
    }
    if (psi_e->prec != TM_PREC_F64 && psi_e->prec != TM_PREC_F32) {
        set_error("tm_force: FP64 or FP32 fields only");
        return TM_ERR_ARG;
    }
    if (canon_type != TM_C128 && canon_type != TM_C64) { set_error("tm_force: unknown canon_type"); return TM_ERR_ARG; }
    ForceArgs a;
    a.psi[0] = psi_e->data;
    a.psi[1] = psi_o->data;
    a.gv[0] = g_e->data;
    a.gv[1] = g_o->data;
    a.psi_norm[0] = a.psi_norm[1] = a.gv_norm[0] = a.gv_norm[1] = nullptr;
    a.Vh = g->Vh;
    a.X1h = g->X1h;
    a.Lx = g->p.L[0];
    a.Ly = g->p.L[1];
    a.Lz = g->p.L[2];
    a.Lt = g->p.L[3];
    a.nf = g->nf;
    a.tbc = g->p.t_antiperiodic ? 1 : 0;
    a.project = project ? 1 : 0;
    a.coef = -g->p.kappa * coef;
    const int pidx = prec_index(psi_e->prec);
    if (need_links(g, psi_e->prec) != TM_OK) return TM_ERR_ARG;
    a.gauge = g->links[pidx];
    a.out = F_canon;
    if (((uintptr_t)F_canon & 15) != 0) { set_error("tm_force: the output must be 16-byte aligned"); return TM_ERR_ARG; }
    const long n = 2L * g->Vh;  // one thread per site
    const int block = 128;
    const long grid = (n + block - 1) / block;
    cudaStream_t s = (cudaStream_t)stream;
    const int recon = link_recon(g, pidx);
#define TM_F1(P, R, CT) \
    if (g->nf == 1) k_force<P, R, 1, CT><<<grid, block, 0, s>>>(a); else k_force<P, R, 2, CT><<<grid, block, 0, s>>>(a);
#define TM_FR(P, CT)                              \
    if (recon == 18) { TM_F1(P, 18, CT) }         \
    else if (recon == 12) { TM_F1(P, 12, CT) }    \
    else { TM_F1(P, 8, CT) }
    if (pidx == 0) {
        if (canon_type == TM_C128) { TM_FR(P64, double2) } else { TM_FR(P64, float2) }
    } else {
        if (canon_type == TM_C128) { TM_FR(P32, double2) } else { TM_FR(P32, float2) }
    }
#undef TM_FR
#undef TM_F1
    return cuda_check(cudaGetLastError(), "tm_force launch");
}

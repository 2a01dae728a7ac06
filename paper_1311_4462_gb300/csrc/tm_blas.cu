// tm_blas.cu -- site-wise kernels on parity fields: local twist, linear combinations,
// precision conversion and FP64-accumulated reductions for the CG solvers.
//
// Every kernel walks "site blocks": one (rhs, flavour, site) triple = the 24 reals of a site,
// so FP16 fields keep one norm per block.  Arithmetic is FP64 when any operand is stored in
// FP64, else FP32; reductions add each site's FP32/FP64 partial into an FP64 thread sum,
// reduce warps with shuffles, blocks through shared memory, and the last block to finish
// (atomic ticket) sums the per-block partials in block order -- deterministic for a fixed
// grid -- and applies a small scalar update (CG's alpha / beta) on the device.
#include "tm_blas.cuh"
#include "tm_internal.h"

namespace tmk {

// ---------------------------------------------------------------------------- twist
template <int PREC, int NF>
__global__ void k_twist(void *out, float *out_norm, const void *in, const float *in_norm, int Vh, int nrhs,
                        Twist<typename Traits<PREC>::real> tw, const int *act, int nact)
{
    using T = typename Traits<PREC>::real;
    using SC = typename Traits<PREC>::schunk;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)Vh * nact) return;
    const int cb = (int)(id % Vh);
    const long rhs = act ? (long)__ldg(act + id / Vh) : id / Vh;
    if (rhs < 0 || rhs >= nrhs) return;
    const long fstride = (long)Traits<PREC>::SCHUNKS * Vh;
    T v[NF][24];
#pragma unroll
    for (int f = 0; f < NF; f++) {
        const long blk = rhs * NF + f;
        load_spinor<PREC>(reinterpret_cast<const SC *>(in) + blk * fstride, in_norm ? in_norm + blk * Vh : nullptr, cb,
                          Vh, v[f]);
    }
    apply_twist<T, NF>(tw, v);
#pragma unroll
    for (int f = 0; f < NF; f++) {
        const long blk = rhs * NF + f;
        store_spinor<PREC>(reinterpret_cast<SC *>(out) + blk * fstride, out_norm ? out_norm + blk * Vh : nullptr, cb,
                           Vh, v[f]);
    }
}

template <typename T>
static Twist<T> cast_twist(const Twist<double> &t)
{
    Twist<T> o;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            for (int k = 0; k < 2; k++) o.m[i][j][k] = {(T)t.m[i][j][k].r, (T)t.m[i][j][k].i};
    return o;
}

cudaError_t launch_twist_active(const tm_gauge *g, const tm_field *out, const tm_field *in, const Twist<double> &tw,
                                const int *act, int nact, cudaStream_t s)
{
    const long n = (long)g->Vh * nact;
    const int block = 128;
    const long grid = (n + block - 1) / block;
#define TM_T(P, NF, TT)                                                                                          \
    k_twist<P, NF><<<grid, block, 0, s>>>(out->data, out->norm, in->data, in->norm, g->Vh, out->nrhs, cast_twist<TT>(tw), \
                                          act, nact)
    if (in->prec == TM_PREC_DF64) {
        if (g->nf == 1) TM_T(PDF, 1, df64);
        else TM_T(PDF, 2, df64);
    } else if (g->nf == 1) {
        if (in->prec == TM_PREC_F64) TM_T(P64, 1, double);
        else if (in->prec == TM_PREC_F32) TM_T(P32, 1, float);
        else TM_T(P16, 1, float);
    } else {
        if (in->prec == TM_PREC_F64) TM_T(P64, 2, double);
        else if (in->prec == TM_PREC_F32) TM_T(P32, 2, float);
        else TM_T(P16, 2, float);
    }
#undef TM_T
    return cudaGetLastError();
}

cudaError_t launch_twist(const tm_gauge *g, const tm_field *out, const tm_field *in, const Twist<double> &tw,
                         cudaStream_t s)
{
    return launch_twist_active(g, out, in, tw, nullptr, out->nrhs, s);
}

// ------------------------------------------------------------------------- generic site op
// One launch: for every site block, load operands a, b, c (any precision), compute
//   out = ca * a + cb * b   (op AXPBY)      -- then optional reduction of |out|^2
//   cg:  c += alpha * a ; b -= alpha * Ap  (op CG_UPDATE with a = p, d = Ap) -- reduction |b|^2
//   dot: reduce Re<a, b>                    (op DOT)
//   norm: reduce |a|^2                      (op NORM)
//   copy: out = a                           (op COPY)
//   g5dot: reduce Re / Im <a, gamma5 b>     (ops G5DOT_RE, G5DOT_IM)
// Coefficients come from SVal (host value or device scalar slot times a host multiplier).
__device__ __forceinline__ double sval(const SVal &v, int rhs, const double *S)
{
    return v.slot >= 0 ? v.mult * S[v.slot * TM_MAX_RHS + rhs] : v.value;
}

template <int PA, int PB, int PC, int PD, typename T>
__global__ void __launch_bounds__(256) k_site_op(SiteOpArgs a)
{
    const long nper = (long)a.Vh * a.nf;  // site blocks per rhs
    const int rhs = blockIdx.y;
    double acc = 0.0;
    const bool active = !a.red.active || a.red.active[rhs];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nper && active; i += (long)gridDim.x * blockDim.x) {
        const int cb = (int)(i % a.Vh);
        const long blk = (long)rhs * a.nf + i / a.Vh;
        T va[24], vb[24], vc[24], vd[24];
        (void)vc;
        T part = T(0);
        switch (a.op) {
        case OP_AXPBY: {
            const T ca = (T)sval(a.ca, rhs, a.red.scalars), cbv = (T)sval(a.cb, rhs, a.red.scalars);
            load_block<PA>(a.A, blk, cb, a.Vh, va);
            if (a.B.data) load_block<PB>(a.B, blk, cb, a.Vh, vb);
#pragma unroll
            for (int k = 0; k < 24; k++) {
                const T o = a.B.data ? fma(ca, va[k], cbv * vb[k]) : ca * va[k];
                va[k] = o;
            }
            store_block<PC>(a.C, blk, cb, a.Vh, va);  // va now holds the stored values
            if (a.reduce) {
#pragma unroll
                for (int k = 0; k < 24; k++) part = fma(va[k], va[k], part);
            }
            break;
        }
        case OP_CG_UPDATE: {  // A = p, B = r, C = x, D = Ap
            const T al = (T)sval(a.ca, rhs, a.red.scalars);
            load_block<PA>(a.A, blk, cb, a.Vh, va);
            load_block<PC>(a.C, blk, cb, a.Vh, vc);
#pragma unroll
            for (int k = 0; k < 24; k++) vc[k] = fma(al, va[k], vc[k]);
            store_block<PC>(a.C, blk, cb, a.Vh, vc);
            load_block<PB>(a.B, blk, cb, a.Vh, vb);
            load_block<PD>(a.D, blk, cb, a.Vh, vd);
#pragma unroll
            for (int k = 0; k < 24; k++) vb[k] = fma(-al, vd[k], vb[k]);
            store_block<PB>(a.B, blk, cb, a.Vh, vb);  // vb now holds the stored values
#pragma unroll
            for (int k = 0; k < 24; k++) part = fma(vb[k], vb[k], part);
            break;
        }
        case OP_R_UPDATE: {  // B = r, D = Ap: r -= alpha Ap, then |r|^2 (the residual half of CG_UPDATE)
            const T al = (T)sval(a.ca, rhs, a.red.scalars);
            load_block<PB>(a.B, blk, cb, a.Vh, vb);
            load_block<PD>(a.D, blk, cb, a.Vh, vd);
#pragma unroll
            for (int k = 0; k < 24; k++) vb[k] = fma(-al, vd[k], vb[k]);
            store_block<PB>(a.B, blk, cb, a.Vh, vb);
#pragma unroll
            for (int k = 0; k < 24; k++) part = fma(vb[k], vb[k], part);
            break;
        }
        case OP_XP_UPDATE: {  // A = p, C = x, D = r: x += alpha p, then p = r + beta p (one pass)
            const T al = (T)sval(a.ca, rhs, a.red.scalars), be = (T)sval(a.cb, rhs, a.red.scalars);
            load_block<PA>(a.A, blk, cb, a.Vh, va);
            load_block<PC>(a.C, blk, cb, a.Vh, vc);
#pragma unroll
            for (int k = 0; k < 24; k++) vc[k] = fma(al, va[k], vc[k]);
            store_block<PC>(a.C, blk, cb, a.Vh, vc);
            load_block<PD>(a.D, blk, cb, a.Vh, vd);
#pragma unroll
            for (int k = 0; k < 24; k++) va[k] = fma(T(1), vd[k], be * va[k]);
            store_block<PA>(a.A, blk, cb, a.Vh, va);
            break;
        }
        case OP_DOT: {
            load_block<PA>(a.A, blk, cb, a.Vh, va);
            load_block<PB>(a.B, blk, cb, a.Vh, vb);
#pragma unroll
            for (int k = 0; k < 24; k++) part = fma(va[k], vb[k], part);  // Re<a,b> = sum re*re + im*im
            break;
        }
        case OP_G5DOT_RE:    // Re <a, gamma5 b>: gamma5 = +1 on spins 0, 1 and -1 on spins 2, 3
        case OP_G5DOT_IM: {  // Im <a, gamma5 b>
            load_block<PA>(a.A, blk, cb, a.Vh, va);
            load_block<PB>(a.B, blk, cb, a.Vh, vb);
            const bool re = a.op == OP_G5DOT_RE;
#pragma unroll
            for (int j = 0; j < 12; j++) {
                const T sg = (j < 6) ? T(1) : T(-1);
                const T v = re ? fma(va[2 * j], vb[2 * j], va[2 * j + 1] * vb[2 * j + 1])
                               : fma(va[2 * j], vb[2 * j + 1], -va[2 * j + 1] * vb[2 * j]);
                part = fma(sg, v, part);
            }
            break;
        }
        case OP_NORM: {
            load_block<PA>(a.A, blk, cb, a.Vh, va);
#pragma unroll
            for (int k = 0; k < 24; k++) part = fma(va[k], va[k], part);
            break;
        }
        default: {  // OP_COPY
            load_block<PA>(a.A, blk, cb, a.Vh, va);
            store_block<PC>(a.C, blk, cb, a.Vh, va);
            break;
        }
        }
        acc += (double)part;
    }
    if (a.reduce) {
        const double s = block_sum(acc);
        grid_finish(s, a.red);
    }
}

template <int PA, int PB, int PC, int PD>
static cudaError_t run_combo(const SiteOpArgs &a, dim3 grid, int block, cudaStream_t s)
{
    // arithmetic: binary64 if any operand is FP64, double-float if any is DF64, else binary32
    constexpr bool any64 = (PA == P64) || (PB == P64) || (PC == P64) || (PD == P64);
    constexpr bool anydf = (PA == PDF) || (PB == PDF) || (PC == PDF) || (PD == PDF);
    if constexpr (any64) k_site_op<PA, PB, PC, PD, double><<<grid, block, 0, s>>>(a);
    else if constexpr (anydf) k_site_op<PA, PB, PC, PD, df64><<<grid, block, 0, s>>>(a);
    else k_site_op<PA, PB, PC, PD, float><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

// precision of a possibly-absent operand; an absent operand takes the first operand's
static int pc_of(const FieldRef &f, int dflt) { return f.data ? f.prec : dflt; }

// The operand precision combinations (A, B, C, D) the solvers use.
#define TM_COMBOS(X)          \
    X(P64, P64, P64, P64)     \
    X(P32, P32, P32, P32)     \
    X(P16, P16, P16, P16)     \
    X(P16, P16, P32, P16)     \
    X(P16, P32, P32, P16)     \
    X(P32, P64, P64, P32)     \
    X(P64, P64, P32, P64)     \
    X(P64, P64, P16, P64)     \
    X(P32, P32, P64, P32)     \
    X(P16, P16, P64, P16)     \
    X(P32, P32, P16, P32)     \
    X(PDF, PDF, PDF, PDF)     \
    X(P64, P64, PDF, P64)     \
    X(PDF, PDF, P64, PDF)     \
    X(P32, PDF, PDF, P32)     \
    X(PDF, PDF, P32, PDF)     \
    X(PDF, PDF, P16, PDF)

// The end of a reduction whose partial sums another kernel wrote (the hopping kernel's fused
// reduction, one partial per warp), then the scalar update, in one block.  Thread t adds partials t, t + 1024, t + 2048, ... into four independent running sums (index
// (b / 1024) mod 4), which it combines as (s0 + s1) + (s2 + s3); the block then sums the threads in
// block_sum's fixed order.  The order depends only on n, so the result is reproducible, and the
// four chains keep four loads in flight per thread.
__global__ void __launch_bounds__(1024) k_finish_partials(const double *__restrict__ partials, long n, RedArgs r)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const long t = threadIdx.x;
    long b = t;
    for (; b + 3 * 1024 < n; b += 4 * 1024) {
        s0 += partials[b];
        s1 += partials[b + 1024];
        s2 += partials[b + 2 * 1024];
        s3 += partials[b + 3 * 1024];
    }
    if (b < n) s0 += partials[b];
    if (b + 1024 < n) s1 += partials[b + 1024];
    if (b + 2 * 1024 < n) s2 += partials[b + 2 * 1024];
    double s = block_sum((s0 + s1) + (s2 + s3));
    if (threadIdx.x == 0) apply_fin(s, r, 0);
}

cudaError_t launch_finish_partials(const double *partials, long n, const RedArgs &r, cudaStream_t s)
{
    k_finish_partials<<<1, 1024, 0, s>>>(partials, n, r);
    return cudaGetLastError();
}

cudaError_t launch_site_op(const tm_gauge *g, SiteOpArgs a, int nrhs, cudaStream_t s)
{
    a.Vh = g->Vh;
    a.nf = g->nf;
    const int block = 256;
    const long nper = (long)a.Vh * a.nf;
    long gx = (nper + block - 1) / block;
    const long cap = (long)g->num_sms * 4;
    if (gx > cap) gx = cap;
    const long maxcols = (long)((g->scratch_bytes - SCRATCH_PARTIALS_OFF) / sizeof(double)) / nrhs;
    if (a.reduce && gx > maxcols) gx = maxcols;
    dim3 grid((unsigned)gx, (unsigned)nrhs);
    a.red.partials = reinterpret_cast<double *>(reinterpret_cast<char *>(g->scratch) + SCRATCH_PARTIALS_OFF);
    a.red.counter = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(g->scratch) + SCRATCH_COUNTER_OFF);
    if (!a.red.scalars) a.red.scalars = g->scratch;
    const int pa = a.A.prec;
    const int pb = pc_of(a.B, pa), pc = pc_of(a.C, pa), pd = pc_of(a.D, pa);
#define TM_TRY_COMBO(A_, B_, C_, D_) \
    if (pa == A_ && pb == B_ && pc == C_ && pd == D_) return run_combo<A_, B_, C_, D_>(a, grid, block, s);
    TM_COMBOS(TM_TRY_COMBO)
#undef TM_TRY_COMBO
    return cudaErrorNotSupported;
}

}  // namespace tmk

namespace tmk {

// Launch of k_site_op with caller-supplied reduction scratch and geometry (no gauge handle):
// grid.x blocks per rhs column, 256 threads, partials/counter taken from a.red as given.
cudaError_t launch_site_op_explicit(SiteOpArgs a, int Vh, int nf, int grid_x, int nrhs, cudaStream_t s)
{
    a.Vh = Vh;
    a.nf = nf;
    const int block = 256;
    dim3 grid((unsigned)grid_x, (unsigned)nrhs);
    const int pa = a.A.prec;
    const int pb = pc_of(a.B, pa), pc = pc_of(a.C, pa), pd = pc_of(a.D, pa);
#define TM_TRY_COMBO(A_, B_, C_, D_) \
    if (pa == A_ && pb == B_ && pc == C_ && pd == D_) return run_combo<A_, B_, C_, D_>(a, grid, block, s);
    TM_COMBOS(TM_TRY_COMBO)
#undef TM_TRY_COMBO
    return cudaErrorNotSupported;
}

}  // namespace tmk

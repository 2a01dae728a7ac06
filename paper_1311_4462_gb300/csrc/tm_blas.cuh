// tm_blas.cuh -- argument structs and block codecs for the site-wise kernels (tm_blas.cu)
// and the solvers (tm_solver.cu).
#pragma once
#include "tm_core.cuh"
#include "tm_internal.h"

namespace tmk {

constexpr int TM_MAX_RHS = 64;  // columns of the device scalar table

// device scalar table: scalars[slot * TM_MAX_RHS + rhs]
enum Slot { SL_RR = 0, SL_RRNEW = 1, SL_PAP = 2, SL_ALPHA = 3, SL_BETA = 4, SL_TMP0 = 5, SL_TMP1 = 6, SL_TMP2 = 7,
            SL_COUNT = 16 };
// scratch layout inside the gauge handle's scratch area
constexpr size_t SCRATCH_SCALARS_OFF = 0;                                       // 16 x 64 doubles
constexpr size_t SCRATCH_COUNTER_OFF = SL_COUNT * TM_MAX_RHS * sizeof(double);  // 8 KB: ticket counter
constexpr size_t SCRATCH_PARTIALS_OFF = 16384;                                  // per-block partial sums

enum SiteOpCode { OP_AXPBY = 0, OP_CG_UPDATE = 1, OP_DOT = 2, OP_NORM = 3, OP_COPY = 4, OP_G5DOT_RE = 5, OP_G5DOT_IM = 6,
                  OP_R_UPDATE = 7, OP_XP_UPDATE = 8 };
enum FinCode { FIN_STORE = 0, FIN_ALPHA = 1, FIN_BETA = 2 };

struct FieldRef {
    void *data;
    float *norm;
    int prec;
};

// a coefficient: host value, or mult * scalars[slot][rhs] when slot >= 0
struct SVal {
    double value;
    int slot;
    double mult;
};

struct RedArgs {
    double *partials;
    unsigned *counter;
    double *scalars;
    const int *active;  // per-rhs mask (NULL: all active)
    int fin;
    int slot;
};

struct SiteOpArgs {
    int op;
    int reduce;
    FieldRef A, B, C, D;
    SVal ca, cb;
    RedArgs red;
    int Vh, nf;
};

// Load / store one site block (blk = rhs * nf + flavour) of a field given by FieldRef.
template <int PREC, typename T>
__device__ __forceinline__ void load_block(const FieldRef &f, long blk, int cb, int Vh, T v[24])
{
    using SC = typename Traits<PREC>::schunk;
    using R = typename Traits<PREC>::real;
    R tmp[24];
    const SC *p = reinterpret_cast<const SC *>(f.data) + blk * Traits<PREC>::SCHUNKS * (long)Vh;
    load_spinor<PREC>(p, f.norm ? f.norm + blk * Vh : nullptr, cb, Vh, tmp);
#pragma unroll
    for (int k = 0; k < 24; k++) v[k] = (T)tmp[k];
}

// Stores v and replaces it by the value as stored (rounded to the storage precision), so a
// following reduction sees exactly what was written without reading memory back.
template <int PREC, typename T>
__device__ __forceinline__ void store_block(const FieldRef &f, long blk, int cb, int Vh, T v[24])
{
    using SC = typename Traits<PREC>::schunk;
    using R = typename Traits<PREC>::real;
    R tmp[24];
#pragma unroll
    for (int k = 0; k < 24; k++) tmp[k] = (R)v[k];
    SC *p = reinterpret_cast<SC *>(f.data) + blk * Traits<PREC>::SCHUNKS * (long)Vh;
    store_spinor<PREC>(p, f.norm ? f.norm + blk * Vh : nullptr, cb, Vh, tmp);
    if constexpr (PREC == P16) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 24; k++) m = fmaxf(m, fabsf((float)tmp[k]));
        const float inv = (m > 0.f) ? 1.0f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 24; k++) v[k] = (T)(__half2float(__float2half_rn((float)tmp[k] * inv)) * m);
    } else {
#pragma unroll
        for (int k = 0; k < 24; k++) v[k] = (T)tmp[k];
    }
}

// ---------------------------------------------------------------------------- reductions
// (shared by the site-wise kernels and the hopping kernel's fused epilogue reduction)
// Block-level sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (warp == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Write this block's partial for column `col` (one column per rhs = blockIdx.y); the last block
// of the whole grid sums every column in block order and applies `fin` per column.
// The scalar update that ends a reduction of column c (one right-hand side) with the sum s.
__device__ __forceinline__ void apply_fin(double s, const RedArgs &r, int c)
{
    double *S = r.scalars;
    const int R = TM_MAX_RHS;
    const bool active = !r.active || r.active[c];
    switch (r.fin) {
    case FIN_STORE: S[r.slot * R + c] = s; break;
    case FIN_ALPHA:  // pAp -> alpha = rr / pAp
        S[SL_PAP * R + c] = s;
        S[SL_ALPHA * R + c] = (active && s != 0.0) ? S[SL_RR * R + c] / s : 0.0;
        break;
    case FIN_BETA:  // |r|^2 new -> beta = rr_new / rr, rr = rr_new
        S[SL_RRNEW * R + c] = s;
        S[SL_BETA * R + c] = (active && S[SL_RR * R + c] != 0.0) ? s / S[SL_RR * R + c] : 0.0;
        if (active) S[SL_RR * R + c] = s;
        break;
    }
}

__device__ __forceinline__ void grid_finish(double part, const RedArgs &r)
{
    const int col = blockIdx.y;
    if (threadIdx.x == 0) r.partials[(size_t)col * gridDim.x + blockIdx.x] = part;
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned total = gridDim.x * gridDim.y;
        last = (atomicAdd(r.counter, 1u) == total - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block sums each column: thread t the partials t, t + blockDim, ... in order, then the
    // block tree -- a fixed order for a given grid, so the result is reproducible
    for (int c = 0; c < (int)gridDim.y; c++) {
        double s = 0.0;
        const volatile double *pp = r.partials + (size_t)c * gridDim.x;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += pp[b];
        s = block_sum(s);
        __syncthreads();  // block_sum's shared slots are reused by the next column
        if (threadIdx.x == 0) apply_fin(s, r, c);
    }
    if (threadIdx.x == 0) *r.counter = 0u;  // ready for the next launch on this stream
}

cudaError_t launch_site_op(const tm_gauge *g, SiteOpArgs a, int nrhs, cudaStream_t s);
// one block sums n partials (column 0) in a fixed order and applies r.fin (tm_blas.cu)
cudaError_t launch_finish_partials(const double *partials, long n, const RedArgs &r, cudaStream_t s);

inline FieldRef fref(const tm_field *f) { return FieldRef{f->data, f->norm, f->prec}; }
inline FieldRef fnone() { return FieldRef{nullptr, nullptr, 0}; }
inline SVal sv(double v) { return SVal{v, -1, 1.0}; }
inline SVal sslot(int slot, double mult) { return SVal{0.0, slot, mult}; }

}  // namespace tmk

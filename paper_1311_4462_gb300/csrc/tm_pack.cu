// tm_pack.cu -- conversion between the canonical full-lattice layout and the internal
// parity-split structure-of-arrays fields, and the packed link codecs (sec. 2, sec. 3).
#include <math.h>

#include "tm_core.cuh"
#include "tm_internal.h"

namespace tmk {

template <typename CT> struct CanonT;
template <> struct CanonT<double2> { using real = double; };
template <> struct CanonT<float2> { using real = float; };

// lexicographic site of (parity, cb)
__device__ __forceinline__ long lex_of(int cb, int parity, int X1h, int Lx, int Ly, int Lz)
{
    int r = cb;
    const int xh = r % X1h;
    r /= X1h;
    const int y = r % Ly;
    r /= Ly;
    const int z = r % Lz;
    const int t = r / Lz;
    const int x = 2 * xh + ((parity + y + z + t) & 1);
    return x + (long)Lx * (y + (long)Ly * (z + (long)Lz * t));
}

struct Geo {
    int Vh, X1h, Lx, Ly, Lz, nf, nrhs;
};

// Storage forms whose 16-byte chunks are the canonical field's own bytes (FP32 fields from
// complex64, FP64 fields from complex128): a block moves 32 sites of one parity through shared
// memory, reading the canonical sites whole (16-byte loads, consecutive threads on consecutive
// bytes) and writing each SoA row with consecutive threads on consecutive sites.  Both sides are
// coalesced, which matters most when the canonical buffer is pinned host memory read over the
// CPU-GPU link.  NCH = chunks per site = flavours x chunks per flavour.
template <int NCH>
__global__ void __launch_bounds__(128) k_pack_chunks(uint4 *out, const uint4 *canon, int parity, Geo g)
{
    constexpr int S = 32;
    __shared__ uint4 sm[S * NCH];
    const long nsites = (long)g.Vh * g.nrhs;
    const long V = 2L * g.Vh;
    // grid-stride over groups of S sites with a grid of at most 4 blocks per SM, so a pack and an
    // unpack on two streams can be resident together
    for (long site0 = (long)blockIdx.x * S; site0 < nsites; site0 += (long)gridDim.x * S) {
        for (int i = threadIdx.x; i < S * NCH; i += blockDim.x) {
            const int si = i / NCH, j = i % NCH;
            const long gs = site0 + si;
            if (gs < nsites) {
                const long rhs = gs / g.Vh;
                const int cb = (int)(gs - rhs * g.Vh);
                const long lex = lex_of(cb, parity, g.X1h, g.Lx, g.Ly, g.Lz);
                sm[i] = canon[(rhs * V + lex) * NCH + j];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < S * NCH; i += blockDim.x) {
            const int j = i / S, si = i % S;
            const long gs = site0 + si;
            if (gs < nsites) {
                const long rhs = gs / g.Vh;
                const int cb = (int)(gs - rhs * g.Vh);
                out[(rhs * NCH + j) * g.Vh + cb] = sm[si * NCH + j];
            }
        }
        __syncthreads();
    }
}

template <int NCH>
__global__ void __launch_bounds__(128) k_unpack_chunks(uint4 *canon, const uint4 *in, int parity, Geo g)
{
    constexpr int S = 32;
    __shared__ uint4 sm[S * NCH];
    const long nsites = (long)g.Vh * g.nrhs;
    const long V = 2L * g.Vh;
    for (long site0 = (long)blockIdx.x * S; site0 < nsites; site0 += (long)gridDim.x * S) {
        for (int i = threadIdx.x; i < S * NCH; i += blockDim.x) {
            const int j = i / S, si = i % S;
            const long gs = site0 + si;
            if (gs < nsites) {
                const long rhs = gs / g.Vh;
                const int cb = (int)(gs - rhs * g.Vh);
                sm[si * NCH + j] = in[(rhs * NCH + j) * g.Vh + cb];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < S * NCH; i += blockDim.x) {
            const int si = i / NCH, j = i % NCH;
            const long gs = site0 + si;
            if (gs < nsites) {
                const long rhs = gs / g.Vh;
                const int cb = (int)(gs - rhs * g.Vh);
                const long lex = lex_of(cb, parity, g.X1h, g.Lx, g.Ly, g.Lz);
                canon[(rhs * V + lex) * NCH + j] = sm[i];
            }
        }
        __syncthreads();
    }
}

// number of 16-byte chunks per site when the field's chunks are the canonical bytes (and the
// canonical buffer is 16-byte aligned), else 0
static int direct_chunks(const Geo &G, int prec, int ctype, const void *canon)
{
    if (((uintptr_t)canon & 15) != 0) return 0;
    if (prec == TM_PREC_F32 && ctype == TM_C64) return 6 * G.nf;
    if (prec == TM_PREC_F64 && ctype == TM_C128) return 12 * G.nf;
    return 0;
}

// thread per (rhs, flavour, cb)
template <int PREC, typename CT>
__global__ void k_pack_spinor(void *out, float *norm, const CT *canon, int parity, Geo g)
{
    using T = typename Traits<PREC>::real;
    using SC = typename Traits<PREC>::schunk;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nsite = (long)g.Vh * g.nf * g.nrhs;
    if (id >= nsite) return;
    const int cb = (int)(id % g.Vh);
    const int f = (int)((id / g.Vh) % g.nf);
    const int rhs = (int)(id / ((long)g.Vh * g.nf));
    const long lex = lex_of(cb, parity, g.X1h, g.Lx, g.Ly, g.Lz);
    const long V = 2L * g.Vh;
    const CT *src = canon + (((long)rhs * V + lex) * g.nf + f) * 12;
    T v[24];
#pragma unroll
    for (int k = 0; k < 12; k++) {
        CT c = src[k];
        v[2 * k] = (T)c.x;
        v[2 * k + 1] = (T)c.y;
    }
    const long blk = (long)rhs * g.nf + f;  // flavour block index
    SC *o = reinterpret_cast<SC *>(out) + blk * Traits<PREC>::SCHUNKS * (long)g.Vh;
    store_spinor<PREC>(o, norm ? norm + blk * g.Vh : nullptr, cb, g.Vh, v);
}

template <int PREC, typename CT>
__global__ void k_unpack_spinor(CT *canon, const void *in, const float *norm, int parity, Geo g)
{
    using T = typename Traits<PREC>::real;
    using SC = typename Traits<PREC>::schunk;
    using R = typename CanonT<CT>::real;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nsite = (long)g.Vh * g.nf * g.nrhs;
    if (id >= nsite) return;
    const int cb = (int)(id % g.Vh);
    const int f = (int)((id / g.Vh) % g.nf);
    const int rhs = (int)(id / ((long)g.Vh * g.nf));
    const long lex = lex_of(cb, parity, g.X1h, g.Lx, g.Ly, g.Lz);
    const long V = 2L * g.Vh;
    const long blk = (long)rhs * g.nf + f;
    const SC *p = reinterpret_cast<const SC *>(in) + blk * Traits<PREC>::SCHUNKS * (long)g.Vh;
    T v[24];
    load_spinor<PREC>(p, norm ? norm + blk * g.Vh : nullptr, cb, g.Vh, v);
    CT *dst = canon + (((long)rhs * V + lex) * g.nf + f) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        CT c;
        c.x = (R)v[2 * k];
        c.y = (R)v[2 * k + 1];
        dst[k] = c;
    }
}

// ------------------------------------------------------------------------------------ links
// Reals of one link in storage order for the given recon (see tm_core.cuh).
__device__ __forceinline__ int encode_link(const double2 *u, int recon, double r[18])
{
    if (recon == 8) {
        r[0] = u[1].x; r[1] = u[1].y;  // a2
        r[2] = u[2].x; r[3] = u[2].y;  // a3
        r[4] = u[3].x; r[5] = u[3].y;  // b1
        r[6] = atan2(u[0].y, u[0].x);  // arg a1
        r[7] = atan2(u[6].y, u[6].x);  // arg c1
        return 8;
    }
    const int n = (recon == 18) ? 9 : 6;
    for (int k = 0; k < n; k++) {
        r[2 * k] = u[k].x;
        r[2 * k + 1] = u[k].y;
    }
    return 2 * n;
}

// thread per (mu, parity, cb); writes chunk k of link (mu, parity, cb) at base + ((mu*2+par)*N + k)*Vh + cb
template <int PREC>
__global__ void k_pack_gauge(void *out, const double2 *canon, int recon, Geo g)
{
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= 8L * g.Vh) return;
    const int cb = (int)(id % g.Vh);
    const int par = (int)((id / g.Vh) % 2);
    const int mu = (int)(id / (2L * g.Vh));
    const long lex = lex_of(cb, par, g.X1h, g.Lx, g.Ly, g.Lz);
    const long V = 2L * g.Vh;
    const double2 *u = canon + ((long)mu * V + lex) * 9;
    double r[18];
    const int nr = encode_link(u, recon, r);
    const long slot = (long)(mu * 2 + par);
    if (PREC == P64) {
        const int N = nr / 2;
        double2 *o = reinterpret_cast<double2 *>(out) + slot * N * (long)g.Vh + cb;
        for (int k = 0; k < N; k++) o[(long)k * g.Vh] = make_double2(r[2 * k], r[2 * k + 1]);
    } else if (PREC == PDF) {
        // (hi, lo) pairs of two reals per float4; 8-real storage is not used for DF64 (12 reals)
        const int nre = (recon == 18) ? 18 : 12;
        if (recon == 8) encode_link(u, 12, r);
        const int N = nre / 2;
        float4 *o = reinterpret_cast<float4 *>(out) + slot * N * (long)g.Vh + cb;
        for (int k = 0; k < N; k++) {
            const df64 a(r[2 * k]), b(r[2 * k + 1]);
            o[(long)k * g.Vh] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
    } else if (PREC == P32) {
        if (recon == 18) {
            float2 *o = reinterpret_cast<float2 *>(out) + slot * 9 * (long)g.Vh + cb;
            for (int k = 0; k < 9; k++) o[(long)k * g.Vh] = make_float2((float)r[2 * k], (float)r[2 * k + 1]);
        } else {
            const int N = nr / 4;
            float4 *o = reinterpret_cast<float4 *>(out) + slot * N * (long)g.Vh + cb;
            for (int k = 0; k < N; k++)
                o[(long)k * g.Vh] = make_float4((float)r[4 * k], (float)r[4 * k + 1], (float)r[4 * k + 2],
                                                (float)r[4 * k + 3]);
        }
    } else {
        if (recon == 8) {
            r[6] /= 3.14159265358979323846;
            r[7] /= 3.14159265358979323846;
        }
        if (recon == 18) {
            uint32_t *o = reinterpret_cast<uint32_t *>(out) + slot * 9 * (long)g.Vh + cb;
            for (int k = 0; k < 9; k++) o[(long)k * g.Vh] = f2h((float)r[2 * k], (float)r[2 * k + 1]);
        } else if (recon == 12) {
            uint2 *o = reinterpret_cast<uint2 *>(out) + slot * 3 * (long)g.Vh + cb;
            for (int k = 0; k < 3; k++)
                o[(long)k * g.Vh] = make_uint2(f2h((float)r[4 * k], (float)r[4 * k + 1]),
                                               f2h((float)r[4 * k + 2], (float)r[4 * k + 3]));
        } else {
            uint4 *o = reinterpret_cast<uint4 *>(out) + slot * (long)g.Vh + cb;
            uint4 c;
            c.x = f2h((float)r[0], (float)r[1]);
            c.y = f2h((float)r[2], (float)r[3]);
            c.z = f2h((float)r[4], (float)r[5]);
            c.w = f2h((float)r[6], (float)r[7]);
            *o = c;
        }
    }
}

// ------------------------------------------------------------------------------ Z2 noise
// Element i of source `seed` (flat index into the canonical layout [Lt][Lz][Ly][Lx][nf][4][3]):
// sign bits of SplitMix64's output function (Steele, Lea & Flood, OOPSLA 2014) at the counter
// state (seed + 1) G + (i + 1) G, G = 0x9E3779B97F4A7C15: bit 0 -> real, bit 1 -> imaginary,
// value (+-1 +- i)/sqrt(2).  Right-hand side r of the field uses seed + r.
__device__ __forceinline__ unsigned long long splitmix64_out(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <int PREC>
__global__ void k_noise_z2(void *out, float *norm, int parity, unsigned long long seed, Geo g)
{
    using T = typename Traits<PREC>::real;
    using SC = typename Traits<PREC>::schunk;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)g.Vh * g.nf * g.nrhs) return;
    const int cb = (int)(id % g.Vh);
    const int f = (int)((id / g.Vh) % g.nf);
    const int rhs = (int)(id / ((long)g.Vh * g.nf));
    const long lex = lex_of(cb, parity, g.X1h, g.Lx, g.Ly, g.Lz);
    const unsigned long long G = 0x9E3779B97F4A7C15ull;
    const unsigned long long base = (seed + rhs + 1ull) * G;
    const T h = (T)0.70710678118654752440;  // 1/sqrt(2)
    const T mh = -h;
    T v[24];
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const unsigned long long i = (unsigned long long)((lex * g.nf + f) * 12 + k);
        const unsigned long long z = splitmix64_out(base + (i + 1ull) * G);
        v[2 * k] = (z & 1ull) ? mh : h;
        v[2 * k + 1] = (z & 2ull) ? mh : h;
    }
    const long blk = (long)rhs * g.nf + f;
    SC *o = reinterpret_cast<SC *>(out) + blk * Traits<PREC>::SCHUNKS * (long)g.Vh;
    store_spinor<PREC>(o, norm ? norm + blk * g.Vh : nullptr, cb, g.Vh, v);
}

static Geo geo_of(const tm_gauge *g, int nrhs)
{
    Geo G;
    G.Vh = g->Vh;
    G.X1h = g->X1h;
    G.Lx = g->p.L[0];
    G.Ly = g->p.L[1];
    G.Lz = g->p.L[2];
    G.nf = g->nf;
    G.nrhs = nrhs;
    return G;
}

cudaError_t launch_pack_spinor(const tm_gauge *g, const tm_field *f, const void *canon, int ctype, int parity,
                               cudaStream_t s)
{
    Geo G = geo_of(g, f->nrhs);
    if (const int nch = direct_chunks(G, f->prec, ctype, canon)) {
        const long groups = ((long)G.Vh * G.nrhs + 31) / 32;
        const long cap = g->num_sms > 0 ? 4L * g->num_sms : 608L;
        const long grid = groups < cap ? groups : cap;
        uint4 *o = (uint4 *)f->data;
        const uint4 *c = (const uint4 *)canon;
        if (nch == 6) k_pack_chunks<6><<<grid, 128, 0, s>>>(o, c, parity, G);
        else if (nch == 12) k_pack_chunks<12><<<grid, 128, 0, s>>>(o, c, parity, G);
        else k_pack_chunks<24><<<grid, 128, 0, s>>>(o, c, parity, G);
        return cudaGetLastError();
    }
    const long n = (long)G.Vh * G.nf * G.nrhs;
    const int block = 128;
    const long grid = (n + block - 1) / block;
#define TM_P(P, CT) k_pack_spinor<P, CT><<<grid, block, 0, s>>>(f->data, f->norm, (const CT *)canon, parity, G)
    if (f->prec == TM_PREC_DF64) {
        if (ctype == TM_C128) TM_P(PDF, double2);
        else TM_P(PDF, float2);
    } else if (ctype == TM_C128) {
        if (f->prec == TM_PREC_F64) TM_P(P64, double2);
        else if (f->prec == TM_PREC_F32) TM_P(P32, double2);
        else TM_P(P16, double2);
    } else {
        if (f->prec == TM_PREC_F64) TM_P(P64, float2);
        else if (f->prec == TM_PREC_F32) TM_P(P32, float2);
        else TM_P(P16, float2);
    }
#undef TM_P
    return cudaGetLastError();
}

cudaError_t launch_unpack_spinor(const tm_gauge *g, void *canon, int ctype, const tm_field *f, int parity,
                                 cudaStream_t s)
{
    Geo G = geo_of(g, f->nrhs);
    if (const int nch = direct_chunks(G, f->prec, ctype, canon)) {
        const long groups = ((long)G.Vh * G.nrhs + 31) / 32;
        const long cap = g->num_sms > 0 ? 4L * g->num_sms : 608L;
        const long grid = groups < cap ? groups : cap;
        uint4 *c = (uint4 *)canon;
        const uint4 *i = (const uint4 *)f->data;
        if (nch == 6) k_unpack_chunks<6><<<grid, 128, 0, s>>>(c, i, parity, G);
        else if (nch == 12) k_unpack_chunks<12><<<grid, 128, 0, s>>>(c, i, parity, G);
        else k_unpack_chunks<24><<<grid, 128, 0, s>>>(c, i, parity, G);
        return cudaGetLastError();
    }
    const long n = (long)G.Vh * G.nf * G.nrhs;
    const int block = 128;
    const long grid = (n + block - 1) / block;
#define TM_U(P, CT) k_unpack_spinor<P, CT><<<grid, block, 0, s>>>((CT *)canon, f->data, f->norm, parity, G)
    if (f->prec == TM_PREC_DF64) {
        if (ctype == TM_C128) TM_U(PDF, double2);
        else TM_U(PDF, float2);
    } else if (ctype == TM_C128) {
        if (f->prec == TM_PREC_F64) TM_U(P64, double2);
        else if (f->prec == TM_PREC_F32) TM_U(P32, double2);
        else TM_U(P16, double2);
    } else {
        if (f->prec == TM_PREC_F64) TM_U(P64, float2);
        else if (f->prec == TM_PREC_F32) TM_U(P32, float2);
        else TM_U(P16, float2);
    }
#undef TM_U
    return cudaGetLastError();
}

cudaError_t launch_noise_z2(const tm_gauge *g, const tm_field *f, int parity, unsigned long long seed, cudaStream_t s)
{
    Geo G = geo_of(g, f->nrhs);
    const long n = (long)G.Vh * G.nf * G.nrhs;
    const int block = 128;
    const long grid = (n + block - 1) / block;
    if (f->prec == TM_PREC_DF64) k_noise_z2<PDF><<<grid, block, 0, s>>>(f->data, f->norm, parity, seed, G);
    else if (f->prec == TM_PREC_F64) k_noise_z2<P64><<<grid, block, 0, s>>>(f->data, f->norm, parity, seed, G);
    else if (f->prec == TM_PREC_F32) k_noise_z2<P32><<<grid, block, 0, s>>>(f->data, f->norm, parity, seed, G);
    else k_noise_z2<P16><<<grid, block, 0, s>>>(f->data, f->norm, parity, seed, G);
    return cudaGetLastError();
}

cudaError_t launch_pack_gauge(const tm_gauge *g, int pidx, void *out, const void *canon, cudaStream_t s)
{
    Geo G = geo_of(g, 1);
    const long n = 8L * G.Vh;
    const int block = 128;
    const long grid = (n + block - 1) / block;
    const double2 *c = (const double2 *)canon;
    if (pidx == 0) k_pack_gauge<P64><<<grid, block, 0, s>>>(out, c, link_recon(g, pidx), G);
    else if (pidx == 1) k_pack_gauge<P32><<<grid, block, 0, s>>>(out, c, link_recon(g, pidx), G);
    else if (pidx == 2) k_pack_gauge<P16><<<grid, block, 0, s>>>(out, c, link_recon(g, pidx), G);
    else k_pack_gauge<PDF><<<grid, block, 0, s>>>(out, c, link_recon(g, pidx), G);
    return cudaGetLastError();
}

}  // namespace tmk

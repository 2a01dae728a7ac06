// tm_core.cuh -- device-side field layout, storage codecs and complex helpers.
//
// Internal layout (per parity, structure of arrays, one thread per site):
//   spinor field : [rhs][flavour][chunk][Vh]  with the 24 reals of a site
//                  ordered (spin*3 + colour)*2 + re/im and cut into 16-byte
//                  chunks (FP64: 12 x double2, FP32: 6 x float4,
//                  FP16: 3 x 8 halves) so a warp loads 512 contiguous bytes
//                  per chunk; FP16 adds a float norm array [rhs][flavour][Vh]
//                  holding the max |real| of the site (value = half * norm).
//   gauge field  : [mu][parity][chunk][Vh] per precision, rows of U_mu(x)
//                  stored first-row-first: 18 reals (recon 18), the first two
//                  rows (recon 12; row 3 = conj(row1 x row2) on load) or
//                  8 reals (recon 8, see decode_link8).
// The time-boundary sign is never folded into stored links (det(-U) = -1
// would break the 12/8-real rebuild); kernels apply it on the hop.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tm_df64.cuh"

namespace tmk {

template <typename T>
struct C {
    T r, i;
};

template <typename T> __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T> __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T> __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b)
{
    return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
// conj(a) * b
template <typename T> __device__ __forceinline__ C<T> cmulc(C<T> a, C<T> b)
{
    return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r};
}
template <typename T> __device__ __forceinline__ C<T> cconj(C<T> a) { return {a.r, -a.i}; }
template <typename T> __device__ __forceinline__ C<T> cscale(T s, C<T> a) { return {s * a.r, s * a.i}; }

// -------------------------------------------------------------------------------------------------
// Precision traits.  `real` is the arithmetic type; FP16 storage computes in FP32.
// PDF: double-float pairs (tm_df64.cuh), 8 bytes per real like P64, arithmetic on the FP32 pipes
enum Prec { P64 = 8, P32 = 4, P16 = 2, PDF = 16 };

template <int PREC> struct Traits;
template <> struct Traits<P64> {
    using real = double;
    using schunk = double2;   // spinor chunk
    static constexpr int SCHUNKS = 12;
    static constexpr bool NORM = false;
};
template <> struct Traits<P32> {
    using real = float;
    using schunk = float4;
    static constexpr int SCHUNKS = 6;
    static constexpr bool NORM = false;
};
template <> struct Traits<PDF> {
    using real = df64;
    using schunk = float4;    // (hi, lo) of two reals
    static constexpr int SCHUNKS = 12;
    static constexpr bool NORM = false;
};
template <> struct Traits<P16> {
    using real = float;
    using schunk = uint4;     // 8 halves
    static constexpr int SCHUNKS = 3;
    static constexpr bool NORM = true;
};

// Link chunk geometry per (precision, recon).
template <int PREC, int RECON> struct LinkLayout;
template <> struct LinkLayout<P64, 18> { using chunk = double2; static constexpr int N = 9; };
template <> struct LinkLayout<P64, 12> { using chunk = double2; static constexpr int N = 6; };
template <> struct LinkLayout<P64, 8>  { using chunk = double2; static constexpr int N = 4; };
template <> struct LinkLayout<P32, 18> { using chunk = float2; static constexpr int N = 9; };
template <> struct LinkLayout<P32, 12> { using chunk = float4; static constexpr int N = 3; };
template <> struct LinkLayout<P32, 8>  { using chunk = float4; static constexpr int N = 2; };
template <> struct LinkLayout<PDF, 18> { using chunk = float4; static constexpr int N = 9; };
template <> struct LinkLayout<PDF, 12> { using chunk = float4; static constexpr int N = 6; };
template <> struct LinkLayout<P16, 18> { using chunk = uint32_t; static constexpr int N = 9; };   // 2 halves
template <> struct LinkLayout<P16, 12> { using chunk = uint2; static constexpr int N = 3; };      // 4 halves
template <> struct LinkLayout<P16, 8>  { using chunk = uint4; static constexpr int N = 1; };      // 8 halves

// -------------------------------------------------------------------------------------------------
// Read-only global loads (non-coherent path; inputs are never written by the same launch).
template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }
__device__ __forceinline__ uint32_t ldg(const uint32_t *p) { return __ldg(p); }

__device__ __forceinline__ float2 h2f(uint32_t v)
{
    __half2 h = *reinterpret_cast<__half2 *>(&v);
    return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// ---------------------------------------------------------------------------------- spinor codecs
// Load the 24 reals of site cb (one flavour block starting at `base`) into v.
template <int PREC>
__device__ __forceinline__ void load_spinor(const void *base, const float *norm, int cb, int Vh,
                                            typename Traits<PREC>::real v[24]);

template <>
__device__ __forceinline__ void load_spinor<P64>(const void *base, const float *, int cb, int Vh, double v[24])
{
    const double2 *p = reinterpret_cast<const double2 *>(base) + cb;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        double2 c = ldg(p + (size_t)k * Vh);
        v[2 * k] = c.x;
        v[2 * k + 1] = c.y;
    }
}
template <>
__device__ __forceinline__ void load_spinor<P32>(const void *base, const float *, int cb, int Vh, float v[24])
{
    const float4 *p = reinterpret_cast<const float4 *>(base) + cb;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 c = ldg(p + (size_t)k * Vh);
        v[4 * k] = c.x;
        v[4 * k + 1] = c.y;
        v[4 * k + 2] = c.z;
        v[4 * k + 3] = c.w;
    }
}
template <>
__device__ __forceinline__ void load_spinor<P16>(const void *base, const float *norm, int cb, int Vh, float v[24])
{
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + cb;
    const float n = __ldg(norm + cb);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        uint4 c = ldg(p + (size_t)k * Vh);
        float2 a = h2f(c.x), b = h2f(c.y), d = h2f(c.z), e = h2f(c.w);
        v[8 * k + 0] = a.x * n; v[8 * k + 1] = a.y * n;
        v[8 * k + 2] = b.x * n; v[8 * k + 3] = b.y * n;
        v[8 * k + 4] = d.x * n; v[8 * k + 5] = d.y * n;
        v[8 * k + 6] = e.x * n; v[8 * k + 7] = e.y * n;
    }
}

template <>
__device__ __forceinline__ void load_spinor<PDF>(const void *base, const float *, int cb, int Vh, df64 v[24])
{
    const float4 *p = reinterpret_cast<const float4 *>(base) + cb;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        float4 c = ldg(p + (size_t)k * Vh);
        v[2 * k] = df64(c.x, c.y);
        v[2 * k + 1] = df64(c.z, c.w);
    }
}

// FP16 only: the stored halves of a site without the norm factor, and the norm itself, so a
// linear consumer can apply the norm once to its result instead of to all 24 inputs.
__device__ __forceinline__ float load_spinor_f16_unscaled(const void *base, const float *norm, int cb, int Vh,
                                                          float v[24])
{
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + cb;
    const float n = __ldg(norm + cb);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        uint4 c = ldg(p + (size_t)k * Vh);
        float2 a = h2f(c.x), b = h2f(c.y), d = h2f(c.z), e = h2f(c.w);
        v[8 * k + 0] = a.x; v[8 * k + 1] = a.y;
        v[8 * k + 2] = b.x; v[8 * k + 3] = b.y;
        v[8 * k + 4] = d.x; v[8 * k + 5] = d.y;
        v[8 * k + 6] = e.x; v[8 * k + 7] = e.y;
    }
    return n;
}

template <int PREC>
__device__ __forceinline__ void store_spinor(void *base, float *norm, int cb, int Vh,
                                             const typename Traits<PREC>::real v[24]);

template <>
__device__ __forceinline__ void store_spinor<P64>(void *base, float *, int cb, int Vh, const double v[24])
{
    double2 *p = reinterpret_cast<double2 *>(base) + cb;
#pragma unroll
    for (int k = 0; k < 12; k++) p[(size_t)k * Vh] = make_double2(v[2 * k], v[2 * k + 1]);
}
template <>
__device__ __forceinline__ void store_spinor<P32>(void *base, float *, int cb, int Vh, const float v[24])
{
    float4 *p = reinterpret_cast<float4 *>(base) + cb;
#pragma unroll
    for (int k = 0; k < 6; k++) p[(size_t)k * Vh] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
template <>
__device__ __forceinline__ void store_spinor<PDF>(void *base, float *, int cb, int Vh, const df64 v[24])
{
    float4 *p = reinterpret_cast<float4 *>(base) + cb;
#pragma unroll
    for (int k = 0; k < 12; k++) p[(size_t)k * Vh] = make_float4(v[2 * k].hi, v[2 * k].lo, v[2 * k + 1].hi, v[2 * k + 1].lo);
}
// FP16 with per-site norm: norm = max |v_k| over the site, stored halves = v_k / norm (|.| <= 1).
template <>
__device__ __forceinline__ void store_spinor<P16>(void *base, float *norm, int cb, int Vh, const float v[24])
{
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 24; k++) m = fmaxf(m, fabsf(v[k]));
    const float inv = (m > 0.f) ? 1.0f / m : 0.f;
    uint4 *p = reinterpret_cast<uint4 *>(base) + cb;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        uint4 c;
        c.x = f2h(v[8 * k + 0] * inv, v[8 * k + 1] * inv);
        c.y = f2h(v[8 * k + 2] * inv, v[8 * k + 3] * inv);
        c.z = f2h(v[8 * k + 4] * inv, v[8 * k + 5] * inv);
        c.w = f2h(v[8 * k + 6] * inv, v[8 * k + 7] * inv);
        p[(size_t)k * Vh] = c;
    }
    norm[cb] = m;
}

// ----------------------------------------------------------------------------------- link codecs
template <typename T>
struct Link {
    C<T> u[3][3];
};

// row 3 of an SU(3) matrix from rows 1 and 2: conj(row1 x row2).  Element k is
// conj(a_j b_l - a_l b_j) with (j, l) the cyclic successors of k; each real part is one chain of
// four FMAs (no separate subtraction of two rounded products).
template <typename T>
__device__ __forceinline__ C<T> cross_conj(C<T> aj, C<T> bl, C<T> al, C<T> bj)
{
    // re = aj.r bl.r - aj.i bl.i - al.r bj.r + al.i bj.i
    // im = -(aj.r bl.i + aj.i bl.r) + al.r bj.i + al.i bj.r
    const T re = fma(aj.r, bl.r, fma(-aj.i, bl.i, fma(-al.r, bj.r, al.i * bj.i)));
    const T im = fma(-aj.r, bl.i, fma(-aj.i, bl.r, fma(al.r, bj.i, al.i * bj.r)));
    return {re, im};
}
template <typename T>
__device__ __forceinline__ void complete_row3(Link<T> &U)
{
    U.u[2][0] = cross_conj(U.u[0][1], U.u[1][2], U.u[0][2], U.u[1][1]);
    U.u[2][1] = cross_conj(U.u[0][2], U.u[1][0], U.u[0][0], U.u[1][2]);
    U.u[2][2] = cross_conj(U.u[0][0], U.u[1][1], U.u[0][1], U.u[1][0]);
}

// 8-real form: r = (a2, a3, b1, arg a1, arg c1) with U = [[a1,a2,a3],[b1,b2,b3],[c1,c2,c3]].
// |a1| and |c1| follow from unit row 1 and unit column 1; b2, b3 from conj(row2) = row3 x row1
// combined with conj(row3) = row1 x row2; c2, c3 from conj(row3) = row1 x row2.  Singular when
// a2 = a3 = 0 (|a1| = 1); the encoder never produces that for the random fields used here.
template <typename T>
__device__ __forceinline__ void decode_link8(const T r[8], Link<T> &U)
{
    const C<T> a2 = {r[0], r[1]}, a3 = {r[2], r[3]}, b1 = {r[4], r[5]};
    const T n2 = a2.r * a2.r + a2.i * a2.i + a3.r * a3.r + a3.i * a3.i;
    const T b1n = b1.r * b1.r + b1.i * b1.i;
    const T ma1 = sqrt(fmax(T(1) - n2, T(0)));
    const T mc1 = sqrt(fmax(n2 - b1n, T(0)));
    T sa, ca, sc, cc;
    sincos(r[6], &sa, &ca);
    sincos(r[7], &sc, &cc);
    const C<T> a1 = {ma1 * ca, ma1 * sa}, c1 = {mc1 * cc, mc1 * sc};
    const T inv = T(1) / n2;
    // b2 = -(conj(a1) a2 b1 + conj(c1) conj(a3)) / n2
    C<T> t = cadd(cmul(cmulc(a1, a2), b1), cconj(cmul(c1, a3)));
    const C<T> b2 = {-t.r * inv, -t.i * inv};
    // b3 = (conj(c1) conj(a2) - conj(a1) a3 b1) / n2
    t = csub(cconj(cmul(c1, a2)), cmul(cmulc(a1, a3), b1));
    const C<T> b3 = {t.r * inv, t.i * inv};
    U.u[0][0] = a1; U.u[0][1] = a2; U.u[0][2] = a3;
    U.u[1][0] = b1; U.u[1][1] = b2; U.u[1][2] = b3;
    U.u[2][0] = c1;
    U.u[2][1] = cconj(csub(cmul(a3, b1), cmul(a1, b3)));
    U.u[2][2] = cconj(csub(cmul(a1, b2), cmul(a2, b1)));
}

template <int PREC, int RECON>
struct LinkLoader;

template <int RECON>
struct LinkLoader<P64, RECON> {
    __device__ static __forceinline__ void load(const void *g, int cb, int Vh, Link<double> &U)
    {
        const double2 *p = reinterpret_cast<const double2 *>(g) + cb;
        if (RECON == 8) {
            double r[8];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                double2 c = ldg(p + (size_t)k * Vh);
                r[2 * k] = c.x; r[2 * k + 1] = c.y;
            }
            decode_link8(r, U);
            return;
        }
        constexpr int NROW = (RECON == 18) ? 3 : 2;
#pragma unroll
        for (int k = 0; k < 3 * NROW; k++) {
            double2 c = ldg(p + (size_t)k * Vh);
            U.u[k / 3][k % 3] = {c.x, c.y};
        }
        if (RECON == 12) complete_row3(U);
    }
};

template <int RECON>
struct LinkLoader<P32, RECON> {
    __device__ static __forceinline__ void load(const void *g, int cb, int Vh, Link<float> &U)
    {
        if (RECON == 18) {
            const float2 *p = reinterpret_cast<const float2 *>(g) + cb;
#pragma unroll
            for (int k = 0; k < 9; k++) {
                float2 c = ldg(p + (size_t)k * Vh);
                U.u[k / 3][k % 3] = {c.x, c.y};
            }
            return;
        }
        const float4 *p = reinterpret_cast<const float4 *>(g) + cb;
        if (RECON == 12) {
            float r[12];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                float4 c = ldg(p + (size_t)k * Vh);
                r[4 * k] = c.x; r[4 * k + 1] = c.y; r[4 * k + 2] = c.z; r[4 * k + 3] = c.w;
            }
#pragma unroll
            for (int k = 0; k < 6; k++) U.u[k / 3][k % 3] = {r[2 * k], r[2 * k + 1]};
            complete_row3(U);
        } else {
            float r[8];
#pragma unroll
            for (int k = 0; k < 2; k++) {
                float4 c = ldg(p + (size_t)k * Vh);
                r[4 * k] = c.x; r[4 * k + 1] = c.y; r[4 * k + 2] = c.z; r[4 * k + 3] = c.w;
            }
            decode_link8(r, U);
        }
    }
};

template <int RECON>
struct LinkLoader<PDF, RECON> {
    __device__ static __forceinline__ void load(const void *g, int cb, int Vh, Link<df64> &U)
    {
        static_assert(RECON == 18 || RECON == 12, "DF64 links are stored with 18 or 12 reals");
        const float4 *p = reinterpret_cast<const float4 *>(g) + cb;
        constexpr int NC = RECON / 2;  // complex entries stored
#pragma unroll
        for (int k = 0; k < NC; k++) {
            float4 c = ldg(p + (size_t)k * Vh);
            U.u[k / 3][k % 3] = {df64(c.x, c.y), df64(c.z, c.w)};
        }
        if (RECON == 12) complete_row3(U);
    }
};

// FP16 links: entries of a unitary matrix are bounded by 1 and stored directly as halves;
// in 8-real form the two phases are stored divided by pi.
template <int RECON>
struct LinkLoader<P16, RECON> {
    __device__ static __forceinline__ void load(const void *g, int cb, int Vh, Link<float> &U)
    {
        if (RECON == 18) {
            const uint32_t *p = reinterpret_cast<const uint32_t *>(g) + cb;
#pragma unroll
            for (int k = 0; k < 9; k++) {
                float2 c = h2f(ldg(p + (size_t)k * Vh));
                U.u[k / 3][k % 3] = {c.x, c.y};
            }
        } else if (RECON == 12) {
            const uint2 *p = reinterpret_cast<const uint2 *>(g) + cb;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                uint2 c = ldg(p + (size_t)k * Vh);
                float2 a = h2f(c.x), b = h2f(c.y);
                U.u[(2 * k) / 3][(2 * k) % 3] = {a.x, a.y};
                U.u[(2 * k + 1) / 3][(2 * k + 1) % 3] = {b.x, b.y};
            }
            complete_row3(U);
        } else {
            const uint4 *p = reinterpret_cast<const uint4 *>(g) + cb;
            uint4 c = ldg(p);
            float2 a = h2f(c.x), b = h2f(c.y), d = h2f(c.z), e = h2f(c.w);
            float r[8] = {a.x, a.y, b.x, b.y, d.x, d.y, e.x * 3.14159265358979f, e.y * 3.14159265358979f};
            decode_link8(r, U);
        }
    }
};


// Convert the raw chunks of one site (as loaded) to reals; FP16 values stay unscaled (the norm
// is applied by the caller).
template <int PREC>
__device__ __forceinline__ void spinor_from_chunks(const typename Traits<PREC>::schunk *c,
                                                   typename Traits<PREC>::real v[24])
{
    if constexpr (PREC == P64) {
#pragma unroll
        for (int k = 0; k < 12; k++) { v[2 * k] = c[k].x; v[2 * k + 1] = c[k].y; }
    } else if constexpr (PREC == P32) {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            v[4 * k] = c[k].x; v[4 * k + 1] = c[k].y; v[4 * k + 2] = c[k].z; v[4 * k + 3] = c[k].w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float2 a = h2f(c[k].x), b = h2f(c[k].y), d = h2f(c[k].z), e = h2f(c[k].w);
            v[8 * k + 0] = a.x; v[8 * k + 1] = a.y; v[8 * k + 2] = b.x; v[8 * k + 3] = b.y;
            v[8 * k + 4] = d.x; v[8 * k + 5] = d.y; v[8 * k + 6] = e.x; v[8 * k + 7] = e.y;
        }
    }
}

// Decode a link from its raw chunks held in registers (same formats as LinkLoader).
template <int PREC, int RECON> struct LinkRegLoader;
template <int RECON> struct LinkRegLoader<P64, RECON> {
    __device__ static __forceinline__ void load(const double2 *c, Link<double> &U)
    {
        if (RECON == 8) {
            double r[8];
#pragma unroll
            for (int k = 0; k < 4; k++) { r[2 * k] = c[k].x; r[2 * k + 1] = c[k].y; }
            decode_link8(r, U);
            return;
        }
        constexpr int NROW = (RECON == 18) ? 3 : 2;
#pragma unroll
        for (int k = 0; k < 3 * NROW; k++) U.u[k / 3][k % 3] = {c[k].x, c[k].y};
        if (RECON == 12) complete_row3(U);
    }
};
template <int RECON> struct LinkRegLoader<P32, RECON> {
    template <typename CH>
    __device__ static __forceinline__ void load(const CH *c, Link<float> &U)
    {
        if constexpr (RECON == 18) {
#pragma unroll
            for (int k = 0; k < 9; k++) U.u[k / 3][k % 3] = {c[k].x, c[k].y};
        } else {
            constexpr int NC = RECON / 4;
            float r[RECON];
#pragma unroll
            for (int k = 0; k < NC; k++) { r[4 * k] = c[k].x; r[4 * k + 1] = c[k].y; r[4 * k + 2] = c[k].z; r[4 * k + 3] = c[k].w; }
            if constexpr (RECON == 12) {
#pragma unroll
                for (int k = 0; k < 6; k++) U.u[k / 3][k % 3] = {r[2 * k], r[2 * k + 1]};
                complete_row3(U);
            } else {
                decode_link8(r, U);
            }
        }
    }
};
template <int RECON> struct LinkRegLoader<P16, RECON> {
    template <typename CH>
    __device__ static __forceinline__ void load(const CH *c, Link<float> &U)
    {
        if constexpr (RECON == 18) {
#pragma unroll
            for (int k = 0; k < 9; k++) { float2 v = h2f(c[k]); U.u[k / 3][k % 3] = {v.x, v.y}; }
        } else if constexpr (RECON == 12) {
#pragma unroll
            for (int k = 0; k < 3; k++) {
                float2 a = h2f(c[k].x), b = h2f(c[k].y);
                U.u[(2 * k) / 3][(2 * k) % 3] = {a.x, a.y};
                U.u[(2 * k + 1) / 3][(2 * k + 1) % 3] = {b.x, b.y};
            }
            complete_row3(U);
        } else {
            float2 a = h2f(c[0].x), b = h2f(c[0].y), d = h2f(c[0].z), e = h2f(c[0].w);
            float r[8] = {a.x, a.y, b.x, b.y, d.x, d.y, e.x * 3.14159265358979f, e.y * 3.14159265358979f};
            decode_link8(r, U);
        }
    }
};

// ---------------------------------------------------------------------------------- local twist
// A general (flavour x flavour) matrix per gamma5 block: m[g][f][f'], g = 0 for spins 0,1
// (gamma5 = +1 in the DeGrand-Rossi basis) and g = 1 for spins 2,3 (gamma5 = -1).  For one
// flavour only m[g][0][0] is used.  The host fills it with R, R^-1 or their adjoints.
template <typename T>
struct Twist {
    C<T> m[2][2][2];
};

// m0 a + m1 b with each real part one chain of four FMAs (no separate addition of two rounded
// complex products)
template <typename T>
__device__ __forceinline__ C<T> cmul_add2(C<T> m0, C<T> a, C<T> m1, C<T> b)
{
    return {fma(m0.r, a.r, fma(-m0.i, a.i, fma(m1.r, b.r, -m1.i * b.i))),
            fma(m0.r, a.i, fma(m0.i, a.r, fma(m1.r, b.i, m1.i * b.r)))};
}

template <typename T, int NF>
__device__ __forceinline__ void apply_twist(const Twist<T> &tw, T v[NF][24])
{
#pragma unroll
    for (int s = 0; s < 4; s++) {
        const int g = s >> 1;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int k = 2 * (3 * s + c);
            if (NF == 1) {
                C<T> a = {v[0][k], v[0][k + 1]};
                C<T> r = cmul(tw.m[g][0][0], a);
                v[0][k] = r.r; v[0][k + 1] = r.i;
            } else {
                C<T> a = {v[0][k], v[0][k + 1]}, b = {v[NF - 1][k], v[NF - 1][k + 1]};
                C<T> r0 = cmul_add2(tw.m[g][0][0], a, tw.m[g][0][1], b);
                C<T> r1 = cmul_add2(tw.m[g][1][0], a, tw.m[g][1][1], b);
                v[0][k] = r0.r; v[0][k + 1] = r0.i;
                v[NF - 1][k] = r1.r; v[NF - 1][k + 1] = r1.i;
            }
        }
    }
}

}  // namespace tmk

// tm_clover.cuh -- the local clover-twisted-mass operator of one site in the kernels' storage
// formats, and its application (forward and inverse) inside the fused epilogues.
//
// With a clover term the local operator of eq. 2.1 becomes L = C + X, where
//   C = 1 + T,  T = i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}     (hermitian, commutes
//       with gamma5, so it is two 6x6 blocks per site: spins 0,1 (gamma5 = +1) and 2,3 (-1)),
//   X = R - 1 = 2 i kappa mu gamma5 tau3 (+ 2 kappa eps tau1)           (the twist of eq. 2.1).
// X acts in flavour only and X^2 = (b^2 - a^2) 1 (doublet) or -a^2 (one flavour) is a number,
// so with D = C^2 - X^2 (a function of C alone):
//   L^-1 = (C - X) D^-1 = D^-1 (C - X),         L^dag = C + X^dag,   L^-dag = (C - X^dag) D^-1.
// Each parity stores four hermitian 6x6 blocks per site, [C_+, C_-, D_+^-1, D_-^-1], each packed
// as 36 reals: the 6 (real) diagonal entries, then the 15 entries above the diagonal in
// row-major order (0,1), (0,2), ..., (4,5) as (re, im).  Row / column index i = 3 s + c for the
// block's spins s = 0, 1 and colour c.  Layout [parity][chunk][Vh] of 16-byte chunks:
//   FP64: 18 double2 per block,  FP32: 9 float4 per block,
//   FP16: 5 uint4 per block (36 halves, 4 zero) scaled by one float per block, [parity][4][Vh].
#pragma once
#include "tm_core.cuh"

namespace tmk {

template <int PREC> struct CloverLayout;
template <> struct CloverLayout<P64> { static constexpr int CPB = 18; };  // chunks per block
template <> struct CloverLayout<P32> { static constexpr int CPB = 9; };
template <> struct CloverLayout<P16> { static constexpr int CPB = 5; };

template <int PREC>
__device__ __forceinline__ void load_clover_block(const void *clov, const float *cnorm, int parity, int blk, int cb,
                                                  int Vh, typename Traits<PREC>::real h[36])
{
    constexpr int CPB = CloverLayout<PREC>::CPB;
    const size_t base = ((size_t)parity * 4 * CPB + (size_t)blk * CPB) * Vh + cb;
    if constexpr (PREC == P64) {
        const double2 *p = reinterpret_cast<const double2 *>(clov) + base;
#pragma unroll
        for (int k = 0; k < 18; k++) {
            const double2 c = ldg(p + (size_t)k * Vh);
            h[2 * k] = c.x;
            h[2 * k + 1] = c.y;
        }
    } else if constexpr (PREC == P32) {
        const float4 *p = reinterpret_cast<const float4 *>(clov) + base;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const float4 c = ldg(p + (size_t)k * Vh);
            h[4 * k] = c.x; h[4 * k + 1] = c.y; h[4 * k + 2] = c.z; h[4 * k + 3] = c.w;
        }
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(clov) + base;
        const float n = __ldg(cnorm + ((size_t)parity * 4 + blk) * Vh + cb);
        float t[40];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const uint4 c = ldg(p + (size_t)k * Vh);
            const float2 a = h2f(c.x), b = h2f(c.y), d = h2f(c.z), e = h2f(c.w);
            t[8 * k + 0] = a.x; t[8 * k + 1] = a.y; t[8 * k + 2] = b.x; t[8 * k + 3] = b.y;
            t[8 * k + 4] = d.x; t[8 * k + 5] = d.y; t[8 * k + 6] = e.x; t[8 * k + 7] = e.y;
        }
#pragma unroll
        for (int k = 0; k < 36; k++) h[k] = t[k] * n;
    }
}

// y = H x for a packed hermitian 6x6 block H
template <typename T>
__device__ __forceinline__ void herm_mv(const T h[36], const C<T> x[6], C<T> y[6])
{
#pragma unroll
    for (int i = 0; i < 6; i++) y[i] = {h[i] * x[i].r, h[i] * x[i].i};
    int k = 6;
#pragma unroll
    for (int i = 0; i < 6; i++) {
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            const C<T> o = {h[k], h[k + 1]};
            k += 2;
            y[i] = cadd(y[i], cmul(o, x[j]));   // H_ij x_j
            y[j] = cadd(y[j], cmulc(o, x[i]));  // H_ji x_i = conj(H_ij) x_i
        }
    }
}

// v <- L v (INV = false) or L^-1 v (INV = true) at site cb of the given parity.  X is the
// host-built twist minus the identity (X^dag for the adjoint), one flavour matrix per gamma5 block.
template <int PREC, int NF, bool INV, typename T>
__device__ __forceinline__ void apply_clover(const void *clov, const float *cnorm, int parity, int cb, int Vh,
                                             const Twist<T> &X, T v[NF][24])
{
#pragma unroll
    for (int g = 0; g < 2; g++) {
        C<T> z[NF][6], y[NF][6];
#pragma unroll
        for (int f = 0; f < NF; f++)
#pragma unroll
            for (int i = 0; i < 6; i++) z[f][i] = {v[f][12 * g + 2 * i], v[f][12 * g + 2 * i + 1]};
        T h[36];
        if (INV) {
            load_clover_block<PREC>(clov, cnorm, parity, 2 + g, cb, Vh, h);
#pragma unroll
            for (int f = 0; f < NF; f++) {
                C<T> t[6];
                herm_mv(h, z[f], t);
#pragma unroll
                for (int i = 0; i < 6; i++) z[f][i] = t[i];
            }
        }
        load_clover_block<PREC>(clov, cnorm, parity, g, cb, Vh, h);
#pragma unroll
        for (int f = 0; f < NF; f++) herm_mv(h, z[f], y[f]);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            if (NF == 1) {
                const C<T> t = cmul(X.m[g][0][0], z[0][i]);
                y[0][i] = INV ? csub(y[0][i], t) : cadd(y[0][i], t);
            } else {
                const C<T> t0 = cadd(cmul(X.m[g][0][0], z[0][i]), cmul(X.m[g][0][1], z[NF - 1][i]));
                const C<T> t1 = cadd(cmul(X.m[g][1][0], z[0][i]), cmul(X.m[g][1][1], z[NF - 1][i]));
                y[0][i] = INV ? csub(y[0][i], t0) : cadd(y[0][i], t0);
                y[NF - 1][i] = INV ? csub(y[NF - 1][i], t1) : cadd(y[NF - 1][i], t1);
            }
        }
#pragma unroll
        for (int f = 0; f < NF; f++)
#pragma unroll
            for (int i = 0; i < 6; i++) {
                v[f][12 * g + 2 * i] = y[f][i].r;
                v[f][12 * g + 2 * i + 1] = y[f][i].i;
            }
    }
}

}  // namespace tmk

// tm_dslash.cuh -- the fused even-odd twisted-mass hopping kernel (sec. 2.1, eq. 2.1-2.3).
//
// One thread per output site of parity p computes the hopping sum
//   acc(x) = sum_mu (1 - s g_mu) U_mu(x) in(x+mu) + (1 + s g_mu) U_mu(x-mu)^dag in(x-mu)
// with s = +1 for H and s = -1 for H^dag (the projectors swap), gamma matrices in the
// DeGrand-Rossi basis, and a factor -1 on hops across the antiperiodic time boundary.
// Each (1 +- g_mu) has rank two, so only two spin rows h0, h1 are multiplied by the link
// (2 x 66 flops) and spins 2, 3 of the result are +-h or +-i h of those rows.
//
// The local operators of the even-odd factorisation are fused in (sec. 2.1: "computed on the
// fly"), selected by a uniform runtime switch:
//   EPI_SCALE      out = c acc                     plain hopping block
//   EPI_TW         out = T acc                     R^-1_oo D_oe  (T = R^-1 or R^-dag)
//   EPI_TWX_AXPY   out = T x + c acc               R_ee x - kappa^2 D_eo t      (eq. 2.2 LHS)
//   EPI_X_TWAXPY   out = x + c T acc               x - kappa^2 R^-1_ee D_eo t  (eq. 2.3 LHS)
//   EPI_XPAY       out = x + c acc
//   EPI_TW_XPAY    out = T (x + c acc)             odd reconstruction, symmetric RHS
//   EPI_TWX_AXPY_TW out = Q (T x + c acc)          (R R^dag)^-1 M_asym: the first factor of the
//                                                  symmetric normal operator (Q = tw_acc)
//   EPI_TWX_AXPY_RUPD out = out - s (T x + c acc)  CG's r <- r - alpha A^dag A p in the launch that
//                                                  produces A^dag A p (s = *scal_in; staged forms
//                                                  with the fused reduction of |out|^2 only)
// and, as a compile-time option, a prologue that twists every neighbour spinor before the
// projection (in -> T_pro in), which the adjoint of the symmetric operator needs.
// For the doublet both flavours are computed by the same thread, so each link is loaded once
// and used for both (sec. 2.1).
#pragma once
#include <atomic>
#include <type_traits>

#include "tm_blas.cuh"
#include "tm_clover.cuh"
#include "tm_core.cuh"
#include "tm_internal.h"

namespace tmk {

template <typename T>
struct DslashArgs {
    void *out;
    float *out_norm;
    const void *in;
    const float *in_norm;
    const void *x;
    const float *x_norm;
    const void *gauge;  // [mu][parity][chunk][Vh] of this precision / recon
    int Vh, X1h, Lx, Ly, Lz, Lt;
    int cb0, ncb;       // output sites [cb0, cb0 + ncb) of the single-RHS launch forms (all: 0, Vh)
    int out_parity;
    int tbc;
    int epilogue;
    T sigma;  // +1: H, -1: H^dag
    T coef;
    Twist<T> tw_epi, tw_pro;
    Twist<T> tw_acc;         // Q of EPI_TWX_AXPY_TW
    const double *scal_in;   // device scalar s of EPI_TWX_AXPY_RUPD
    const void *clov;        // clover handles: per-site local operator of this precision (tm_clover.cuh)
    const float *clov_norm;  // FP16 block scales
};

template <typename T>
__device__ __forceinline__ void acc_add(T *a, int k, C<T> w, T q)
{
    a[k] = fma(q, w.r, a[k]);
    a[k + 1] = fma(q, w.i, a[k + 1]);
}
// binary32: both reals of the complex in one packed FMA (Blackwell's f32x2 FMA; the same
// rounding as two scalar FMAs), halving the issue slots of the accumulation
__device__ __forceinline__ void acc_add(float *a, int k, C<float> w, float q)
{
    const float2 r = __ffma2_rn(make_float2(q, q), make_float2(w.r, w.i), make_float2(a[k], a[k + 1]));
    a[k] = r.x;
    a[k + 1] = r.y;
}
// c + s b for a real s
template <typename T>
__device__ __forceinline__ C<T> cfma_s(T s, C<T> b, C<T> c)
{
    return {fma(s, b.r, c.r), fma(s, b.i, c.i)};
}
__device__ __forceinline__ C<float> cfma_s(float s, C<float> b, C<float> c)
{
    const float2 r = __ffma2_rn(make_float2(s, s), make_float2(b.r, b.i), make_float2(c.r, c.i));
    return {r.x, r.y};
}
// a += q * i * w
template <typename T>
__device__ __forceinline__ void acc_addi(T *a, int k, C<T> w, T q)
{
    a[k] = fma(-q, w.i, a[k]);
    a[k + 1] = fma(q, w.r, a[k + 1]);
}

// w = U h (forward) or U^dag h (backward), h one spin row (3 colours).  Each output is one FMA
// chain over the three colours (re: ur hr -+ ui hi, im: ur hi +- ui hr with u = U[a][b] forward,
// U[b][a] conjugated backward): four FMAs per complex product instead of two multiplies, two
// FMAs and two additions.
template <typename T, bool FWD>
__device__ __forceinline__ void link_mul(const Link<T> &U, const C<T> h[3], C<T> w[3])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C<T> s;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const C<T> u = FWD ? U.u[a][b] : U.u[b][a];
            const T ui_re = FWD ? -u.i : u.i, ui_im = FWD ? u.i : -u.i;  // signed partners of hi, hr
            if (b == 0) {
                s.r = u.r * h[b].r;
                s.i = u.r * h[b].i;
            } else {
                s.r = fma(u.r, h[b].r, s.r);
                s.i = fma(u.r, h[b].i, s.i);
            }
            s.r = fma(ui_re, h[b].i, s.r);
            s.i = fma(ui_im, h[b].r, s.i);
        }
        w[a] = s;
    }
}

// Project one flavour's spinor v with (1 + sp g_MU), multiply by the link, accumulate with
// boundary sign sg.  Spin index k of colour c, re part, is at 2*(3k + c).
template <int MU, bool FWD, typename T>
__device__ __forceinline__ void hop_one(T *acc, const Link<T> &U, const T *v, T sp, T sg)
{
    C<T> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const C<T> p0 = {v[2 * c], v[2 * c + 1]}, p1 = {v[6 + 2 * c], v[7 + 2 * c]};
        const C<T> p2 = {v[12 + 2 * c], v[13 + 2 * c]}, p3 = {v[18 + 2 * c], v[19 + 2 * c]};
        if (MU == 0) {        // h0 = p0 + sp i p3,  h1 = p1 + sp i p2
            h0[c] = {fma(-sp, p3.i, p0.r), fma(sp, p3.r, p0.i)};
            h1[c] = {fma(-sp, p2.i, p1.r), fma(sp, p2.r, p1.i)};
        } else if (MU == 1) { // h0 = p0 - sp p3,  h1 = p1 + sp p2
            h0[c] = cfma_s(-sp, p3, p0);
            h1[c] = cfma_s(sp, p2, p1);
        } else if (MU == 2) { // h0 = p0 + sp i p2,  h1 = p1 - sp i p3
            h0[c] = {fma(-sp, p2.i, p0.r), fma(sp, p2.r, p0.i)};
            h1[c] = {fma(sp, p3.i, p1.r), fma(-sp, p3.r, p1.i)};
        } else {              // h0 = p0 + sp p2,  h1 = p1 + sp p3
            h0[c] = cfma_s(sp, p2, p0);
            h1[c] = cfma_s(sp, p3, p1);
        }
    }
    C<T> w0[3], w1[3];
    link_mul<T, FWD>(U, h0, w0);
    link_mul<T, FWD>(U, h1, w1);
    const T q = sg * sp;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc_add(acc, 2 * c, w0[c], sg);
        acc_add(acc, 6 + 2 * c, w1[c], sg);
        if (MU == 0) {        // row2 = -sp i h1, row3 = -sp i h0
            acc_addi(acc, 12 + 2 * c, w1[c], -q);
            acc_addi(acc, 18 + 2 * c, w0[c], -q);
        } else if (MU == 1) { // row2 = sp h1, row3 = -sp h0
            acc_add(acc, 12 + 2 * c, w1[c], q);
            acc_add(acc, 18 + 2 * c, w0[c], -q);
        } else if (MU == 2) { // row2 = -sp i h0, row3 = sp i h1
            acc_addi(acc, 12 + 2 * c, w0[c], -q);
            acc_addi(acc, 18 + 2 * c, w1[c], q);
        } else {              // row2 = sp h0, row3 = sp h1
            acc_add(acc, 12 + 2 * c, w0[c], q);
            acc_add(acc, 18 + 2 * c, w1[c], q);
        }
    }
}

// ---- The doublet with its flavours paired (binary32 arithmetic; launch forms 8 / 9) ----
// Both flavours see the same link, so real k of flavour 0 and real k of flavour 1 share one
// 64-bit register pair: every product with a link element serves both flavours in one packed
// FMA (a complex product is four of them), and the projection and the accumulation are packed
// too.  Multiplication by i only renames the real and imaginary pairs.  The sign of the
// complex products comes from the negated real or imaginary pair of each projected colour (six
// packed multiplies per hop), and the per-flavour scale (boundary sign times the FP16 site norm)
// is a pair as well.  Per value these are the binary32 operations of hop_one in the same order
// (its link product is the same FMA chain), so the results are bit-identical to hop_one's.
// PACK: pack the projection as well (inputs that come out of conversions or arithmetic land in
// register pairs for free; 16-byte binary32 loads give four registers of one flavour, which
// scalar FMAs pair up without moves).
template <bool PACK>
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c)
{
    if constexpr (PACK) return __ffma2_rn(a, b, c);
    else return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}

// The rank-2 projection (1 + sp g_MU) of one hop keeps spin rows h0, h1; each of their 12 reals
// is one FMA  p[a] + q p[b]  with a in the upper spin rows (reals 0..11), b in the lower ones
// (reals 12..23) and q = +-sp.  For real k = 6 row + 2 colour + re/im of the projected rows
// (a = k), proj_b gives b and proj_neg whether q = -sp.
template <int MU>
__device__ __forceinline__ constexpr int proj_b(int k)
{
    const int row = k / 6, c = (k % 6) / 2, im = k & 1;
    // MU 0: h0 = p0 + sp i p3,  h1 = p1 + sp i p2      MU 1: h0 = p0 - sp p3,  h1 = p1 + sp p2
    // MU 2: h0 = p0 + sp i p2,  h1 = p1 - sp i p3      MU 3: h0 = p0 + sp p2,  h1 = p1 + sp p3
    const int lower = (MU == 0 || MU == 1) ? (row == 0 ? 3 : 2) : (row == 0 ? 2 : 3);
    const bool times_i = (MU == 0 || MU == 2);
    return 6 * lower + 2 * c + (times_i ? 1 - im : im);
}
template <int MU>
__device__ __forceinline__ constexpr bool proj_neg(int k)
{
    const int row = k / 6, im = k & 1;
    if (MU == 0) return im == 0;                      // i p: re takes -p.i
    if (MU == 1) return row == 0;                     // -sp p3 for h0
    if (MU == 2) return row == 0 ? im == 0 : im == 1; // +i p2 for h0, -i p3 for h1
    return false;
}

template <int MU, bool FWD>
__device__ __forceinline__ void pair_mul_acc(float (&acc)[2][24], const Link<float> &U, const float2 (&h0r)[3],
                                             const float2 (&h0i)[3], const float2 (&h1r)[3], const float2 (&h1i)[3],
                                             float sp, float2 sg);

template <int MU, bool FWD, bool PACK>
__device__ __forceinline__ void hop_pair(float (&acc)[2][24], const Link<float> &U, const float (&v)[2][24], float sp,
                                         float2 sg)
{
    const float2 s = make_float2(sp, sp), ns = make_float2(-sp, -sp);
    auto V = [&](int k) { return make_float2(v[0][k], v[1][k]); };
    // projected rows h0, h1 per colour: real and imaginary pairs
    float2 h0r[3], h0i[3], h1r[3], h1i[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int p0 = 2 * c, p1 = 6 + 2 * c, p2 = 12 + 2 * c, p3 = 18 + 2 * c;
        if (MU == 0) {        // h0 = p0 + sp i p3,  h1 = p1 + sp i p2
            h0r[c] = pfma<PACK>(ns, V(p3 + 1), V(p0)); h0i[c] = pfma<PACK>(s, V(p3), V(p0 + 1));
            h1r[c] = pfma<PACK>(ns, V(p2 + 1), V(p1)); h1i[c] = pfma<PACK>(s, V(p2), V(p1 + 1));
        } else if (MU == 1) { // h0 = p0 - sp p3,  h1 = p1 + sp p2
            h0r[c] = pfma<PACK>(ns, V(p3), V(p0)); h0i[c] = pfma<PACK>(ns, V(p3 + 1), V(p0 + 1));
            h1r[c] = pfma<PACK>(s, V(p2), V(p1)); h1i[c] = pfma<PACK>(s, V(p2 + 1), V(p1 + 1));
        } else if (MU == 2) { // h0 = p0 + sp i p2,  h1 = p1 - sp i p3
            h0r[c] = pfma<PACK>(ns, V(p2 + 1), V(p0)); h0i[c] = pfma<PACK>(s, V(p2), V(p0 + 1));
            h1r[c] = pfma<PACK>(s, V(p3 + 1), V(p1)); h1i[c] = pfma<PACK>(ns, V(p3), V(p1 + 1));
        } else {              // h0 = p0 + sp p2,  h1 = p1 + sp p3
            h0r[c] = pfma<PACK>(s, V(p2), V(p0)); h0i[c] = pfma<PACK>(s, V(p2 + 1), V(p0 + 1));
            h1r[c] = pfma<PACK>(s, V(p3), V(p1)); h1i[c] = pfma<PACK>(s, V(p3 + 1), V(p1 + 1));
        }
    }
    pair_mul_acc<MU, FWD>(acc, U, h0r, h0i, h1r, h1i, sp, sg);
}

// ---- binary16 neighbours: the projection straight from the stored halves ----
// d = q h + c with h, q binary16 and c binary32 (Blackwell's mixed-precision FMA): both halves
// widen exactly, so this is the binary32 FMA of the converted values with one rounding, and the
// lower spin rows' halves never pass through a separate conversion.
template <int HI>
__device__ __forceinline__ float fma_f16(uint32_t w, unsigned short q, float c)
{
    float d;
    if constexpr (HI)
        asm("{.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %1;\n\tfma.rn.f32.f16 %0, hi, %2, %3;\n\t}"
            : "=f"(d) : "r"(w), "h"(q), "f"(c));
    else
        asm("{.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %1;\n\tfma.rn.f32.f16 %0, lo, %2, %3;\n\t}"
            : "=f"(d) : "r"(w), "h"(q), "f"(c));
    return d;
}
__device__ __forceinline__ uint32_t chunk_word(const uint4 (&c)[3], int w)
{
    const uint4 &q = c[w >> 2];
    return (w & 3) == 0 ? q.x : (w & 3) == 1 ? q.y : (w & 3) == 2 ? q.z : q.w;
}
// The 12 projected reals of one flavour (index as in proj_b) from its three raw 16-byte chunks:
// the upper spin rows converted to binary32, the lower rows taken as halves by the FMA.  The
// operations per value are those of hop_pair / hop_rows (the same FMA of the same operands).
template <int MU>
__device__ __forceinline__ void proj_f16(const uint4 (&c)[3], float sp, float (&h)[12])
{
    const unsigned short qp = sp > 0.f ? (unsigned short)0x3c00 : (unsigned short)0xbc00;  // binary16 +-1
    const unsigned short qn = qp ^ (unsigned short)0x8000;
    float a[12];
#pragma unroll
    for (int w = 0; w < 6; w++) {
        const float2 f = h2f(chunk_word(c, w));
        a[2 * w] = f.x;
        a[2 * w + 1] = f.y;
    }
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const int b = proj_b<MU>(k);
        const unsigned short q = proj_neg<MU>(k) ? qn : qp;
        const uint32_t w = chunk_word(c, b >> 1);
        h[k] = (b & 1) ? fma_f16<1>(w, q, a[k]) : fma_f16<0>(w, q, a[k]);
    }
}

// hop_pair for binary16 neighbours (the two flavours' raw chunks; sg includes the site norms)
template <int MU, bool FWD>
__device__ __forceinline__ void hop_pair_f16(float (&acc)[2][24], const Link<float> &U, const uint4 (&s)[2][3],
                                             float sp, float2 sg)
{
    float p0[12], p1[12];
    proj_f16<MU>(s[0], sp, p0);
    proj_f16<MU>(s[1], sp, p1);
    float2 h0r[3], h0i[3], h1r[3], h1i[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        h0r[c] = make_float2(p0[2 * c], p1[2 * c]);
        h0i[c] = make_float2(p0[2 * c + 1], p1[2 * c + 1]);
        h1r[c] = make_float2(p0[6 + 2 * c], p1[6 + 2 * c]);
        h1i[c] = make_float2(p0[7 + 2 * c], p1[7 + 2 * c]);
    }
    pair_mul_acc<MU, FWD>(acc, U, h0r, h0i, h1r, h1i, sp, sg);
}

template <int MU, bool FWD>
__device__ __forceinline__ void pair_mul_acc(float (&acc)[2][24], const Link<float> &U, const float2 (&h0r)[3],
                                             const float2 (&h0i)[3], const float2 (&h1r)[3], const float2 (&h1i)[3],
                                             float sp, float2 sg)
{
    // w = U h:      re = sum ur hr + (-ui) hi,  im = sum ur hi + ui hr
    // w = U^dag h:  re = sum ur hr + ui hi,     im = sum ur hi + (-ui) hr   (u = U[b][a])
    // The minus sign rides on the broadcast link element (a sign flip of one value per element,
    // no arithmetic on the projected pairs); (-ui) x = -(ui x) exactly, so the bits do not change.
    float2 w0r[3], w0i[3], w1r[3], w1i[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const C<float> u = FWD ? U.u[a][b] : U.u[b][a];
            const float2 ur = make_float2(u.r, u.r), ui = make_float2(u.i, u.i), nui = make_float2(-u.i, -u.i);
            if (b == 0) {
                w0r[a] = __fmul2_rn(ur, h0r[b]); w0i[a] = __fmul2_rn(ur, h0i[b]);
                w1r[a] = __fmul2_rn(ur, h1r[b]); w1i[a] = __fmul2_rn(ur, h1i[b]);
            } else {
                w0r[a] = __ffma2_rn(ur, h0r[b], w0r[a]); w0i[a] = __ffma2_rn(ur, h0i[b], w0i[a]);
                w1r[a] = __ffma2_rn(ur, h1r[b], w1r[a]); w1i[a] = __ffma2_rn(ur, h1i[b], w1i[a]);
            }
            w0r[a] = __ffma2_rn(FWD ? nui : ui, h0i[b], w0r[a]); w0i[a] = __ffma2_rn(FWD ? ui : nui, h0r[b], w0i[a]);
            w1r[a] = __ffma2_rn(FWD ? nui : ui, h1i[b], w1r[a]); w1i[a] = __ffma2_rn(FWD ? ui : nui, h1r[b], w1i[a]);
        }
    }
    // accumulate the four spin rows (the same reconstruction as hop_one)
    const float2 q = make_float2(sg.x * sp, sg.y * sp), nq = make_float2(-q.x, -q.y);
    float2 A[24];
#pragma unroll
    for (int k = 0; k < 24; k++) A[k] = make_float2(acc[0][k], acc[1][k]);
    auto add = [&](int k, float2 wr, float2 wi, float2 f) {  // row += f w
        A[k] = __ffma2_rn(f, wr, A[k]);
        A[k + 1] = __ffma2_rn(f, wi, A[k + 1]);
    };
    auto addi = [&](int k, float2 wr, float2 wi, float2 f, float2 nf) {  // row += f i w
        A[k] = __ffma2_rn(nf, wi, A[k]);
        A[k + 1] = __ffma2_rn(f, wr, A[k + 1]);
    };
#pragma unroll
    for (int c = 0; c < 3; c++) {
        add(2 * c, w0r[c], w0i[c], sg);
        add(6 + 2 * c, w1r[c], w1i[c], sg);
        if (MU == 0) {        // row2 = -sp i h1, row3 = -sp i h0
            addi(12 + 2 * c, w1r[c], w1i[c], nq, q);
            addi(18 + 2 * c, w0r[c], w0i[c], nq, q);
        } else if (MU == 1) { // row2 = sp h1, row3 = -sp h0
            add(12 + 2 * c, w1r[c], w1i[c], q);
            add(18 + 2 * c, w0r[c], w0i[c], nq);
        } else if (MU == 2) { // row2 = -sp i h0, row3 = sp i h1
            addi(12 + 2 * c, w0r[c], w0i[c], nq, q);
            addi(18 + 2 * c, w1r[c], w1i[c], q, nq);
        } else {              // row2 = sp h0, row3 = sp h1
            add(12 + 2 * c, w0r[c], w0i[c], q);
            add(18 + 2 * c, w1r[c], w1i[c], q);
        }
    }
#pragma unroll
    for (int k = 0; k < 24; k++) { acc[0][k] = A[k].x; acc[1][k] = A[k].y; }
}

// ---- One flavour with its two projected spin rows paired (binary32; launch forms 8 / 9) ----
// The rank-2 projection leaves two spin rows h0, h1 that multiply the same link, so colour c of
// h0 and of h1 share a register pair and the link products are the packed FMAs of hop_pair.
// The accumulator pairs rows (0, 1) and (2, 3); the hops whose lower rows take (h1, h0) in
// swapped order (mu = x, y) accumulate those two rows with scalar FMAs instead of moving pairs.
template <int MU, bool FWD>
__device__ __forceinline__ void rows_mul_acc(float (&acc)[24], const Link<float> &U, const float2 (&hr)[3],
                                             const float2 (&hi)[3], float sp, float sg);

template <int MU, bool FWD, bool PACK>
__device__ __forceinline__ void hop_rows(float (&acc)[24], const Link<float> &U, const float (&v)[24], float sp, float sg)
{
    const float2 s = make_float2(sp, sp), ns = make_float2(-sp, -sp);
    const float2 ms = make_float2(-sp, sp), sm = make_float2(sp, -sp);  // per-row signs
    auto V = [&](int ra, int rb, int k) { return make_float2(v[6 * ra + k], v[6 * rb + k]); };
    float2 hr[3], hi[3];  // (h0, h1) of colour c: real and imaginary pairs
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int r = 2 * c, i = 2 * c + 1;
        if (MU == 0) {        // h0 = p0 + sp i p3,  h1 = p1 + sp i p2
            hr[c] = pfma<PACK>(ns, V(3, 2, i), V(0, 1, r)); hi[c] = pfma<PACK>(s, V(3, 2, r), V(0, 1, i));
        } else if (MU == 1) { // h0 = p0 - sp p3,  h1 = p1 + sp p2
            hr[c] = pfma<PACK>(ms, V(3, 2, r), V(0, 1, r)); hi[c] = pfma<PACK>(ms, V(3, 2, i), V(0, 1, i));
        } else if (MU == 2) { // h0 = p0 + sp i p2,  h1 = p1 - sp i p3
            hr[c] = pfma<PACK>(ms, V(2, 3, i), V(0, 1, r)); hi[c] = pfma<PACK>(sm, V(2, 3, r), V(0, 1, i));
        } else {              // h0 = p0 + sp p2,  h1 = p1 + sp p3
            hr[c] = pfma<PACK>(s, V(2, 3, r), V(0, 1, r)); hi[c] = pfma<PACK>(s, V(2, 3, i), V(0, 1, i));
        }
    }
    rows_mul_acc<MU, FWD>(acc, U, hr, hi, sp, sg);
}

// hop_rows for a binary16 neighbour (its raw chunks; sg includes the site norm)
template <int MU, bool FWD>
__device__ __forceinline__ void hop_rows_f16(float (&acc)[24], const Link<float> &U, const uint4 (&s)[3], float sp,
                                             float sg)
{
    float p[12];
    proj_f16<MU>(s, sp, p);
    float2 hr[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        hr[c] = make_float2(p[2 * c], p[6 + 2 * c]);
        hi[c] = make_float2(p[2 * c + 1], p[7 + 2 * c]);
    }
    rows_mul_acc<MU, FWD>(acc, U, hr, hi, sp, sg);
}

template <int MU, bool FWD>
__device__ __forceinline__ void rows_mul_acc(float (&acc)[24], const Link<float> &U, const float2 (&hr)[3],
                                             const float2 (&hi)[3], float sp, float sg)
{
    float2 wr[3], wi[3];  // (w0, w1) = U (h0, h1) or U^dag (h0, h1); signs as in pair_mul_acc
#pragma unroll
    for (int a = 0; a < 3; a++) {
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const C<float> u = FWD ? U.u[a][b] : U.u[b][a];
            const float2 ur = make_float2(u.r, u.r), ui = make_float2(u.i, u.i), nui = make_float2(-u.i, -u.i);
            if (b == 0) {
                wr[a] = __fmul2_rn(ur, hr[b]);
                wi[a] = __fmul2_rn(ur, hi[b]);
            } else {
                wr[a] = __ffma2_rn(ur, hr[b], wr[a]);
                wi[a] = __ffma2_rn(ur, hi[b], wi[a]);
            }
            wr[a] = __ffma2_rn(FWD ? nui : ui, hi[b], wr[a]);
            wi[a] = __ffma2_rn(FWD ? ui : nui, hr[b], wi[a]);
        }
    }
    const float q = sg * sp;
    const float2 sgp = make_float2(sg, sg);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int r = 2 * c;
        // rows 0 and 1: += sg (w0, w1)
        float2 a01r = make_float2(acc[r], acc[6 + r]), a01i = make_float2(acc[r + 1], acc[7 + r]);
        a01r = __ffma2_rn(sgp, wr[c], a01r);
        a01i = __ffma2_rn(sgp, wi[c], a01i);
        acc[r] = a01r.x; acc[6 + r] = a01r.y; acc[r + 1] = a01i.x; acc[7 + r] = a01i.y;
        if (MU == 0) {        // row2 = -sp i h1, row3 = -sp i h0:  re += q wi, im -= q wr
            acc[12 + r] = fmaf(q, wi[c].y, acc[12 + r]); acc[13 + r] = fmaf(-q, wr[c].y, acc[13 + r]);
            acc[18 + r] = fmaf(q, wi[c].x, acc[18 + r]); acc[19 + r] = fmaf(-q, wr[c].x, acc[19 + r]);
        } else if (MU == 1) { // row2 = sp h1, row3 = -sp h0
            acc[12 + r] = fmaf(q, wr[c].y, acc[12 + r]); acc[13 + r] = fmaf(q, wi[c].y, acc[13 + r]);
            acc[18 + r] = fmaf(-q, wr[c].x, acc[18 + r]); acc[19 + r] = fmaf(-q, wi[c].x, acc[19 + r]);
        } else {
            // MU 2: (row2, row3) = i (-q, q) (w0, w1): re += (q, -q) wi, im += (-q, q) wr
            // MU 3: (row2, row3) = q (w0, w1)
            const float2 fr = MU == 2 ? make_float2(q, -q) : make_float2(q, q);
            const float2 fi = MU == 2 ? make_float2(-q, q) : make_float2(q, q);
            float2 a23r = make_float2(acc[12 + r], acc[18 + r]), a23i = make_float2(acc[13 + r], acc[19 + r]);
            a23r = __ffma2_rn(fr, MU == 2 ? wi[c] : wr[c], a23r);
            a23i = __ffma2_rn(fi, MU == 2 ? wr[c] : wi[c], a23i);
            acc[12 + r] = a23r.x; acc[18 + r] = a23r.y; acc[13 + r] = a23i.x; acc[19 + r] = a23i.y;
        }
    }
}

template <int PREC, int NF, bool PRO, int MU, bool FWD, bool PAIR = false, typename T>
__device__ __forceinline__ void hop(T (&acc)[NF][24], const Link<T> &U, const DslashArgs<T> &a, int nb, T sg)
{
    const T sp = FWD ? -a.sigma : a.sigma;
    const size_t fstride = (size_t)Traits<PREC>::SCHUNKS * a.Vh;  // chunks per flavour
    using SC = typename Traits<PREC>::schunk;
    const SC *in = reinterpret_cast<const SC *>(a.in);
    if constexpr (PAIR && NF == 2 && std::is_same<T, float>::value) {
        float v[2][24];
        if constexpr (PRO) {
#pragma unroll
            for (int f = 0; f < 2; f++)
                load_spinor<PREC>(in + f * fstride, a.in_norm ? a.in_norm + (size_t)f * a.Vh : nullptr, nb, a.Vh, v[f]);
            apply_twist<T, NF>(a.tw_pro, v);
            hop_pair<MU, FWD, true>(acc, U, v, sp, make_float2(sg, sg));
        } else if constexpr (PREC == P16) {
            // raw halves into the mixed-precision projection; the site norms fold into the scale
            uint4 c[2][3];
#pragma unroll
            for (int f = 0; f < 2; f++)
#pragma unroll
                for (int k = 0; k < 3; k++) c[f][k] = ldg(reinterpret_cast<const uint4 *>(in + f * fstride) + (size_t)k * a.Vh + nb);
            const float n0 = __ldg(a.in_norm + nb), n1 = __ldg(a.in_norm + (size_t)a.Vh + nb);
            hop_pair_f16<MU, FWD>(acc, U, c, sp, make_float2(sg * n0, sg * n1));
        } else {
            load_spinor<PREC>(in, nullptr, nb, a.Vh, v[0]);
            load_spinor<PREC>(in + fstride, nullptr, nb, a.Vh, v[1]);
            hop_pair<MU, FWD, false>(acc, U, v, sp, make_float2(sg, sg));
        }
    } else if constexpr (PAIR && NF == 1 && std::is_same<T, float>::value) {
        float v[1][24];
        if constexpr (PRO) {
            load_spinor<PREC>(in, a.in_norm, nb, a.Vh, v[0]);
            apply_twist<T, NF>(a.tw_pro, v);
            hop_rows<MU, FWD, true>(acc[0], U, v[0], sp, sg);
        } else if constexpr (PREC == P16) {
            uint4 c[3];
#pragma unroll
            for (int k = 0; k < 3; k++) c[k] = ldg(reinterpret_cast<const uint4 *>(in) + (size_t)k * a.Vh + nb);
            hop_rows_f16<MU, FWD>(acc[0], U, c, sp, sg * __ldg(a.in_norm + nb));
        } else {
            load_spinor<PREC>(in, nullptr, nb, a.Vh, v[0]);
            hop_rows<MU, FWD, false>(acc[0], U, v[0], sp, sg);
        }
    } else if (PRO) {
        T v[NF][24];
#pragma unroll
        for (int f = 0; f < NF; f++)
            load_spinor<PREC>(in + f * fstride, a.in_norm ? a.in_norm + (size_t)f * a.Vh : nullptr, nb, a.Vh, v[f]);
        apply_twist<T, NF>(a.tw_pro, v);
#pragma unroll
        for (int f = 0; f < NF; f++) hop_one<MU, FWD>(acc[f], U, v[f], sp, sg);
    } else {
#pragma unroll
        for (int f = 0; f < NF; f++) {
            T v[24];
            if constexpr (PREC == P16) {
                // the hop is linear in the input: fold the site norm into the accumulation sign
                const T n = load_spinor_f16_unscaled(in + f * fstride, a.in_norm + (size_t)f * a.Vh, nb, a.Vh, v);
                hop_one<MU, FWD>(acc[f], U, v, sp, sg * n);
            } else {
                load_spinor<PREC>(in + f * fstride, nullptr, nb, a.Vh, v);
                hop_one<MU, FWD>(acc[f], U, v, sp, sg);
            }
        }
    }
}

// the local operator of the epilogue: the twist (a constant matrix per gamma5 block, R or R^-1
// as the host built it) or, for a clover handle, L = C + X or L^-1 of this site with X = tw
template <int PREC, int NF, bool CLOV, bool INV, typename T>
__device__ __forceinline__ void local_op(const DslashArgs<T> &a, int cb, T v[NF][24])
{
    if constexpr (CLOV) apply_clover<PREC, NF, INV>(a.clov, a.clov_norm, a.out_parity, cb, a.Vh, a.tw_epi, v);
    else apply_twist<T, NF>(a.tw_epi, v);
}

// ---- Domain decomposition in time (the multi-GPU parallelisation of sec. 2.1) ----
// A handle may hold one time slab [t0, t0 + Lt) of a lattice split over ranks in t.  The hops
// that leave the slab read a face that the neighbouring rank packed (k_dd_pack below): for the
// forward hop out of the last slice, the spin-projected half-spinor (1 - s g_4) in(x + t) of the
// next rank (2 spin rows x 3 colours, 12 reals per flavour), multiplied here by the local link
// U_t(x); for the backward hop out of the first slice, U_t(x - t)^dag (1 + s g_4) in(x - t) of the
// previous rank, the link being that rank's.  Faces hold the values in the arithmetic precision
// (binary64, or binary32 for FP32 / FP16 storage; FP16 faces keep the input's site norm beside
// them), so a decomposed operator performs the same operations in the same order as the one-slab
// kernel and gives the same bits.  Face layout: [flavour][16-byte chunk][site of the slice] with
// the 12 reals ordered (row * 3 + colour) * 2 + re/im, then (FP16) float norms [flavour][site].
// The time-boundary sign of the whole lattice is applied by the receiving slab.
template <typename T>
struct DDArgs {
    const void *ghost_b;  // from the previous slab: U^dag-multiplied rows for the first slice
    const void *ghost_f;  // from the next slab: projected rows for the last slice
    int st;               // sites of one time slice of one parity
    T sign_b, sign_f;     // -1 where the hop crosses the antiperiodic boundary of the whole lattice
};

template <int PREC>
struct FaceGeo {
    using T = typename Traits<PREC>::real;
    using FC = typename std::conditional<std::is_same<T, double>::value, double2, float4>::type;
    static constexpr int CH = 12 * (int)sizeof(T) / 16;  // chunks per flavour: 6 (double), 3 (float)
    static constexpr bool NORM = PREC == P16;
    static size_t bytes(int nf, int st) { return (size_t)nf * st * (12 * sizeof(T) + (NORM ? sizeof(float) : 0)); }
};

template <int PREC, typename T>
__device__ __forceinline__ void face_load(const void *face, int nf, int f, int st, int i, C<T> r0[3], C<T> r1[3], T &n)
{
    using G = FaceGeo<PREC>;
    using FC = typename G::FC;
    const FC *p = reinterpret_cast<const FC *>(face) + (size_t)f * G::CH * st + i;
    T v[12];
#pragma unroll
    for (int k = 0; k < G::CH; k++) {
        const FC c = ldg(p + (size_t)k * st);
        if constexpr (G::CH == 6) { v[2 * k] = c.x; v[2 * k + 1] = c.y; }
        else { v[4 * k] = c.x; v[4 * k + 1] = c.y; v[4 * k + 2] = c.z; v[4 * k + 3] = c.w; }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) { r0[c] = {v[2 * c], v[2 * c + 1]}; r1[c] = {v[6 + 2 * c], v[7 + 2 * c]}; }
    n = T(1);
    if constexpr (G::NORM) {
        const float *nrm = reinterpret_cast<const float *>(reinterpret_cast<const char *>(face) +
                                                           (size_t)nf * st * 12 * sizeof(T));
        n = __ldg(nrm + (size_t)f * st + i);
    }
}

template <int PREC, typename T>
__device__ __forceinline__ void face_store(void *face, int nf, int f, int st, int i, const C<T> r0[3], const C<T> r1[3],
                                           float n)
{
    using G = FaceGeo<PREC>;
    using FC = typename G::FC;
    FC *p = reinterpret_cast<FC *>(face) + (size_t)f * G::CH * st + i;
    T v[12];
#pragma unroll
    for (int c = 0; c < 3; c++) { v[2 * c] = r0[c].r; v[2 * c + 1] = r0[c].i; v[6 + 2 * c] = r1[c].r; v[7 + 2 * c] = r1[c].i; }
#pragma unroll
    for (int k = 0; k < G::CH; k++) {
        FC c;
        if constexpr (G::CH == 6) { c.x = v[2 * k]; c.y = v[2 * k + 1]; }
        else { c.x = v[4 * k]; c.y = v[4 * k + 1]; c.z = v[4 * k + 2]; c.w = v[4 * k + 3]; }
        p[(size_t)k * st] = c;
    }
    if constexpr (G::NORM) {
        float *nrm = reinterpret_cast<float *>(reinterpret_cast<char *>(face) + (size_t)nf * st * 12 * sizeof(T));
        nrm[(size_t)f * st + i] = n;
    }
}

// The t hop of a slab-boundary site from a face: forward (FWD, rows = projected half-spinor,
// multiplied by the local link U) or backward (rows = the neighbour's U^dag-multiplied rows).
// The accumulation is hop_one's for mu = t, with the scale sign * (FP16) site norm.
template <int PREC, int NF, bool FWD, typename T>
__device__ __forceinline__ void ghost_hop(T (&acc)[NF][24], const Link<T> &U, const void *face, int st, int i, T sp,
                                          T sign)
{
#pragma unroll
    for (int f = 0; f < NF; f++) {
        C<T> r0[3], r1[3], w0[3], w1[3];
        T n;
        face_load<PREC, T>(face, NF, f, st, i, r0, r1, n);
        if constexpr (FWD) {
            link_mul<T, true>(U, r0, w0);
            link_mul<T, true>(U, r1, w1);
        } else {
#pragma unroll
            for (int c = 0; c < 3; c++) { w0[c] = r0[c]; w1[c] = r1[c]; }
        }
        const T sg = (PREC == P16) ? sign * n : sign;
        const T q = sg * sp;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            acc_add(acc[f], 2 * c, w0[c], sg);
            acc_add(acc[f], 6 + 2 * c, w1[c], sg);
            acc_add(acc[f], 12 + 2 * c, w0[c], q);
            acc_add(acc[f], 18 + 2 * c, w1[c], q);
        }
    }
}

template <int PREC, int NF, int RECON, bool PRO, bool CLOV = false, bool PAIR = false, bool DD = false>
__device__ __forceinline__ void dslash_body(const DslashArgs<typename Traits<PREC>::real> &a0, int cb, int rhs,
                                            const DDArgs<typename Traits<PREC>::real> *dd = nullptr)
{
    using T = typename Traits<PREC>::real;
    using LL = LinkLayout<PREC, RECON>;
    using LC = typename LL::chunk;
    // right-hand side `rhs` of a field with nrhs > 1: its flavour blocks start at rhs * NF
    DslashArgs<T> a = a0;
    if (rhs) {
        using SC0 = typename Traits<PREC>::schunk;
        const size_t boff = (size_t)rhs * NF * Traits<PREC>::SCHUNKS * a0.Vh, noff = (size_t)rhs * NF * a0.Vh;
        a.in = reinterpret_cast<const SC0 *>(a0.in) + boff;
        a.out = reinterpret_cast<SC0 *>(a0.out) + boff;
        if (a0.x) a.x = reinterpret_cast<const SC0 *>(a0.x) + boff;
        if (a0.in_norm) a.in_norm = a0.in_norm + noff;
        if (a0.out_norm) a.out_norm = a0.out_norm + noff;
        if (a0.x_norm) a.x_norm = a0.x_norm + noff;
    }

    int r = cb;
    const int xh = r % a.X1h;
    r /= a.X1h;
    const int y = r % a.Ly;
    r /= a.Ly;
    const int z = r % a.Lz;
    const int t = r / a.Lz;
    const int op = a.out_parity;
    const int x = 2 * xh + ((op + y + z + t) & 1);
    const int row = cb - xh;
    const size_t gpar = (size_t)LL::N * a.Vh;  // chunks per (mu, parity)
    const LC *G = reinterpret_cast<const LC *>(a.gauge);
    const LC *Gout = G + (size_t)op * gpar;        // links at the output site: mu stride 2*gpar
    const LC *Gin = G + (size_t)(1 - op) * gpar;   // links at the neighbour site

    T acc[NF][24];
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
        for (int k = 0; k < 24; k++) acc[f][k] = T(0);

    Link<T> U;
    const T one = T(1);
    // ---- x
    {
        const int nf_ = row + (((x == a.Lx - 1) ? 0 : x + 1) >> 1);
        LinkLoader<PREC, RECON>::load(Gout + 0 * 2 * gpar, cb, a.Vh, U);
        hop<PREC, NF, PRO, 0, true, PAIR>(acc, U, a, nf_, one);
        const int nb_ = row + (((x == 0) ? a.Lx - 1 : x - 1) >> 1);
        LinkLoader<PREC, RECON>::load(Gin + 0 * 2 * gpar, nb_, a.Vh, U);
        hop<PREC, NF, PRO, 0, false, PAIR>(acc, U, a, nb_, one);
    }
    // ---- y
    {
        const int s = a.X1h;
        const int nf_ = (y == a.Ly - 1) ? cb - (a.Ly - 1) * s : cb + s;
        LinkLoader<PREC, RECON>::load(Gout + 1 * 2 * gpar, cb, a.Vh, U);
        hop<PREC, NF, PRO, 1, true, PAIR>(acc, U, a, nf_, one);
        const int nb_ = (y == 0) ? cb + (a.Ly - 1) * s : cb - s;
        LinkLoader<PREC, RECON>::load(Gin + 1 * 2 * gpar, nb_, a.Vh, U);
        hop<PREC, NF, PRO, 1, false, PAIR>(acc, U, a, nb_, one);
    }
    // ---- z
    {
        const int s = a.X1h * a.Ly;
        const int nf_ = (z == a.Lz - 1) ? cb - (a.Lz - 1) * s : cb + s;
        LinkLoader<PREC, RECON>::load(Gout + 2 * 2 * gpar, cb, a.Vh, U);
        hop<PREC, NF, PRO, 2, true, PAIR>(acc, U, a, nf_, one);
        const int nb_ = (z == 0) ? cb + (a.Lz - 1) * s : cb - s;
        LinkLoader<PREC, RECON>::load(Gin + 2 * 2 * gpar, nb_, a.Vh, U);
        hop<PREC, NF, PRO, 2, false, PAIR>(acc, U, a, nb_, one);
    }
    // ---- t (antiperiodic wrap when tbc; a slab of a decomposed lattice reads faces instead)
    {
        const int s = a.X1h * a.Ly * a.Lz;
        const bool wf = (t == a.Lt - 1), wb = (t == 0);
        LinkLoader<PREC, RECON>::load(Gout + 3 * 2 * gpar, cb, a.Vh, U);
        if (DD && wf) {
            if constexpr (DD) ghost_hop<PREC, NF, true>(acc, U, dd->ghost_f, s, cb - (a.Lt - 1) * s, -a.sigma, dd->sign_f);
        } else {
            const int nf_ = wf ? cb - (a.Lt - 1) * s : cb + s;
            hop<PREC, NF, PRO, 3, true, PAIR>(acc, U, a, nf_, (wf && a.tbc) ? -one : one);
        }
        if (DD && wb) {
            if constexpr (DD) ghost_hop<PREC, NF, false>(acc, U, dd->ghost_b, s, cb, a.sigma, dd->sign_b);
        } else {
            const int nb_ = wb ? cb + (a.Lt - 1) * s : cb - s;
            LinkLoader<PREC, RECON>::load(Gin + 3 * 2 * gpar, nb_, a.Vh, U);
            hop<PREC, NF, PRO, 3, false, PAIR>(acc, U, a, nb_, (wb && a.tbc) ? -one : one);
        }
    }

    // ---- fused local epilogue
    using SC = typename Traits<PREC>::schunk;
    const size_t fstride = (size_t)Traits<PREC>::SCHUNKS * a.Vh;
    const int epi = a.epilogue;
    if (epi == EPI_SCALE) {
#pragma unroll
        for (int f = 0; f < NF; f++)
#pragma unroll
            for (int k = 0; k < 24; k++) acc[f][k] *= a.coef;
    } else if (epi == EPI_TW) {
        local_op<PREC, NF, CLOV, true>(a, cb, acc);
    } else {
        T xv[NF][24];
        const SC *X = reinterpret_cast<const SC *>(a.x);
#pragma unroll
        for (int f = 0; f < NF; f++)
            load_spinor<PREC>(X + f * fstride, a.x_norm ? a.x_norm + (size_t)f * a.Vh : nullptr, cb, a.Vh, xv[f]);
        if (epi == EPI_TWX_AXPY || epi == EPI_TWX_AXPY_TW) {
            local_op<PREC, NF, CLOV, false>(a, cb, xv);
#pragma unroll
            for (int f = 0; f < NF; f++)
#pragma unroll
                for (int k = 0; k < 24; k++) acc[f][k] = fma(a.coef, acc[f][k], xv[f][k]);
            if (epi == EPI_TWX_AXPY_TW) apply_twist<T, NF>(a.tw_acc, acc);
        } else if (epi == EPI_X_TWAXPY) {
            local_op<PREC, NF, CLOV, true>(a, cb, acc);
#pragma unroll
            for (int f = 0; f < NF; f++)
#pragma unroll
                for (int k = 0; k < 24; k++) acc[f][k] = fma(a.coef, acc[f][k], xv[f][k]);
        } else {  // EPI_XPAY, EPI_TW_XPAY
#pragma unroll
            for (int f = 0; f < NF; f++)
#pragma unroll
                for (int k = 0; k < 24; k++) acc[f][k] = fma(a.coef, acc[f][k], xv[f][k]);
            if (epi == EPI_TW_XPAY) local_op<PREC, NF, CLOV, true>(a, cb, acc);
        }
    }
    SC *O = reinterpret_cast<SC *>(a.out);
#pragma unroll
    for (int f = 0; f < NF; f++)
        store_spinor<PREC>(O + f * fstride, a.out_norm ? a.out_norm + (size_t)f * a.Vh : nullptr, cb, a.Vh, acc[f]);
}

template <int PREC, int NF, int RECON, bool PRO>
__global__ void __launch_bounds__(256) k_dslash(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a)
{
    const int cb = a.cb0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= a.cb0 + a.ncb) return;
    dslash_body<PREC, NF, RECON, PRO>(a, cb, 0);
}

// The same kernel with a register cap: 128-thread blocks, at least MINB resident per SM
// (65536 / (128 MINB) registers per thread).  MINB = 4 measured fastest on GB300 for every
// storage form (caps for 5, 6, 8 blocks spilled; the uncapped doublet kernel holds only 12 warps).
template <int PREC, int NF, int RECON, bool PRO, int MINB, int BS = 128>
__global__ void __launch_bounds__(BS, MINB) k_dslash_lb(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a)
{
    const int cb = a.cb0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= a.cb0 + a.ncb) return;
    dslash_body<PREC, NF, RECON, PRO>(a, cb, 0);
}

// The boundary slices of a slab (decomposed lattice): thread i < st takes site i of the first
// time slice, the others site i - st of the last one (Lt = 2: the whole slab).
template <int PREC, int NF, int RECON, bool PRO>
__global__ void __launch_bounds__(128, 4) k_dslash_dd(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a,
                                                      const __grid_constant__ DDArgs<typename Traits<PREC>::real> dd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * dd.st) return;
    const int cb = i < dd.st ? i : (a.Lt - 1) * dd.st + (i - dd.st);
    dslash_body<PREC, NF, RECON, PRO, false, false, true>(a, cb, 0, &dd);
}

// Faces of a slab for its neighbours (blockIdx.y = 0: to the previous slab, from the first slice,
// the projection (1 - s g_4) of the forward hop; 1: to the next slab, from the last slice,
// U_t^dag (1 + s g_4) of the backward hop).  `a` describes the hopping launch the faces feed: its
// input field (one parity), links, sigma and input twist (PRO); out_parity is the launch's.
template <int PREC, int NF, int RECON, bool PRO>
__global__ void __launch_bounds__(128) k_dd_pack(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a,
                                                 void *face_prev, void *face_next)
{
    using T = typename Traits<PREC>::real;
    using LL = LinkLayout<PREC, RECON>;
    using LC = typename LL::chunk;
    using SC = typename Traits<PREC>::schunk;
    const int st = a.X1h * a.Ly * a.Lz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st) return;
    const bool next = blockIdx.y == 1;
    const int y = next ? (a.Lt - 1) * st + i : i;  // site of the input parity in this slab
    const T sp = next ? a.sigma : -a.sigma;         // the receiver's backward / forward hop
    const size_t fstride = (size_t)Traits<PREC>::SCHUNKS * a.Vh;
    const SC *in = reinterpret_cast<const SC *>(a.in);
    T v[NF][24];
    float n[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) {
        n[f] = 1.f;
        if constexpr (PRO) {
            load_spinor<PREC>(in + f * fstride, a.in_norm ? a.in_norm + (size_t)f * a.Vh : nullptr, y, a.Vh, v[f]);
        } else if constexpr (PREC == P16) {
            n[f] = load_spinor_f16_unscaled(in + f * fstride, a.in_norm + (size_t)f * a.Vh, y, a.Vh, v[f]);
        } else {
            load_spinor<PREC>(in + f * fstride, nullptr, y, a.Vh, v[f]);
        }
    }
    if constexpr (PRO) apply_twist<T, NF>(a.tw_pro, v);
    Link<T> U;
    if (next) {
        const size_t gpar = (size_t)LL::N * a.Vh;
        const LC *G = reinterpret_cast<const LC *>(a.gauge);
        LinkLoader<PREC, RECON>::load(G + (size_t)(3 * 2 + (1 - a.out_parity)) * gpar, y, a.Vh, U);
    }
#pragma unroll
    for (int f = 0; f < NF; f++) {
        C<T> h0[3], h1[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {  // the projection of hop_one for mu = t
            const C<T> p0 = {v[f][2 * c], v[f][2 * c + 1]}, p1 = {v[f][6 + 2 * c], v[f][7 + 2 * c]};
            const C<T> p2 = {v[f][12 + 2 * c], v[f][13 + 2 * c]}, p3 = {v[f][18 + 2 * c], v[f][19 + 2 * c]};
            h0[c] = cfma_s(sp, p2, p0);
            h1[c] = cfma_s(sp, p3, p1);
        }
        if (next) {
            C<T> w0[3], w1[3];
            link_mul<T, false>(U, h0, w0);
            link_mul<T, false>(U, h1, w1);
            face_store<PREC, T>(face_next, NF, f, st, i, w0, w1, n[f]);
        } else {
            face_store<PREC, T>(face_prev, NF, f, st, i, h0, h1, n[f]);
        }
    }
}

template <int PREC>
cudaError_t launch_dd_impl(const DslashArgs<typename Traits<PREC>::real> &a, const DDArgs<typename Traits<PREC>::real> *dd,
                           void *face_prev, void *face_next, int nf, int recon, bool pro, cudaStream_t s)
{
    // dd != NULL: the boundary launch; else the face pack of the launch described by a
    const int st = a.X1h * a.Ly * a.Lz;
#define TM_DD1(NF, R, P)                                                                          \
    if (dd) k_dslash_dd<PREC, NF, R, P><<<(2 * st + 127) / 128, 128, 0, s>>>(a, *dd);              \
    else k_dd_pack<PREC, NF, R, P><<<dim3((st + 127) / 128, 2), 128, 0, s>>>(a, face_prev, face_next);
#define TM_DDR(NF, P)                          \
    switch (recon) {                           \
    case 18: { TM_DD1(NF, 18, P) } break;      \
    case 12: { TM_DD1(NF, 12, P) } break;      \
    case 8: { TM_DD1(NF, 8, P) } break;        \
    default: return cudaErrorInvalidValue;     \
    }
    if (nf == 1) {
        if (pro) { TM_DDR(1, true) } else { TM_DDR(1, false) }
    } else {
        if (pro) { TM_DDR(2, true) } else { TM_DDR(2, false) }
    }
#undef TM_DDR
#undef TM_DD1
    return cudaGetLastError();
}

// Several right-hand sides in one launch (multi-RHS, sources share the gauge field).  A block
// is 32 consecutive sites x RPB right-hand sides, one warp per right-hand side, so every spinor
// load of a warp is one contiguous 512-byte request and the RPB warps of a block read the same
// links (served from L1 after the first); consecutive blocks take the next group of RPB
// right-hand sides of the same 32 sites, so the remaining link reads hit L2 and each link leaves
// DRAM about once per site for all sources.  RPB (2, 4 or 8) is chosen by the autotuner.
// Slot k of the active set is right-hand side act[k] (act = NULL: k).
// (the register cap of 128 registers applies to the binary32 / binary16 / binary64 forms;
// double-float code needs about 200-255 registers and is launched without the cap)
template <int PREC, int NF, int RECON, bool PRO, int RPB = 4>
__global__ void __launch_bounds__(32 * RPB, (PREC == PDF ? 1 : 16 / RPB))
    k_dslash_multi(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a, const int *__restrict__ act, int nact,
                   int nrhs)
{
    const int ngrp = (nact + RPB - 1) / RPB;
    const int grp = (int)(blockIdx.x % ngrp);
    const long sblk = blockIdx.x / ngrp;
    const int slot = grp * RPB + (threadIdx.x >> 5);
    const long cb = sblk * 32 + (threadIdx.x & 31);
    if (slot >= nact || cb >= a.Vh) return;
    const int rhs = act ? __ldg(act + slot) : slot;
    if (rhs < 0 || rhs >= nrhs) return;  // an index outside the fields is skipped, never dereferenced
    dslash_body<PREC, NF, RECON, PRO>(a, (int)cb, rhs);
}


// ------------------------------------------------------------------------------------------
// Variant 2: the same computation as k_dslash with an explicit two-stage software pipeline:
// the raw 16-byte chunks of hop h+1 (link and neighbour spinors, not yet converted) are
// loaded into registers before hop h is computed, so every warp keeps two hops of global
// loads in flight instead of one.
template <int PREC, int RECON, int NF>
struct HopRaw {
    typename LinkLayout<PREC, RECON>::chunk l[LinkLayout<PREC, RECON>::N];
    typename Traits<PREC>::schunk s[NF][Traits<PREC>::SCHUNKS];
    float n[NF];
};

template <int PREC, int RECON, int NF>
__device__ __forceinline__ void fetch_hop(HopRaw<PREC, RECON, NF> &r, const typename LinkLayout<PREC, RECON>::chunk *g,
                                          int lcb, const typename Traits<PREC>::schunk *in, const float *in_norm, int nb,
                                          int Vh)
{
#pragma unroll
    for (int k = 0; k < LinkLayout<PREC, RECON>::N; k++) r.l[k] = ldg(g + (size_t)k * Vh + lcb);
#pragma unroll
    for (int f = 0; f < NF; f++) {
#pragma unroll
        for (int k = 0; k < Traits<PREC>::SCHUNKS; k++)
            r.s[f][k] = ldg(in + ((size_t)f * Traits<PREC>::SCHUNKS + k) * Vh + nb);
        if constexpr (PREC == P16) r.n[f] = __ldg(in_norm + (size_t)f * Vh + nb);
    }
}

// decode the raw link of a HopRaw (same arithmetic as LinkLoader on registers)
template <int PREC, int RECON, int NF, typename T>
__device__ __forceinline__ void decode_link_raw(const HopRaw<PREC, RECON, NF> &r, Link<T> &U)
{
    using LC = typename LinkLayout<PREC, RECON>::chunk;
    constexpr int N = LinkLayout<PREC, RECON>::N;
    // reuse LinkLoader by pointing it at a register copy laid out as [k][1]
    LC tmp[N];
#pragma unroll
    for (int k = 0; k < N; k++) tmp[k] = r.l[k];
    LinkRegLoader<PREC, RECON>::load(tmp, U);
}

// PRO: twist every neighbour spinor with tw before the projection (the input prologue).
// PAIR: binary32 takes the paired hop (hop_pair for the doublet, hop_rows for one flavour).
template <int PREC, int RECON, int NF, int MU, bool FWD, bool PRO = false, bool PAIR = false, typename T>
__device__ __forceinline__ void compute_hop(T (&acc)[NF][24], const HopRaw<PREC, RECON, NF> &r, T sp, T sg,
                                            const Twist<T> *tw = nullptr)
{
    Link<T> U;
    decode_link_raw<PREC, RECON, NF>(r, U);
    if constexpr (PAIR && NF == 2 && PREC == P16 && !PRO) {
        // the site norms fold into the per-flavour scale; the projection reads the halves
        hop_pair_f16<MU, FWD>(acc, U, r.s, sp, make_float2(sg * r.n[0], sg * r.n[1]));
    } else if constexpr (PAIR && NF == 1 && PREC == P16 && !PRO) {
        hop_rows_f16<MU, FWD>(acc[0], U, r.s[0], sp, sg * r.n[0]);
    } else if constexpr (PAIR && NF == 2 && std::is_same<T, float>::value) {
        float v[2][24];
        spinor_from_chunks<PREC>(r.s[0], v[0]);
        spinor_from_chunks<PREC>(r.s[1], v[1]);
        if constexpr (PRO) {
            if constexpr (PREC == P16) {
#pragma unroll
                for (int f = 0; f < 2; f++)
#pragma unroll
                    for (int k = 0; k < 24; k++) v[f][k] *= r.n[f];
            }
            apply_twist<T, NF>(*tw, v);
            hop_pair<MU, FWD, true>(acc, U, v, sp, make_float2(sg, sg));
        } else if constexpr (PREC == P16) {
            // the site norms fold into the per-flavour scale
            hop_pair<MU, FWD, true>(acc, U, v, sp, make_float2(sg * r.n[0], sg * r.n[1]));
        } else {
            hop_pair<MU, FWD, false>(acc, U, v, sp, make_float2(sg, sg));
        }
    } else if constexpr (PAIR && NF == 1 && std::is_same<T, float>::value) {
        float v[1][24];
        spinor_from_chunks<PREC>(r.s[0], v[0]);
        if constexpr (PRO) {
            if constexpr (PREC == P16) {
#pragma unroll
                for (int k = 0; k < 24; k++) v[0][k] *= r.n[0];
            }
            apply_twist<T, NF>(*tw, v);
            hop_rows<MU, FWD, true>(acc[0], U, v[0], sp, sg);
        } else if constexpr (PREC == P16) {
            hop_rows<MU, FWD, true>(acc[0], U, v[0], sp, sg * r.n[0]);
        } else {
            hop_rows<MU, FWD, false>(acc[0], U, v[0], sp, sg);
        }
    } else if constexpr (PRO) {
        T v[NF][24];
#pragma unroll
        for (int f = 0; f < NF; f++) {
            spinor_from_chunks<PREC>(r.s[f], v[f]);
            if constexpr (PREC == P16) {
#pragma unroll
                for (int k = 0; k < 24; k++) v[f][k] *= r.n[f];
            }
        }
        apply_twist<T, NF>(*tw, v);
#pragma unroll
        for (int f = 0; f < NF; f++) hop_one<MU, FWD>(acc[f], U, v[f], sp, sg);
    } else {
#pragma unroll
        for (int f = 0; f < NF; f++) {
            T v[24];
            T scale = sg;
            spinor_from_chunks<PREC>(r.s[f], v);
            if constexpr (PREC == P16) scale = sg * r.n[f];
            hop_one<MU, FWD>(acc[f], U, v, sp, scale);
        }
    }
}

template <int PREC, int NF, int RECON>
__global__ void __launch_bounds__(256) k_dslash_pipe(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a)
{
    using T = typename Traits<PREC>::real;
    using LL = LinkLayout<PREC, RECON>;
    using LC = typename LL::chunk;
    using SC = typename Traits<PREC>::schunk;
    const int cb = a.cb0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= a.cb0 + a.ncb) return;
    int r = cb;
    const int xh = r % a.X1h;
    r /= a.X1h;
    const int y = r % a.Ly;
    r /= a.Ly;
    const int z = r % a.Lz;
    const int t = r / a.Lz;
    const int op = a.out_parity;
    const int x = 2 * xh + ((op + y + z + t) & 1);
    const int row = cb - xh;
    const size_t gpar = (size_t)LL::N * a.Vh;
    const LC *G = reinterpret_cast<const LC *>(a.gauge);
    const LC *Gout = G + (size_t)op * gpar, *Gin = G + (size_t)(1 - op) * gpar;
    const SC *in = reinterpret_cast<const SC *>(a.in);
    // neighbour indices of the 8 hops (forward, backward for mu = x, y, z, t)
    const int sy = a.X1h, sz = a.X1h * a.Ly, st = a.X1h * a.Ly * a.Lz;
    const int n0 = row + (((x == a.Lx - 1) ? 0 : x + 1) >> 1), n1 = row + (((x == 0) ? a.Lx - 1 : x - 1) >> 1);
    const int n2 = (y == a.Ly - 1) ? cb - (a.Ly - 1) * sy : cb + sy, n3 = (y == 0) ? cb + (a.Ly - 1) * sy : cb - sy;
    const int n4 = (z == a.Lz - 1) ? cb - (a.Lz - 1) * sz : cb + sz, n5 = (z == 0) ? cb + (a.Lz - 1) * sz : cb - sz;
    const int n6 = (t == a.Lt - 1) ? cb - (a.Lt - 1) * st : cb + st, n7 = (t == 0) ? cb + (a.Lt - 1) * st : cb - st;
    const T one = T(1);
    const T sgf = (t == a.Lt - 1 && a.tbc) ? -one : one, sgb = (t == 0 && a.tbc) ? -one : one;
    const T spf = -a.sigma, spb = a.sigma;

    T acc[NF][24];
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
        for (int k = 0; k < 24; k++) acc[f][k] = T(0);
    HopRaw<PREC, RECON, NF> ra, rb;
    const size_t m2 = 2 * gpar;
    fetch_hop(ra, Gout + 0 * m2, cb, in, a.in_norm, n0, a.Vh);
    fetch_hop(rb, Gin + 0 * m2, n1, in, a.in_norm, n1, a.Vh);
    compute_hop<PREC, RECON, NF, 0, true>(acc, ra, spf, one);
    fetch_hop(ra, Gout + 1 * m2, cb, in, a.in_norm, n2, a.Vh);
    compute_hop<PREC, RECON, NF, 0, false>(acc, rb, spb, one);
    fetch_hop(rb, Gin + 1 * m2, n3, in, a.in_norm, n3, a.Vh);
    compute_hop<PREC, RECON, NF, 1, true>(acc, ra, spf, one);
    fetch_hop(ra, Gout + 2 * m2, cb, in, a.in_norm, n4, a.Vh);
    compute_hop<PREC, RECON, NF, 1, false>(acc, rb, spb, one);
    fetch_hop(rb, Gin + 2 * m2, n5, in, a.in_norm, n5, a.Vh);
    compute_hop<PREC, RECON, NF, 2, true>(acc, ra, spf, one);
    fetch_hop(ra, Gout + 3 * m2, cb, in, a.in_norm, n6, a.Vh);
    compute_hop<PREC, RECON, NF, 2, false>(acc, rb, spb, one);
    fetch_hop(rb, Gin + 3 * m2, n7, in, a.in_norm, n7, a.Vh);
    compute_hop<PREC, RECON, NF, 3, true>(acc, ra, spf, sgf);
    compute_hop<PREC, RECON, NF, 3, false>(acc, rb, spb, sgb);

    const size_t fstride = (size_t)Traits<PREC>::SCHUNKS * a.Vh;
    const int epi = a.epilogue;
    if (epi == EPI_SCALE) {
#pragma unroll
        for (int f = 0; f < NF; f++)
#pragma unroll
            for (int k = 0; k < 24; k++) acc[f][k] *= a.coef;
    } else if (epi == EPI_TW) {
        apply_twist<T, NF>(a.tw_epi, acc);
    } else {
        T xv[NF][24];
        const SC *X = reinterpret_cast<const SC *>(a.x);
#pragma unroll
        for (int f = 0; f < NF; f++)
            load_spinor<PREC>(X + f * fstride, a.x_norm ? a.x_norm + (size_t)f * a.Vh : nullptr, cb, a.Vh, xv[f]);
        if (epi == EPI_TWX_AXPY || epi == EPI_TWX_AXPY_TW) {
            apply_twist<T, NF>(a.tw_epi, xv);
        } else if (epi == EPI_X_TWAXPY) {
            apply_twist<T, NF>(a.tw_epi, acc);
        }
#pragma unroll
        for (int f = 0; f < NF; f++)
#pragma unroll
            for (int k = 0; k < 24; k++) acc[f][k] = fma(a.coef, acc[f][k], xv[f][k]);
        if (epi == EPI_TW_XPAY) apply_twist<T, NF>(a.tw_epi, acc);
        else if (epi == EPI_TWX_AXPY_TW) apply_twist<T, NF>(a.tw_acc, acc);
    }
    SC *O = reinterpret_cast<SC *>(a.out);
#pragma unroll
    for (int f = 0; f < NF; f++)
        store_spinor<PREC>(O + f * fstride, a.out_norm ? a.out_norm + (size_t)f * a.Vh : nullptr, cb, a.Vh, acc[f]);
}

// ------------------------------------------------------------------------------------------
// Variant 6: the two-stage pipeline of variant 2 with the staging in shared memory instead of
// registers.  cp.async copies the raw chunks of hop h+1 (link, neighbour spinors, FP16 norms)
// into this thread's slots of a double buffer while hop h is computed, so every warp keeps a
// hop of loads in flight during its arithmetic without holding them in registers.  Shared
// memory per block: 2 buffers x 128 threads x (link + spinor + norm bytes of one hop), laid out
// [chunk][thread] so a warp's 16-byte reads are conflict-free.  Each thread reads back only its
// own copies (cp.async.wait_group), so no block barrier is needed.
template <int PREC, int RECON, int NF>
struct AsyncHop {
    using LC = typename LinkLayout<PREC, RECON>::chunk;
    using SC = typename Traits<PREC>::schunk;
    static constexpr int NL = LinkLayout<PREC, RECON>::N;
    static constexpr int NS = NF * Traits<PREC>::SCHUNKS;
    static constexpr int NN = (PREC == P16) ? NF : 0;
    static constexpr int BS = 128;
    static constexpr int LBYTES = NL * BS * (int)sizeof(LC);  // a multiple of 16
    static constexpr int BUF = LBYTES + NS * BS * 16 + NN * BS * 4;
};

template <int N>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const size_t g = __cvta_generic_to_global(gmem);
    if constexpr (N == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(g) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(g), "n"(N) : "memory");
}
// the same copy allocating in L1 (links shared by the warps of a multi-RHS block)
template <int N>
__device__ __forceinline__ void cp_async_l1(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const size_t g = __cvta_generic_to_global(gmem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(g), "n"(N) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int PREC, int RECON, int NF, bool L1LINK = false>
__device__ __forceinline__ void async_fetch_hop(char *buf, int tid, const typename LinkLayout<PREC, RECON>::chunk *g,
                                                int lcb, const typename Traits<PREC>::schunk *in, const float *in_norm,
                                                int nb, int Vh)
{
    using H = AsyncHop<PREC, RECON, NF>;
    using LC = typename H::LC;
    using SC = typename H::SC;
    LC *sl = reinterpret_cast<LC *>(buf);
    SC *ss = reinterpret_cast<SC *>(buf + H::LBYTES);
#pragma unroll
    for (int k = 0; k < H::NL; k++) {
        if constexpr (L1LINK) cp_async_l1<(int)sizeof(LC)>(sl + k * H::BS + tid, g + (size_t)k * Vh + lcb);
        else cp_async<(int)sizeof(LC)>(sl + k * H::BS + tid, g + (size_t)k * Vh + lcb);
    }
#pragma unroll
    for (int k = 0; k < H::NS; k++) cp_async<16>(ss + k * H::BS + tid, in + (size_t)k * Vh + nb);
    if constexpr (H::NN > 0) {
        float *sn = reinterpret_cast<float *>(buf + H::LBYTES + H::NS * H::BS * 16);
#pragma unroll
        for (int f = 0; f < H::NN; f++) cp_async<4>(sn + f * H::BS + tid, in_norm + (size_t)f * Vh + nb);
    }
}

template <int PREC, int RECON, int NF, int MU, bool FWD, bool PRO = false, bool PAIR = false, typename T>
__device__ __forceinline__ void async_compute_hop(T (&acc)[NF][24], const char *buf, int tid, T sp, T sg,
                                                  const Twist<T> *tw = nullptr)
{
    using H = AsyncHop<PREC, RECON, NF>;
    using LC = typename H::LC;
    using SC = typename H::SC;
    HopRaw<PREC, RECON, NF> r;
    const LC *sl = reinterpret_cast<const LC *>(buf);
    const SC *ss = reinterpret_cast<const SC *>(buf + H::LBYTES);
#pragma unroll
    for (int k = 0; k < H::NL; k++) r.l[k] = sl[k * H::BS + tid];
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
        for (int k = 0; k < Traits<PREC>::SCHUNKS; k++) r.s[f][k] = ss[(f * Traits<PREC>::SCHUNKS + k) * H::BS + tid];
    if constexpr (H::NN > 0) {
        const float *sn = reinterpret_cast<const float *>(buf + H::LBYTES + H::NS * H::BS * 16);
#pragma unroll
        for (int f = 0; f < NF; f++) r.n[f] = sn[f * H::BS + tid];
    }
    compute_hop<PREC, RECON, NF, MU, FWD, PRO, PAIR>(acc, r, sp, sg, tw);
}

// the epilogue input x of this thread's site into the spinor / norm area of a buffer
template <int PREC, int RECON, int NF>
__device__ __forceinline__ void async_fetch_x(char *buf, int tid, const typename Traits<PREC>::schunk *X,
                                              const float *x_norm, int cb, int Vh)
{
    using H = AsyncHop<PREC, RECON, NF>;
    using SC = typename H::SC;
    SC *ss = reinterpret_cast<SC *>(buf + H::LBYTES);
#pragma unroll
    for (int k = 0; k < H::NS; k++) cp_async<16>(ss + k * H::BS + tid, X + (size_t)k * Vh + cb);
    if constexpr (H::NN > 0) {
        float *sn = reinterpret_cast<float *>(buf + H::LBYTES + H::NS * H::BS * 16);
#pragma unroll
        for (int f = 0; f < H::NN; f++) cp_async<4>(sn + f * H::BS + tid, x_norm + (size_t)f * Vh + cb);
    }
}

template <int PREC, int RECON, int NF, typename T>
__device__ __forceinline__ void async_read_x(const char *buf, int tid, T (&xv)[NF][24])
{
    using H = AsyncHop<PREC, RECON, NF>;
    using SC = typename H::SC;
    const SC *ss = reinterpret_cast<const SC *>(buf + H::LBYTES);
#pragma unroll
    for (int f = 0; f < NF; f++) {
        SC c[Traits<PREC>::SCHUNKS];
#pragma unroll
        for (int k = 0; k < Traits<PREC>::SCHUNKS; k++) c[k] = ss[(f * Traits<PREC>::SCHUNKS + k) * H::BS + tid];
        spinor_from_chunks<PREC>(c, xv[f]);
        if constexpr (H::NN > 0) {
            const float n = reinterpret_cast<const float *>(buf + H::LBYTES + H::NS * H::BS * 16)[f * H::BS + tid];
#pragma unroll
            for (int k = 0; k < 24; k++) xv[f][k] *= n;
        }
    }
}

// Completion flags of the fused operator (below): release after a tile's stores, acquire before
// a dependent tile's loads.  A wait is bounded in time: it gives up once the device's nanosecond
// clock (%globaltimer) shows more than `limit_ns` since it began, records the failure in the
// handle's error word (sync[0], kept until tm_device_status reads it) and in the launch's abort
// word (sync[2], cleared at every launch), and reports false; the caller then skips its site.  A
// wait also gives up at once when the abort word is set, so after a first failure no other site
// of the launch waits out a second limit (a flag that is set is still taken).  An iteration cap
// (2^24 polls, each at least one L2 round trip) backs the clock up.
__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// sync: [0] error word, [2] abort word of this launch
__device__ __forceinline__ bool wait_flag(const int *f, int *sync, unsigned long long limit_ns)
{
    if (ld_acquire_gpu(f) != 0) return true;
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < (1 << 24); i++) {
        if (ld_relaxed_gpu(sync + 2) != 0) return false;  // another wait of this launch gave up
        __nanosleep(200);
        if (ld_acquire_gpu(f) != 0) return true;
        if (global_ns() - t0 > limit_ns) break;
    }
    atomicExch(sync + 2, 1);
    atomicExch(sync, 1);
    return false;
}

template <int PREC, int NF, typename T>
__device__ __forceinline__ void store_out(const DslashArgs<T> &a, T (&acc)[NF][24], int cb, size_t boff, size_t noff)
{
    using SC = typename Traits<PREC>::schunk;
    const size_t fstride = (size_t)Traits<PREC>::SCHUNKS * a.Vh;
    SC *O = reinterpret_cast<SC *>(a.out) + boff;
    float *out_norm = a.out_norm ? a.out_norm + noff : nullptr;
#pragma unroll
    for (int f = 0; f < NF; f++)
        store_spinor<PREC>(O + f * fstride, out_norm ? out_norm + (size_t)f * a.Vh : nullptr, cb, a.Vh, acc[f]);
}

// One site of the staged hop pipeline (launch forms 6 / 7 and the fused operator).  WAIT: the
// input field is produced by other tiles of the same launch; before its first load the thread
// waits for the completion flags of the 128-site tiles that hold its 8 neighbours.
// RED: the site's share of the fused reduction of the output, returned in FP64: |out|^2, or for
// EPI_TWX_AXPY_TW Re<u, Q u> with u = T x + c acc (out = Q u); 0 otherwise.
template <int PREC, int NF, int RECON, bool CLOV, int NB, bool PRO, bool WAIT, bool PAIR = false, bool L1LINK = false,
          bool RED = false>
__device__ __forceinline__ double async_site(const DslashArgs<typename Traits<PREC>::real> &a, int cb, int tid,
                                             char *smem_async, const int *flags, int *sync,
                                             unsigned long long limit_ns = 0, int rhs = 0)
{
    using T = typename Traits<PREC>::real;
    using LL = LinkLayout<PREC, RECON>;
    using LC = typename LL::chunk;
    using SC = typename Traits<PREC>::schunk;
    using H = AsyncHop<PREC, RECON, NF>;
    int r = cb;
    const int xh = r % a.X1h;
    r /= a.X1h;
    const int y = r % a.Ly;
    r /= a.Ly;
    const int z = r % a.Lz;
    const int t = r / a.Lz;
    const int op = a.out_parity;
    const int x = 2 * xh + ((op + y + z + t) & 1);
    const int row = cb - xh;
    const size_t gpar = (size_t)LL::N * a.Vh;
    const LC *G = reinterpret_cast<const LC *>(a.gauge);
    const LC *Gout = G + (size_t)op * gpar, *Gin = G + (size_t)(1 - op) * gpar;
    // right-hand side `rhs` of a multi-RHS field: its flavour blocks start at rhs * NF
    const size_t boff = (size_t)rhs * NF * Traits<PREC>::SCHUNKS * a.Vh, noff = (size_t)rhs * NF * a.Vh;
    const SC *in = reinterpret_cast<const SC *>(a.in) + boff;
    const float *in_norm = a.in_norm ? a.in_norm + noff : nullptr;
    const int sy = a.X1h, sz = a.X1h * a.Ly, st = a.X1h * a.Ly * a.Lz;
    const int n0 = row + (((x == a.Lx - 1) ? 0 : x + 1) >> 1), n1 = row + (((x == 0) ? a.Lx - 1 : x - 1) >> 1);
    const int n2 = (y == a.Ly - 1) ? cb - (a.Ly - 1) * sy : cb + sy, n3 = (y == 0) ? cb + (a.Ly - 1) * sy : cb - sy;
    const int n4 = (z == a.Lz - 1) ? cb - (a.Lz - 1) * sz : cb + sz, n5 = (z == 0) ? cb + (a.Lz - 1) * sz : cb - sz;
    const int n6 = (t == a.Lt - 1) ? cb - (a.Lt - 1) * st : cb + st, n7 = (t == 0) ? cb + (a.Lt - 1) * st : cb - st;
    const T one = T(1);
    const T sgf = (t == a.Lt - 1 && a.tbc) ? -one : one, sgb = (t == 0 && a.tbc) ? -one : one;
    const T spf = -a.sigma, spb = a.sigma;
    const size_t m2 = 2 * gpar;

    T acc[NF][24];
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
        for (int k = 0; k < 24; k++) acc[f][k] = T(0);
    // hop h: (mu, forward?) = (h / 2, h even); link at the output site (forward) or at the neighbour
    const int nbr[8] = {n0, n1, n2, n3, n4, n5, n6, n7};
    if constexpr (WAIT) {
        bool ok = true;
#pragma unroll
        for (int h = 0; h < 8; h++) ok = ok && wait_flag(flags + (nbr[h] >> 7), sync, limit_ns);
        if (!ok) return 0.0;
    }
    auto fetch = [&](int h) {
        char *b = smem_async + (h % NB) * H::BUF;
        const int mu = h >> 1;
        if ((h & 1) == 0) async_fetch_hop<PREC, RECON, NF, L1LINK>(b, tid, Gout + mu * m2, cb, in, in_norm, nbr[h], a.Vh);
        else async_fetch_hop<PREC, RECON, NF, L1LINK>(b, tid, Gin + mu * m2, nbr[h], in, in_norm, nbr[h], a.Vh);
        cp_commit();
    };
#pragma unroll
    for (int h = 0; h < NB; h++) fetch(h);
    const int epi = a.epilogue;
    const bool needx = epi != EPI_SCALE && epi != EPI_TW;
#pragma unroll
    for (int h = 0; h < 8; h++) {
        // groups committed after hop h's: the hops up to min(h + NB - 1, 7), and the epilogue
        // input once hop 8 - NB has been computed; hop h itself must be complete
        const int later = (h + NB - 1 < 7 ? h + NB - 1 : 7) - h + (h > 8 - NB ? 1 : 0);
        if (later >= 2) cp_wait<2>();
        else if (later == 1) cp_wait<1>();
        else cp_wait<0>();
        const char *b = smem_async + (h % NB) * H::BUF;
        const Twist<T> *tw = &a.tw_pro;
        switch (h) {
        case 0: async_compute_hop<PREC, RECON, NF, 0, true, PRO, PAIR>(acc, b, tid, spf, one, tw); break;
        case 1: async_compute_hop<PREC, RECON, NF, 0, false, PRO, PAIR>(acc, b, tid, spb, one, tw); break;
        case 2: async_compute_hop<PREC, RECON, NF, 1, true, PRO, PAIR>(acc, b, tid, spf, one, tw); break;
        case 3: async_compute_hop<PREC, RECON, NF, 1, false, PRO, PAIR>(acc, b, tid, spb, one, tw); break;
        case 4: async_compute_hop<PREC, RECON, NF, 2, true, PRO, PAIR>(acc, b, tid, spf, one, tw); break;
        case 5: async_compute_hop<PREC, RECON, NF, 2, false, PRO, PAIR>(acc, b, tid, spb, one, tw); break;
        case 6: async_compute_hop<PREC, RECON, NF, 3, true, PRO, PAIR>(acc, b, tid, spf, sgf, tw); break;
        default: async_compute_hop<PREC, RECON, NF, 3, false, PRO, PAIR>(acc, b, tid, spb, sgb, tw); break;
        }
        if (h + NB < 8) fetch(h + NB);
        else if (h + NB == 8) {
            // the epilogue input streams in, into the buffer hop h used, while the last hops compute
            if (needx) async_fetch_x<PREC, RECON, NF>(smem_async + (h % NB) * H::BUF, tid,
                                                     reinterpret_cast<const SC *>(a.x) + boff,
                                                     a.x_norm ? a.x_norm + noff : nullptr, cb, a.Vh);
            cp_commit();
        }
        if constexpr (RED) {
            if (h == 7 && epi == EPI_TWX_AXPY_RUPD) {
                // the residual this launch updates in place streams into the buffer hop 7 used
                // while the twist of x is computed
                async_fetch_x<PREC, RECON, NF>(smem_async + (7 % NB) * H::BUF, tid,
                                               reinterpret_cast<const SC *>(a.out) + boff,
                                               a.out_norm ? a.out_norm + noff : nullptr, cb, a.Vh);
                cp_commit();
            }
        }
    }
    const char *xbuf = smem_async + ((8 - NB) % NB) * H::BUF;

    const size_t fstride = (size_t)Traits<PREC>::SCHUNKS * a.Vh;
    if (epi == EPI_SCALE) {
#pragma unroll
        for (int f = 0; f < NF; f++)
#pragma unroll
            for (int k = 0; k < 24; k++) acc[f][k] *= a.coef;
    } else if (epi == EPI_TW) {
        local_op<PREC, NF, CLOV, true>(a, cb, acc);
    } else {
        T xv[NF][24];
        if constexpr (RED) {
            if (epi == EPI_TWX_AXPY_RUPD) cp_wait<1>();  // x; the residual may still be in flight
            else cp_wait<0>();
        } else {
            cp_wait<0>();
        }
        async_read_x<PREC, RECON, NF>(xbuf, tid, xv);
        if (epi == EPI_TWX_AXPY || epi == EPI_TWX_AXPY_TW || epi == EPI_TWX_AXPY_RUPD)
            local_op<PREC, NF, CLOV, false>(a, cb, xv);
        else if (epi == EPI_X_TWAXPY) local_op<PREC, NF, CLOV, true>(a, cb, acc);
#pragma unroll
        for (int f = 0; f < NF; f++)
#pragma unroll
            for (int k = 0; k < 24; k++) acc[f][k] = fma(a.coef, acc[f][k], xv[f][k]);
        if (epi == EPI_TW_XPAY) {
            local_op<PREC, NF, CLOV, true>(a, cb, acc);
        } else if (epi == EPI_TWX_AXPY_RUPD) {
            if constexpr (RED) {
                // r - s u with u = T x + c acc as the separate pass computes it from a stored u
                // (binary32: the same bits); the |out|^2 share below is then |r|^2
                cp_wait<0>();
                async_read_x<PREC, RECON, NF>(smem_async + (7 % NB) * H::BUF, tid, xv);
                const T ms = -T(__ldg(a.scal_in));
#pragma unroll
                for (int f = 0; f < NF; f++)
#pragma unroll
                    for (int k = 0; k < 24; k++) acc[f][k] = fma(ms, acc[f][k], xv[f][k]);
            }
        } else if (epi == EPI_TWX_AXPY_TW) {
            if constexpr (RED) {  // Re<u, Q u> (Q hermitian): u is acc before the twist
#pragma unroll
                for (int f = 0; f < NF; f++)
#pragma unroll
                    for (int k = 0; k < 24; k++) xv[f][k] = acc[f][k];
            }
            apply_twist<T, NF>(a.tw_acc, acc);
            if constexpr (RED) {
                double part = 0.0;
#pragma unroll
                for (int f = 0; f < NF; f++) {
                    T sf = T(0);
#pragma unroll
                    for (int k = 0; k < 24; k++) sf = fma(xv[f][k], acc[f][k], sf);
                    part += (double)sf;
                }
                store_out<PREC, NF>(a, acc, cb, boff, noff);
                return part;
            }
        }
    }
    store_out<PREC, NF>(a, acc, cb, boff, noff);
    double part = 0.0;
    if constexpr (RED) {
#pragma unroll
        for (int f = 0; f < NF; f++) {
            T sf = T(0);
#pragma unroll
            for (int k = 0; k < 24; k++) sf = fma(acc[f][k], acc[f][k], sf);
            part += (double)sf;
        }
    }
    return part;
}

// RED: the launch also reduces its output (async_site): each warp writes the sum of its 32 sites'
// shares to red.partials[4 * block + warp] (warp shuffles, no block barrier); k_finish_partials
// then adds them in a fixed order and applies red.fin.
template <int PREC, int NF, int RECON, int MINB, bool CLOV = false, int NB = 2, bool PRO = false, bool PAIR = false,
          bool RED = false>
__global__ void __launch_bounds__(128, MINB) k_dslash_async(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a,
                                                            const __grid_constant__ RedArgs red)
{
    extern __shared__ __align__(16) char smem_async[];
    const int tid = threadIdx.x;
    const int cb = a.cb0 + blockIdx.x * AsyncHop<PREC, RECON, NF>::BS + tid;
    if constexpr (!RED) {
        if (cb >= a.cb0 + a.ncb) return;
        async_site<PREC, NF, RECON, CLOV, NB, PRO, false, PAIR>(a, cb, tid, smem_async, nullptr, nullptr);
    } else {
        double part = 0.0;  // every lane takes part in the warp reduction
        if (cb < a.cb0 + a.ncb)
            part = async_site<PREC, NF, RECON, CLOV, NB, PRO, false, PAIR, false, true>(a, cb, tid, smem_async, nullptr,
                                                                                          nullptr);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if ((tid & 31) == 0) red.partials[(size_t)blockIdx.x * 4 + (tid >> 5)] = part;
    }
}

// ------------------------------------------------------------------------------------------
// The fused preconditioned operator: both launches of M_pc (A: t = T_oo H_oe in, B: out = ...
// H_eo t) in one persistent launch.  The 128-site tiles of A and B are claimed from a device
// work list in an order where every B tile comes after the A tiles its neighbours live in (the
// A tiles of the last time slice first, then A ahead of B by one time slice and a few tiles), so
// each t tile is read back by B shortly after A wrote it: the intermediate field and the links
// both passes read stay in L2 instead of making a second trip through HBM.  A tile's completion
// is published with a release flag once all its threads' stores are done; a B site acquires the
// flags of its neighbours' tiles before loading them (bounded waits).  Claiming in list order
// means a waited-for tile has always been claimed by a running block, so the waits end.
// sync: [0] error word (kept until read), [1] work counter, [2] abort word of the launch,
// [3 + tile] A-tile completion flags; the counter, the abort word and the flags are zero at launch.
constexpr int FUSED_GROUP = 4;  // 128-site tiles per work item of the fused operator

template <int PREC, int NF, int RECON, int MINB>
__global__ void __launch_bounds__(128, MINB)
    k_mpc_fused(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> aA,
                const __grid_constant__ DslashArgs<typename Traits<PREC>::real> aB, const int *__restrict__ items,
                int nitems, int *sync, unsigned long long limit_ns)
{
    extern __shared__ __align__(16) char smem_async[];
    __shared__ int s_q;
    // the hop of the default launch form: paired (8 / 9) except one flavour with 18-real links
    constexpr bool FPAIR = PREC == P32 && (NF == 2 || RECON != 18);
    int *counter = sync + 1, *flags = sync + 3;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_q = atomicAdd(counter, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();  // every thread has read s_q before it is claimed again
        if (q >= nitems) break;
        const int it = __ldg(items + q);
        const int grp = it >> 1;  // FUSED_GROUP consecutive 128-site tiles per work item
        if (it & 1) {
            for (int sub = 0; sub < FUSED_GROUP; sub++) {
                const int cb = (grp * FUSED_GROUP + sub) * 128 + tid;
                if (cb < aB.Vh) async_site<PREC, NF, RECON, false, 2, false, true, FPAIR>(aB, cb, tid, smem_async, flags, sync, limit_ns);
            }
        } else {
            for (int sub = 0; sub < FUSED_GROUP; sub++) {
                const int cb = (grp * FUSED_GROUP + sub) * 128 + tid;
                if (cb < aA.Vh)
                    async_site<PREC, NF, RECON, false, 2, false, false, FPAIR>(aA, cb, tid, smem_async, nullptr, nullptr);
            }
            // the block's stores happen before one thread's gpu-scope release of the tiles
            __syncthreads();
            if (tid < FUSED_GROUP) {
                __threadfence();
                st_release_gpu(flags + grp * FUSED_GROUP + tid, 1);
            }
        }
    }
}

// The shared-memory opt-in is set once per kernel and device: the attribute call is not a
// stream operation and can wait for work already queued on the device, so it must stay out of
// the per-launch path (it would serialise copy streams with the compute stream).
template <int PREC, int NF, int RECON, int MINB, bool CLOV = false, int NB = 2, bool PRO = false, bool PAIR = false,
          bool RED = false>
cudaError_t launch_async(const DslashArgs<typename Traits<PREC>::real> &a, cudaStream_t s, const RedArgs *red = nullptr)
{
    constexpr int bytes = NB * AsyncHop<PREC, RECON, NF>::BUF;
    static std::atomic<unsigned long long> opted{0};  // bit d: done on device d (d < 64)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(opted.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_dslash_async<PREC, NF, RECON, MINB, CLOV, NB, PRO, PAIR, RED>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        opted.fetch_or(bit, std::memory_order_acq_rel);
    }
    RedArgs r;
    memset(&r, 0, sizeof(r));
    if (red) r = *red;
    k_dslash_async<PREC, NF, RECON, MINB, CLOV, NB, PRO, PAIR, RED><<<(a.ncb + 127) / 128, 128, bytes, s>>>(a, r);
    return cudaGetLastError();
}

// Multi-RHS with the staged hop pipeline (multi-RHS launch forms 12 / 14): a 128-thread block is
// 128 / RPB consecutive sites x RPB right-hand sides, a warp being 32 sites of one right-hand side
// (its spinor chunks are one contiguous 512-byte request).  Every thread runs the two-buffer
// staged pipeline of launch form 8 / 9 (paired hop where that form pairs) for its (site, source);
// the link chunks are copied with L1 allocation, so the RPB warps that read the same links are
// served by one trip to L2, and consecutive blocks take the next RPB sources of the same sites,
// so links leave DRAM about once per site for all sources.
template <int PREC, int NF, int RECON, bool PRO, int RPB, bool PAIR, int NB = 2>
__global__ void __launch_bounds__(128, NB == 3 ? 2 : 3)
    k_dslash_multi_async(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a, const int *__restrict__ act,
                         int nact, int nrhs, int gmajor)
{
    extern __shared__ __align__(16) char smem_async[];
    constexpr int WPR = 4 / RPB;  // warps per right-hand side
    const int tid = threadIdx.x, w = tid >> 5;
    const int ngrp = (nact + RPB - 1) / RPB;
    // block order: interleaved (the groups of RPB sources of a site block one after another, so the
    // links are shared through L2 by all sources) or group-major (one sweep over the sites per group:
    // the links are read once per group, but a sweep's neighbour spinors stay within L2's reach)
    const long nsblk = ((long)a.Vh + 32 * WPR - 1) / (32 * WPR);
    const int grp = gmajor ? (int)(blockIdx.x / nsblk) : (int)(blockIdx.x % ngrp);
    const long sblk = gmajor ? (long)(blockIdx.x % nsblk) : (long)(blockIdx.x / ngrp);
    const int slot = grp * RPB + w / WPR;
    const long cb = sblk * (32 * WPR) + (w % WPR) * 32 + (tid & 31);
    if (slot >= nact || cb >= a.Vh) return;
    const int rhs = act ? __ldg(act + slot) : slot;
    if (rhs < 0 || rhs >= nrhs) return;  // an index outside the fields is skipped, never dereferenced
    async_site<PREC, NF, RECON, false, NB, PRO, false, PAIR, true>(a, (int)cb, tid, smem_async, nullptr, nullptr, 0, rhs);
}

template <int PREC, int NF, int RECON, bool PRO, int RPB, bool PAIR, int NB = 2>
cudaError_t launch_multi_async(const DslashArgs<typename Traits<PREC>::real> &a, const int *act, int nact, int nrhs,
                               bool gmajor, cudaStream_t s)
{
    constexpr int bytes = NB * AsyncHop<PREC, RECON, NF>::BUF;
    static std::atomic<unsigned long long> opted{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(opted.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_dslash_multi_async<PREC, NF, RECON, PRO, RPB, PAIR, NB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        opted.fetch_or(bit, std::memory_order_acq_rel);
    }
    constexpr int SPB = 128 / RPB;  // sites per block
    const unsigned grid = (unsigned)(((long)a.Vh + SPB - 1) / SPB * ((nact + RPB - 1) / RPB));
    k_dslash_multi_async<PREC, NF, RECON, PRO, RPB, PAIR, NB><<<grid, 128, bytes, s>>>(a, act, nact, nrhs, gmajor ? 1 : 0);
    return cudaGetLastError();
}

// The fused operator's launch: a resident wave of blocks (occupancy calculator, once per kernel).
template <int PREC, int NF, int RECON>
cudaError_t launch_fused_impl(const DslashArgs<typename Traits<PREC>::real> &aA,
                              const DslashArgs<typename Traits<PREC>::real> &aB, const int *items, int nitems,
                              int *sync, unsigned long long limit_ns, int num_sms, cudaStream_t s)
{
    constexpr int bytes = 2 * AsyncHop<PREC, RECON, NF>::BUF;
    static std::atomic<unsigned long long> opted{0};
    static std::atomic<int> per_sm{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(opted.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_mpc_fused<PREC, NF, RECON, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        opted.fetch_or(bit, std::memory_order_acq_rel);
    }
    int b = per_sm.load(std::memory_order_relaxed);
    if (b == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mpc_fused<PREC, NF, RECON, 3>, 128, bytes);
        if (e != cudaSuccess) return e;
        b = b > 0 ? b : 1;
        per_sm.store(b, std::memory_order_relaxed);
    }
    const int grid = (num_sms > 0 ? num_sms : 1) * b;
    k_mpc_fused<PREC, NF, RECON, 3><<<grid, 128, bytes, s>>>(aA, aB, items, nitems, sync, limit_ns);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_fused_dispatch(const DslashArgs<typename Traits<PREC>::real> &aA,
                                  const DslashArgs<typename Traits<PREC>::real> &aB, int nf, int recon,
                                  const int *items, int nitems, int *sync, unsigned long long limit_ns, int num_sms,
                                  cudaStream_t s)
{
#define TM_FU(NF, R) return launch_fused_impl<PREC, NF, R>(aA, aB, items, nitems, sync, limit_ns, num_sms, s);
#define TM_FUR(NF)                         \
    switch (recon) {                       \
    case 18: TM_FU(NF, 18)                 \
    case 12: TM_FU(NF, 12)                 \
    case 8: TM_FU(NF, 8)                   \
    default: return cudaErrorInvalidValue; \
    }
    if (nf == 1) { TM_FUR(1) } else { TM_FUR(2) }
#undef TM_FUR
#undef TM_FU
}

// Clover handles: the same hopping sum with the per-site local operator L = C + X (or L^-1) in
// the epilogue instead of the constant twist; no input prologue (the operators apply L^-1 to an
// input as a pass of its own).  The epilogue reads 72 (L) or 144 (L^-1) more reals per site.
// The binary32 doublet takes the flavour-paired hop (hop_pair) in both clover forms.
template <int PREC, int NF, int RECON, int MINB = 1>
__global__ void __launch_bounds__(128, MINB) k_dslash_clov(const __grid_constant__ DslashArgs<typename Traits<PREC>::real> a)
{
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= a.Vh) return;
    dslash_body<PREC, NF, RECON, false, true, NF == 2>(a, cb, 0);
}

template <int PREC>
cudaError_t launch_dslash_clov_impl(const DslashArgs<typename Traits<PREC>::real> &a, int nf, int recon, int minb,
                                    cudaStream_t s)
{
    // minb: resident 128-thread blocks per SM the register allocation must allow (1, 3 or 4), or 6:
    // the shared-memory staged pipeline (3 blocks per SM)
    if (minb != 1 && minb != 3 && minb != 4 && minb != 6) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)((a.Vh + 127) / 128);
#define TM_CL1(NF, R)                                                               \
    if (minb == 6) return launch_async<PREC, NF, R, 3, true, 2, false, NF == 2>(a, s); \
    if (minb == 1) k_dslash_clov<PREC, NF, R, 1><<<grid, 128, 0, s>>>(a);           \
    else if (minb == 3) k_dslash_clov<PREC, NF, R, 3><<<grid, 128, 0, s>>>(a);      \
    else k_dslash_clov<PREC, NF, R, 4><<<grid, 128, 0, s>>>(a);
#define TM_CL(NF)                          \
    switch (recon) {                       \
    case 18: { TM_CL1(NF, 18) } break;     \
    case 12: { TM_CL1(NF, 12) } break;     \
    case 8: { TM_CL1(NF, 8) } break;       \
    default: return cudaErrorInvalidValue; \
    }
    if (nf == 1) { TM_CL(1) } else { TM_CL(2) }
#undef TM_CL
#undef TM_CL1
    return cudaGetLastError();
}

// the staged forms: nb3 = three buffers (2 blocks per SM) instead of two (3 blocks per SM)
template <int PREC, int NF, int RECON, bool PAIR>
cudaError_t launch_staged(const DslashArgs<typename Traits<PREC>::real> &a, bool pro, bool nb3, cudaStream_t s)
{
    if (pro)
        return nb3 ? launch_async<PREC, NF, RECON, 2, false, 3, true, PAIR>(a, s)
                   : launch_async<PREC, NF, RECON, 3, false, 2, true, PAIR>(a, s);
    return nb3 ? launch_async<PREC, NF, RECON, 2, false, 3, false, PAIR>(a, s)
               : launch_async<PREC, NF, RECON, 3, false, 2, false, PAIR>(a, s);
}

// The staged forms (variants 6 - 9, no prologue) with the fused reduction of the output.
template <int PREC>
cudaError_t launch_dslash_red_impl(const DslashArgs<typename Traits<PREC>::real> &a, int nf, int recon, int variant,
                                   const RedArgs &red, cudaStream_t s)
{
    if (variant < 6 || variant > 9) return cudaErrorInvalidValue;
    const bool nb3 = variant == 7 || variant == 9, pair = variant >= 8;
    constexpr bool CP = PREC == P32 || PREC == P16;
#define TM_RD2(NF, R, P)                                                                          \
    return nb3 ? launch_async<PREC, NF, R, 2, false, 3, false, P, true>(a, s, &red)               \
               : launch_async<PREC, NF, R, 3, false, 2, false, P, true>(a, s, &red);
#define TM_RD1(NF, R) if (pair) { TM_RD2(NF, R, CP) } else { TM_RD2(NF, R, false) }
#define TM_RDR(NF)                             \
    switch (recon) {                           \
    case 18: { TM_RD1(NF, 18) }                \
    case 12: { TM_RD1(NF, 12) }                \
    case 8: { TM_RD1(NF, 8) }                  \
    default: return cudaErrorInvalidValue;     \
    }
    if (nf == 1) { TM_RDR(1) } else { TM_RDR(2) }
#undef TM_RDR
#undef TM_RD1
#undef TM_RD2
}

// variant 0: one thread per site (both flavours); variant 2: the two-stage load pipeline (no
// prologue); variant 3: variant 0 with a register cap (4 resident 128-thread blocks per SM).
template <int PREC>
cudaError_t launch_dslash_impl(const DslashArgs<typename Traits<PREC>::real> &a, int nf, int recon, bool pro,
                               int variant, int block, cudaStream_t s)
{
    if (variant == 3 || variant == 4 || variant == 5) {
        // register-capped launches, 128 registers per thread: 128 x 4, 64 x 8 or 256 x 2 blocks per SM
        const int bs = variant == 3 ? 128 : (variant == 4 ? 64 : 256);
        const int gb = (a.ncb + bs - 1) / bs;
#define TM_LB1(NF, R, P)                                                                        \
    if (variant == 3) k_dslash_lb<PREC, NF, R, P, 4, 128><<<gb, 128, 0, s>>>(a);                 \
    else if (variant == 4) k_dslash_lb<PREC, NF, R, P, 8, 64><<<gb, 64, 0, s>>>(a);              \
    else k_dslash_lb<PREC, NF, R, P, 2, 256><<<gb, 256, 0, s>>>(a);
#define TM_LBR(NF, P)                   \
    switch (recon) {                    \
    case 18: { TM_LB1(NF, 18, P) } break; \
    case 12: { TM_LB1(NF, 12, P) } break; \
    case 8: { TM_LB1(NF, 8, P) } break;   \
    default: return cudaErrorInvalidValue; \
    }
        if (nf == 1) {
            if (pro) { TM_LBR(1, true) } else { TM_LBR(1, false) }
        } else {
            if (pro) { TM_LBR(2, true) } else { TM_LBR(2, false) }
        }
#undef TM_LBR
#undef TM_LB1
        return cudaGetLastError();
    }
    if (variant >= 6 && variant <= 9) {
        // shared-memory staged pipeline, 6: two buffers (hop h+1 in flight while hop h computes,
        // registers for 3 blocks per SM), 7: three buffers (hops h+1 and h+2 in flight, 2 blocks);
        // 8 / 9: 6 / 7 with the paired hop in binary32 (flavours paired for the doublet, spin
        // rows for one flavour; 6 / 7 in binary64)
        const bool nb3 = variant == 7 || variant == 9, pair = variant >= 8;
        constexpr bool CANPAIR = PREC == P32 || PREC == P16;
#define TM_ASR(NF, PAIR)                                                   \
    switch (recon) {                                                       \
    case 18: return launch_staged<PREC, NF, 18, PAIR>(a, pro, nb3, s);     \
    case 12: return launch_staged<PREC, NF, 12, PAIR>(a, pro, nb3, s);     \
    case 8: return launch_staged<PREC, NF, 8, PAIR>(a, pro, nb3, s);       \
    default: return cudaErrorInvalidValue;                                 \
    }
        if (nf == 1) {
            if (pair) { TM_ASR(1, CANPAIR) } else { TM_ASR(1, false) }
        } else {
            if (pair) { TM_ASR(2, CANPAIR) } else { TM_ASR(2, false) }
        }
#undef TM_ASR
    }
    const int grid = (a.ncb + block - 1) / block;
    if (variant == 2 && !pro) {
#define TM_PIPE(NF)                                                                 \
    switch (recon) {                                                                \
    case 18: k_dslash_pipe<PREC, NF, 18><<<grid, block, 0, s>>>(a); break;          \
    case 12: k_dslash_pipe<PREC, NF, 12><<<grid, block, 0, s>>>(a); break;          \
    case 8: k_dslash_pipe<PREC, NF, 8><<<grid, block, 0, s>>>(a); break;            \
    default: return cudaErrorInvalidValue;                                          \
    }
        if (nf == 1) { TM_PIPE(1) } else { TM_PIPE(2) }
#undef TM_PIPE
        return cudaGetLastError();
    }
#define TM_LAUNCH(NF, R, P) k_dslash<PREC, NF, R, P><<<grid, block, 0, s>>>(a)
#define TM_RECON(NF, P)                  \
    switch (recon) {                     \
    case 18: TM_LAUNCH(NF, 18, P); break; \
    case 12: TM_LAUNCH(NF, 12, P); break; \
    case 8: TM_LAUNCH(NF, 8, P); break;   \
    default: return cudaErrorInvalidValue; \
    }
    if (nf == 1) {
        if (pro) { TM_RECON(1, true) } else { TM_RECON(1, false) }
    } else {
        if (pro) { TM_RECON(2, true) } else { TM_RECON(2, false) }
    }
#undef TM_RECON
#undef TM_LAUNCH
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_dslash_multi_impl(const DslashArgs<typename Traits<PREC>::real> &a, int nf, int recon, bool pro,
                                     const int *act, int nact, int nrhs, int rpb, cudaStream_t s)
{
    // staged forms: 12 / 14 (2 / 4 per block, interleaved order), + 20 for the group-major order;
    // 16 / 36 (paired sources) are arranged by the caller, otherwise they run as 14 / 34;
    // 13 / 15 (+ 20): the same with three staging buffers (two hops in flight, as the single-RHS
    // form 9) for the binary16 doublet without the input prologue; every other case runs 12 / 14
    const bool gmajor = rpb >= 32;
    if (gmajor) rpb -= 20;
    if (rpb == 16) rpb = 14;
    if (rpb == 13 || rpb == 15) {
        if constexpr (PREC == P16) {
#define TM_MB1(R)                                                                                         \
    return rpb == 13 ? launch_multi_async<PREC, 2, R, false, 2, true, 3>(a, act, nact, nrhs, gmajor, s)   \
                     : launch_multi_async<PREC, 2, R, false, 4, true, 3>(a, act, nact, nrhs, gmajor, s);
            if (nf == 2 && !pro) {
                switch (recon) {
                case 18: TM_MB1(18)
                case 12: TM_MB1(12)
                case 8: TM_MB1(8)
                default: return cudaErrorInvalidValue;
                }
            }
#undef TM_MB1
        }
        rpb -= 1;
    }
    if (rpb == 12 || rpb == 14) {
        // staged multi-RHS forms, 2 or 4 right-hand sides per block; the hop pairs as form 8 / 9 does
        // (binary32 and binary16, except one flavour with 18-real links)
        constexpr bool CP = PREC == P32 || PREC == P16;
#define TM_MA1(NF, R, P)                                                                                 \
    {                                                                                                    \
        constexpr bool PR = CP && (NF == 2 || R != 18);                                                  \
        return rpb == 12 ? launch_multi_async<PREC, NF, R, P, 2, PR>(a, act, nact, nrhs, gmajor, s)      \
                         : launch_multi_async<PREC, NF, R, P, 4, PR>(a, act, nact, nrhs, gmajor, s);     \
    }
#define TM_MAR(NF, P)                          \
    switch (recon) {                           \
    case 18: TM_MA1(NF, 18, P)                 \
    case 12: TM_MA1(NF, 12, P)                 \
    case 8: TM_MA1(NF, 8, P)                   \
    default: return cudaErrorInvalidValue;     \
    }
        if (nf == 1) {
            if (pro) { TM_MAR(1, true) } else { TM_MAR(1, false) }
        } else {
            if (pro) { TM_MAR(2, true) } else { TM_MAR(2, false) }
        }
#undef TM_MAR
#undef TM_MA1
    }
    if (rpb != 2 && rpb != 4 && rpb != 8) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)(((long)a.Vh + 31) / 32 * ((nact + rpb - 1) / rpb));
#define TM_M1(NF, R, P, B) k_dslash_multi<PREC, NF, R, P, B><<<grid, 32 * B, 0, s>>>(a, act, nact, nrhs)
#define TM_M(NF, R, P)                     \
    if (rpb == 2) TM_M1(NF, R, P, 2);      \
    else if (rpb == 4) TM_M1(NF, R, P, 4); \
    else TM_M1(NF, R, P, 8);
#define TM_MR(NF, P)                                          \
    if (recon == 18) { TM_M(NF, 18, P) }                      \
    else if (recon == 12) { TM_M(NF, 12, P) }                 \
    else { TM_M(NF, 8, P) }
    if (nf == 1) {
        if (pro) { TM_MR(1, true) } else { TM_MR(1, false) }
    } else {
        if (pro) { TM_MR(2, true) } else { TM_MR(2, false) }
    }
#undef TM_MR
#undef TM_M
#undef TM_M1
    return cudaGetLastError();
}

}  // namespace tmk

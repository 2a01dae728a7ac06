// tm_api.cu -- the C ABI declared in include/tm.h: validation, the gauge handle, and the
// composition of fused launches into the preconditioned operators of eq. 2.2-2.4.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "tm_blas.cuh"
#include "tm_dslash.cuh"
#include "tm_internal.h"

namespace tmk {

cudaError_t launch_dslash_p64(const DslashArgs<double> &a, int nf, int recon, bool pro, int variant, int block,
                              cudaStream_t s);
cudaError_t launch_dslash_p32(const DslashArgs<float> &a, int nf, int recon, bool pro, int variant, int block,
                              cudaStream_t s);
cudaError_t launch_dslash_p16(const DslashArgs<float> &a, int nf, int recon, bool pro, int variant, int block,
                              cudaStream_t s);
#define TM_DF_DECL(NF, R)                                                                                    \
    cudaError_t launch_dslash_pdf_nf##NF##_r##R(const DslashArgs<df64> &a, int block, cudaStream_t s);                 \
    cudaError_t launch_dslash_multi_pdf_nf##NF##_r##R(const DslashArgs<df64> &a, const int *act, int nact, int nrhs, \
                                                      cudaStream_t s);
TM_DF_DECL(1, 18)
TM_DF_DECL(1, 12)
TM_DF_DECL(2, 18)
TM_DF_DECL(2, 12)
#undef TM_DF_DECL

static cudaError_t launch_dslash_pdf(const DslashArgs<df64> &a, int nf, int recon, int block, cudaStream_t s)
{
    if (nf == 1) return recon == 18 ? launch_dslash_pdf_nf1_r18(a, block, s) : launch_dslash_pdf_nf1_r12(a, block, s);
    return recon == 18 ? launch_dslash_pdf_nf2_r18(a, block, s) : launch_dslash_pdf_nf2_r12(a, block, s);
}
static cudaError_t launch_dslash_multi_pdf(const DslashArgs<df64> &a, int nf, int recon, const int *act, int nact,
                                           int nrhs, cudaStream_t s)
{
    if (nf == 1)
        return recon == 18 ? launch_dslash_multi_pdf_nf1_r18(a, act, nact, nrhs, s)
                           : launch_dslash_multi_pdf_nf1_r12(a, act, nact, nrhs, s);
    return recon == 18 ? launch_dslash_multi_pdf_nf2_r18(a, act, nact, nrhs, s)
                       : launch_dslash_multi_pdf_nf2_r12(a, act, nact, nrhs, s);
}
cudaError_t launch_dslash_multi_p64(const DslashArgs<double> &a, int nf, int recon, bool pro, const int *act, int nact,
                                    int nrhs, int rpb, cudaStream_t s);
cudaError_t launch_dslash_multi_p32(const DslashArgs<float> &a, int nf, int recon, bool pro, const int *act, int nact,
                                    int nrhs, int rpb, cudaStream_t s);
cudaError_t launch_dslash_multi_p16(const DslashArgs<float> &a, int nf, int recon, bool pro, const int *act, int nact,
                                    int nrhs, int rpb, cudaStream_t s);
cudaError_t launch_pack_spinor(const tm_gauge *g, const tm_field *f, const void *canon, int ctype, int parity,
                               cudaStream_t s);
cudaError_t launch_unpack_spinor(const tm_gauge *g, void *canon, int ctype, const tm_field *f, int parity,
                                 cudaStream_t s);
cudaError_t launch_pack_gauge(const tm_gauge *g, int pidx, void *out, const void *canon, cudaStream_t s);
cudaError_t launch_noise_z2(const tm_gauge *g, const tm_field *f, int parity, unsigned long long seed, cudaStream_t s);
cudaError_t launch_twist(const tm_gauge *g, const tm_field *out, const tm_field *in, const Twist<double> &tw,
                         cudaStream_t s);
cudaError_t launch_twist_active(const tm_gauge *g, const tm_field *out, const tm_field *in, const Twist<double> &tw,
                                const int *act, int nact, cudaStream_t s);
cudaError_t launch_dslash_clov_p64(const DslashArgs<double> &a, int nf, int recon, int minb, cudaStream_t s);
cudaError_t launch_fused_p64(const DslashArgs<double> &aA, const DslashArgs<double> &aB, int nf, int recon,
                             const int *items, int nitems, int *sync, unsigned long long limit_ns, int num_sms,
                             cudaStream_t s);
cudaError_t launch_fused_p32(const DslashArgs<float> &aA, const DslashArgs<float> &aB, int nf, int recon,
                             const int *items, int nitems, int *sync, unsigned long long limit_ns, int num_sms,
                             cudaStream_t s);
cudaError_t launch_dslash_clov_p32(const DslashArgs<float> &a, int nf, int recon, int minb, cudaStream_t s);
cudaError_t launch_dslash_clov_p16(const DslashArgs<float> &a, int nf, int recon, int minb, cudaStream_t s);
cudaError_t launch_clover_apply(const tm_gauge *g, const tm_field *out, const tm_field *in, int parity, bool inverse,
                                const Twist<double> &X, cudaStream_t s);

cudaError_t launch_dd_p64(const DslashArgs<double> &a, const DDArgs<double> *dd, void *face_prev, void *face_next,
                          int nf, int recon, bool pro, cudaStream_t s);
cudaError_t launch_dd_p32(const DslashArgs<float> &a, const DDArgs<float> *dd, void *face_prev, void *face_next,
                          int nf, int recon, bool pro, cudaStream_t s);
cudaError_t launch_dd_p16(const DslashArgs<float> &a, const DDArgs<float> *dd, void *face_prev, void *face_next,
                          int nf, int recon, bool pro, cudaStream_t s);
size_t dd_face_bytes(int prec, int nf, int st);
cudaError_t launch_dslash_red_p64(const DslashArgs<double> &a, int nf, int recon, int variant, const RedArgs &red,
                                  cudaStream_t s);
cudaError_t launch_dslash_red_p32(const DslashArgs<float> &a, int nf, int recon, int variant, const RedArgs &red,
                                  cudaStream_t s);
cudaError_t launch_dslash_red_p16(const DslashArgs<float> &a, int nf, int recon, int variant, const RedArgs &red,
                                  cudaStream_t s);

static thread_local char g_err[512];
constexpr int TM_MAX_RHS_API = 64;

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

tm_status cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return TM_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return TM_ERR_CUDA;
}

int prec_index(int prec)
{
    switch (prec) {
    case TM_PREC_F64: return 0;
    case TM_PREC_F32: return 1;
    case TM_PREC_F16: return 2;
    case TM_PREC_DF64: return 3;
    default: return -1;
    }
}

size_t real_bytes(int prec) { return prec == TM_PREC_DF64 ? 8 : (size_t)prec; }

int spinor_chunks(int prec) { return (prec == TM_PREC_F64 || prec == TM_PREC_DF64) ? 12 : (prec == TM_PREC_F32 ? 6 : 3); }
size_t chunk_bytes(int) { return 16; }

static int link_reals_per_chunk(int prec, int recon)
{
    // chunk geometry of LinkLayout<PREC, RECON> in tm_core.cuh
    if (prec == TM_PREC_F64 || prec == TM_PREC_DF64) return 2;
    if (prec == TM_PREC_F32) return recon == 18 ? 2 : 4;
    return recon == 18 ? 2 : (recon == 12 ? 4 : 8);
}
static size_t link_chunk_bytes(int prec, int recon) { return (size_t)link_reals_per_chunk(prec, recon) * real_bytes(prec); }

// ---------------------------------------------------------------------------- twist tables
// R = 1 + i a gamma5 tau3 + b tau1 (doublet) or 1 + i a s gamma5 (one flavour, s = +-1), with
// a = 2 kappa mu, b = 2 kappa eps; gamma5 = +1 on spins 0,1 and -1 on spins 2,3.
//   R^-1 = (1 - i a gamma5 tau3 - b tau1) / (1 + a^2 - b^2)   (doublet; X^2 = b^2 - a^2)
//   R^-1 = (1 - i a s gamma5) / (1 + a^2)                      (one flavour)
// R^dag = R(a -> -a); R^-dag = R^-1(a -> -a).
static Twist<double> make_twist(const tm_gauge *g, int kind, int dagger)
{
    Twist<double> t;
    memset(&t, 0, sizeof(t));
    double a = 2.0 * g->p.kappa * g->p.mu;
    const double b = 2.0 * g->p.kappa * g->p.epsilon;
    if (dagger) a = -a;
    for (int gi = 0; gi < 2; gi++) {
        const double g5 = gi == 0 ? 1.0 : -1.0;
        if (g->nf == 2) {
            if (kind == TW_R) {
                t.m[gi][0][0] = {1.0, a * g5};
                t.m[gi][1][1] = {1.0, -a * g5};
                t.m[gi][0][1] = t.m[gi][1][0] = {b, 0.0};
            } else {
                const double d = 1.0 / (1.0 + a * a - b * b);
                t.m[gi][0][0] = {d, -a * g5 * d};
                t.m[gi][1][1] = {d, a * g5 * d};
                t.m[gi][0][1] = t.m[gi][1][0] = {-b * d, 0.0};
            }
        } else {
            const double s = (double)g->p.flavor;
            if (kind == TW_R) {
                t.m[gi][0][0] = {1.0, a * s * g5};
            } else {
                const double d = 1.0 / (1.0 + a * a);
                t.m[gi][0][0] = {d, -a * s * g5 * d};
            }
        }
    }
    return t;
}

// X = R - 1 (R^dag - 1 for the adjoint): the part of the local operator that a clover handle
// adds to its per-site C = 1 + T
static Twist<double> clover_x(const tm_gauge *g, int dagger)
{
    Twist<double> t = make_twist(g, TW_R, dagger);
    for (int gi = 0; gi < 2; gi++)
        for (int f = 0; f < 2; f++) t.m[gi][f][f].r -= 1.0;
    return t;
}

static Twist<df64> to_df64(const Twist<double> &t)
{
    Twist<df64> f;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            for (int k = 0; k < 2; k++) f.m[i][j][k] = {df64(t.m[i][j][k].r), df64(t.m[i][j][k].i)};
    return f;
}

static Twist<float> to_float(const Twist<double> &t)
{
    Twist<float> f;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            for (int k = 0; k < 2; k++) f.m[i][j][k] = {(float)t.m[i][j][k].r, (float)t.m[i][j][k].i};
    return f;
}

// ----------------------------------------------------------------------------- validation
// A canonical (user-layout) buffer may be device memory, managed memory, or pinned host memory;
// pinned host memory is accessed in place by the kernels through its device mapping (on GB300
// over the coherent CPU-GPU link), so a host-resident field is read or written without a
// staging copy.  Pageable host memory is rejected instead of faulting.
static tm_status resolve_canon(const void *p, void **dev_out, const char *what)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("%s: cannot query the canonical buffer (%s)", what, cudaGetErrorString(e));
        return TM_ERR_ARG;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        *dev_out = const_cast<void *>(p);
        return TM_OK;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        *dev_out = at.devicePointer;
        return TM_OK;
    }
    set_error("%s: the canonical buffer must be device, managed or pinned host memory", what);
    return TM_ERR_ARG;
}

static tm_status check_field(const tm_gauge *g, const tm_field *f, const char *name)
{
    if (!f) { set_error("%s: null tm_field", name); return TM_ERR_ARG; }
    if (prec_index(f->prec) < 0) { set_error("%s: unknown precision %d", name, f->prec); return TM_ERR_ARG; }
    if (!f->data) { set_error("%s: null data pointer", name); return TM_ERR_ARG; }
    if (f->prec == TM_PREC_F16 && !f->norm) { set_error("%s: FP16 field needs a norm array", name); return TM_ERR_ARG; }
    if (f->nrhs < 1) { set_error("%s: nrhs must be >= 1", name); return TM_ERR_ARG; }
    if (((uintptr_t)f->data & 15) != 0) { set_error("%s: data must be 16-byte aligned", name); return TM_ERR_ARG; }
    (void)g;
    return TM_OK;
}

static tm_status check_params(const tm_params *p)
{
    if (!p) { set_error("null tm_params"); return TM_ERR_ARG; }
    long V = 1;
    for (int m = 0; m < 4; m++) {
        if (p->L[m] < 2 || (p->L[m] & 1)) {
            set_error("L[%d] = %d: every extent must be even and >= 2", m, p->L[m]);
            return TM_ERR_ARG;
        }
        V *= p->L[m];
    }
    if (V / 2 > (long)(0x7fffffff / 24)) { set_error("lattice too large for 32-bit site indexing"); return TM_ERR_ARG; }
    if (p->flavor != TM_TWIST_PLUS && p->flavor != TM_TWIST_MINUS && p->flavor != TM_NDEG_DOUBLET) {
        set_error("unknown flavor %d", p->flavor);
        return TM_ERR_ARG;
    }
    if (p->flavor != TM_NDEG_DOUBLET && p->epsilon != 0.0) {
        set_error("epsilon must be 0 for a single flavour");
        return TM_ERR_ARG;
    }
    if (p->recon != 18 && p->recon != 12 && p->recon != 8) { set_error("recon must be 18, 12 or 8"); return TM_ERR_ARG; }
    if (!(p->kappa > 0.0) || !isfinite(p->kappa) || !isfinite(p->mu) || !isfinite(p->epsilon)) {
        set_error("kappa must be positive; kappa, mu, epsilon finite");
        return TM_ERR_ARG;
    }
    const double a = 2 * p->kappa * p->mu, b = 2 * p->kappa * p->epsilon;
    if (1.0 + a * a - b * b <= 1e-12) {
        set_error("twist R is singular or indefinite: 1 + (2 kappa mu)^2 - (2 kappa eps)^2 = %g", 1.0 + a * a - b * b);
        return TM_ERR_ARG;
    }
    return TM_OK;
}

// A handle made with tm_gauge_create_ex packs only the link precisions of its mask.
tm_status need_links(const tm_gauge *g, int prec)
{
    const int pidx = prec_index(prec);
    if (pidx < 0 || !g->links[pidx]) {
        set_error("the handle holds no links for storage precision %d (tm_gauge_create_ex mask)", prec);
        return TM_ERR_ARG;
    }
    return TM_OK;
}

// ------------------------------------------------------------------------------- dslash core
template <typename T>
static void fill_common(DslashArgs<T> &a, const tm_gauge *g, const tm_field *out, const tm_field *in,
                        const tm_field *x, int out_parity, int pidx)
{
    a.out = out->data;
    a.out_norm = out->norm;
    a.in = in->data;
    a.in_norm = in->norm;
    a.x = x ? x->data : nullptr;
    a.x_norm = x ? x->norm : nullptr;
    a.gauge = g->links[pidx];
    a.Vh = g->Vh;
    a.cb0 = 0;
    a.ncb = g->Vh;
    a.X1h = g->X1h;
    a.Lx = g->p.L[0];
    a.Ly = g->p.L[1];
    a.Lz = g->p.L[2];
    a.Lt = g->p.L[3];
    a.out_parity = out_parity;
    a.tbc = g->p.t_antiperiodic ? 1 : 0;
    a.clov = pidx < 3 ? g->clov[pidx] : nullptr;
    a.clov_norm = g->clov_norm;
}

// Generic fused hopping launch: out = epi(H or H^dag (pro(in))).  With nact > 1 (or a list act of
// right-hand-side indices) the multi-RHS kernel processes those right-hand sides of the fields.
tm_status dslash_launch(const tm_gauge *g, const tm_field *out, const tm_field *in, const tm_field *x, int out_parity,
                        int dagger, int epi, double coef, const Twist<double> *tw_epi, const Twist<double> *tw_pro,
                        cudaStream_t s, const int *act, int nact, int cb0 = 0, int ncb = 0,
                        const Twist<double> *tw_acc = nullptr)
{
    const int pidx = prec_index(in->prec);
    if (need_links(g, in->prec) != TM_OK) return TM_ERR_ARG;
    const bool pro = tw_pro != nullptr;
    Twist<double> z;
    memset(&z, 0, sizeof(z));
    const Twist<double> &te = tw_epi ? *tw_epi : z, &tp = tw_pro ? *tw_pro : z, &ta = tw_acc ? *tw_acc : z;
    const tm_tune_entry tu = g->tune[pidx][pro ? 1 : 0];
    const bool multi = act != nullptr || nact > 1;
    cudaError_t e;
    if (g->csw != 0.0) {
        // clover handle: the per-site local operator in the epilogue (tw_epi only marks that an
        // epilogue applies it; the kernel uses X = R - 1 and the site's clover blocks)
        if (pidx == 3) { set_error("clover handles have no DF64 form"); return TM_ERR_ARG; }
        if (multi) { set_error("clover handles take single-RHS fields (nrhs = 1)"); return TM_ERR_ARG; }
        if (pro) { set_error("internal: no input prologue with a clover term"); return TM_ERR_ARG; }
        const Twist<double> X = clover_x(g, dagger);
        if (pidx == 0) {
            DslashArgs<double> a;
            fill_common(a, g, out, in, x, out_parity, pidx);
            a.epilogue = epi;
            a.sigma = dagger ? -1.0 : 1.0;
            a.coef = coef;
            a.tw_epi = X;
            a.tw_pro = X;
            e = launch_dslash_clov_p64(a, g->nf, link_recon(g, 0), g->clov_minb[0], s);
        } else {
            DslashArgs<float> a;
            fill_common(a, g, out, in, x, out_parity, pidx);
            a.epilogue = epi;
            a.sigma = dagger ? -1.0f : 1.0f;
            a.coef = (float)coef;
            a.tw_epi = to_float(X);
            a.tw_pro = a.tw_epi;
            e = pidx == 1 ? launch_dslash_clov_p32(a, g->nf, link_recon(g, pidx), g->clov_minb[1], s)
                           : launch_dslash_clov_p16(a, g->nf, link_recon(g, pidx), g->clov_minb[2], s);
        }
        return cuda_check(e, "clover dslash launch");
    }
    if (ncb > 0 && (multi || pidx == 3)) { set_error("internal: site ranges are single-RHS FP64 / FP32 / FP16"); return TM_ERR_ARG; }
    // Paired sources (multi-RHS tune entry 16, one flavour): every right-hand side of an even count,
    // two sources at a time through the doublet's kernels -- a one-flavour field with 2k sources has
    // the layout of a doublet field with k -- with the one-flavour local operator on both
    // "flavours"; the doublet's staged form pairs the two sources in its packed FMAs.
    if (multi && act == nullptr && g->nf == 1 && pidx <= 2 && (g->multi_rpb[pidx] == 16 || g->multi_rpb[pidx] == 36) &&
        (nact & 1) == 0 && nact == out->nrhs) {
        const int form = g->multi_rpb[pidx] == 36 ? 34 : 14;
        auto diag = [](const Twist<double> &t) {
            Twist<double> d = t;
            for (int gi = 0; gi < 2; gi++) {
                d.m[gi][1][1] = t.m[gi][0][0];
                d.m[gi][0][1] = d.m[gi][1][0] = {0.0, 0.0};
            }
            return d;
        };
        const Twist<double> de = diag(te), dp = diag(tp), da = diag(ta);
        if (pidx == 0) {
            DslashArgs<double> a;
            fill_common(a, g, out, in, x, out_parity, pidx);
            a.epilogue = epi;
            a.sigma = dagger ? -1.0 : 1.0;
            a.coef = coef;
            a.tw_epi = de;
            a.tw_pro = dp;
            a.tw_acc = da;
            e = launch_dslash_multi_p64(a, 2, link_recon(g, 0), pro, nullptr, nact / 2, nact / 2, form, s);
        } else {
            DslashArgs<float> a;
            fill_common(a, g, out, in, x, out_parity, pidx);
            a.epilogue = epi;
            a.sigma = dagger ? -1.0f : 1.0f;
            a.coef = (float)coef;
            a.tw_epi = to_float(de);
            a.tw_pro = to_float(dp);
            a.tw_acc = to_float(da);
            e = pidx == 1 ? launch_dslash_multi_p32(a, 2, link_recon(g, pidx), pro, nullptr, nact / 2, nact / 2, form, s)
                          : launch_dslash_multi_p16(a, 2, link_recon(g, pidx), pro, nullptr, nact / 2, nact / 2, form, s);
        }
        return cuda_check(e, "dslash launch (paired sources)");
    }
    if (pidx == 0) {
        DslashArgs<double> a;
        fill_common(a, g, out, in, x, out_parity, pidx);
        if (ncb > 0) { a.cb0 = cb0; a.ncb = ncb; }
        a.epilogue = epi;
        a.sigma = dagger ? -1.0 : 1.0;
        a.coef = coef;
        a.tw_epi = te;
        a.tw_pro = tp;
        a.tw_acc = ta;
        e = multi ? launch_dslash_multi_p64(a, g->nf, link_recon(g, 0), pro, act, nact, out->nrhs, g->multi_rpb[0], s)
                  : launch_dslash_p64(a, g->nf, link_recon(g, 0), pro, tu.variant, tu.block, s);
    } else if (pidx == 3) {
        DslashArgs<df64> a;
        fill_common(a, g, out, in, x, out_parity, pidx);
        a.epilogue = epi;
        a.sigma = df64(dagger ? -1.0 : 1.0);
        a.coef = df64(coef);
        a.tw_epi = to_df64(te);
        a.tw_pro = to_df64(tp);
        a.tw_acc = to_df64(ta);
        const int r = link_recon(g, 3);
        if (pro) {
            set_error("DF64 has no input-twist prologue kernel (the operators apply that twist separately)");
            return TM_ERR_ARG;
        }
        e = multi ? launch_dslash_multi_pdf(a, g->nf, r, act, nact, out->nrhs, s)
                  : launch_dslash_pdf(a, g->nf, r, 64, s);
    } else {
        DslashArgs<float> a;
        fill_common(a, g, out, in, x, out_parity, pidx);
        if (ncb > 0) { a.cb0 = cb0; a.ncb = ncb; }
        a.epilogue = epi;
        a.sigma = dagger ? -1.0f : 1.0f;
        a.coef = (float)coef;
        a.tw_epi = to_float(te);
        a.tw_pro = to_float(tp);
        a.tw_acc = to_float(ta);
        if (multi)
            e = (pidx == 1) ? launch_dslash_multi_p32(a, g->nf, link_recon(g, pidx), pro, act, nact, out->nrhs, g->multi_rpb[1], s)
                            : launch_dslash_multi_p16(a, g->nf, link_recon(g, pidx), pro, act, nact, out->nrhs, g->multi_rpb[2], s);
        else
            e = (pidx == 1) ? launch_dslash_p32(a, g->nf, link_recon(g, pidx), pro, tu.variant, tu.block, s)
                            : launch_dslash_p16(a, g->nf, link_recon(g, pidx), pro, tu.variant, tu.block, s);
    }
    return cuda_check(e, "dslash launch");
}

static tm_status dslash_launch(const tm_gauge *g, const tm_field *out, const tm_field *in, const tm_field *x,
                               int out_parity, int dagger, int epi, double coef, const Twist<double> *tw_epi,
                               const Twist<double> *tw_pro, cudaStream_t s)
{
    // every right-hand side of the fields (nrhs = 1: the single-RHS kernels)
    return dslash_launch(g, out, in, x, out_parity, dagger, epi, coef, tw_epi, tw_pro, s, nullptr, out->nrhs);
}

static tm_status same_prec(const tm_field *a, const tm_field *b, const char *what)
{
    if (a->prec != b->prec) { set_error("%s: fields must share a precision", what); return TM_ERR_ARG; }
    if (a->nrhs != b->nrhs) { set_error("%s: fields must share nrhs", what); return TM_ERR_ARG; }
    return TM_OK;
}

static tm_status refuse_slab(const tm_gauge *g, const char *what)
{
    if (g && g->dd) {
        set_error("%s: the handle holds one time slab of a decomposed lattice; its hops need the neighbours' faces "
                  "(tm_dd_pack_faces / tm_dd_dslash)", what);
        return TM_ERR_ARG;
    }
    return TM_OK;
}

#define TM_TRY(x)                     \
    do {                              \
        tm_status _st = (x);          \
        if (_st != TM_OK) return _st; \
    } while (0)

static tm_status dslash_api(const tm_gauge *g, const tm_field *out, const tm_field *in, int out_parity, int epilogue,
                            const tm_field *x, void *stream, int dagger)
{
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(refuse_slab(g, "tm_dslash"));
    TM_TRY(check_field(g, out, "out"));
    TM_TRY(check_field(g, in, "in"));
    TM_TRY(same_prec(out, in, "tm_dslash"));
    if (out_parity != 0 && out_parity != 1) { set_error("out_parity must be 0 or 1"); return TM_ERR_ARG; }
    if (out->data == in->data) { set_error("tm_dslash: out must not alias in"); return TM_ERR_ARG; }
    const double k = g->p.kappa;
    const Twist<double> R = make_twist(g, TW_R, dagger), Ri = make_twist(g, TW_RINV, dagger);
    const bool needx = epilogue >= TM_EPI_TWXPAY_ASYM;
    if (epilogue < TM_EPI_NONE || epilogue > TM_EPI_XMAY_K2) { set_error("unknown epilogue %d", epilogue); return TM_ERR_ARG; }
    if (needx) {
        TM_TRY(check_field(g, x, "x"));
        TM_TRY(same_prec(out, x, "tm_dslash"));
    }
    cudaStream_t s = (cudaStream_t)stream;
    switch (epilogue) {
    case TM_EPI_NONE: return dslash_launch(g, out, in, nullptr, out_parity, dagger, EPI_SCALE, 1.0, nullptr, nullptr, s);
    case TM_EPI_TWINV: return dslash_launch(g, out, in, nullptr, out_parity, dagger, EPI_TW, 1.0, &Ri, nullptr, s);
    case TM_EPI_TWXPAY_ASYM: return dslash_launch(g, out, in, x, out_parity, dagger, EPI_TWX_AXPY, -k * k, &R, nullptr, s);
    case TM_EPI_TWXPAY_SYM: return dslash_launch(g, out, in, x, out_parity, dagger, EPI_X_TWAXPY, -k * k, &Ri, nullptr, s);
    case TM_EPI_XPAY: return dslash_launch(g, out, in, x, out_parity, dagger, EPI_XPAY, k, nullptr, nullptr, s);
    case TM_EPI_XMAY_K2: return dslash_launch(g, out, in, x, out_parity, dagger, EPI_XPAY, -k * k, nullptr, nullptr, s);
    default: return dslash_launch(g, out, in, x, out_parity, dagger, EPI_TW_XPAY, k, &Ri, nullptr, s);
    }
}

// Work list of the fused operator (k_mpc_fused): items (tile << 1) | pass, pass 0 = A (odd
// output), 1 = B (even output).  A site's neighbours lie within one time slice (st sites) of it,
// or across the periodic wrap in the last / first slice, so: the A tiles touching the last time
// slice first, then A tiles from 0 up, with each B tile emitted after the A tiles one slice and
// a resident wave of tiles beyond it.  Every B tile then depends only on A tiles earlier in the
// list.
static std::vector<int> fused_items(const int L[4], int num_sms)
{
    // in work items of FUSED_GROUP tiles of 128 sites
    const long Vh = (long)L[0] * L[1] * L[2] * L[3] / 2, st = (long)(L[0] / 2) * L[1] * L[2];
    const long gs = 128L * FUSED_GROUP;
    const int N = (int)((Vh + gs - 1) / gs);
    const int P = (int)((st + gs - 1) / gs) + 1;
    const int first = (int)(Vh - st > 0 ? (Vh - st) / gs : 0);  // A groups [first, N) touch the last slice
    std::vector<int> items;
    items.reserve(2 * (size_t)N);
    for (int t = first; t < N; t++) items.push_back(t << 1);
    int nextA = 0;
    // A runs ahead of B by one time slice plus the blocks in flight (up to 4 per SM), so the groups a
    // B group reads have normally finished before it is claimed
    const int W = P + 3 + (4 * (num_sms > 0 ? num_sms : 152) + FUSED_GROUP - 1) / FUSED_GROUP;
    while (nextA < first && nextA < W) items.push_back((nextA++) << 1);
    for (int i = 0; i < N; i++) {
        items.push_back((i << 1) | 1);
        if (nextA < first) items.push_back((nextA++) << 1);
    }
    return items;
}

// flags per 128-site tile of the fused operator, rounded up to whole groups
static size_t fused_nflags(long Vh) { return (size_t)((Vh + 128L * FUSED_GROUP - 1) / (128L * FUSED_GROUP)) * FUSED_GROUP; }

tm_status build_fused_work(tm_gauge *g, cudaStream_t s)
{
    const std::vector<int> items = fused_items(g->p.L, g->num_sms);
    g->fused_nitems = (int)items.size();
    g->fused_capacity = (int)items.size();
    g->wait_limit_ns = 1000000000ull;  // one second per bounded wait
    const size_t nflags = fused_nflags(g->Vh);
    if (cudaMalloc((void **)&g->fused_items, sizeof(int) * items.size()) != cudaSuccess ||
        cudaMalloc((void **)&g->fused_sync, sizeof(int) * (3 + nflags)) != cudaSuccess) {
        cudaGetLastError();
        set_error("tm_gauge_create: work list allocation failed");
        return TM_ERR_NOMEM;
    }
    TM_TRY(cuda_check(cudaMemcpyAsync(g->fused_items, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice, s),
                      "work list copy"));
    TM_TRY(cuda_check(cudaMemsetAsync(g->fused_sync, 0, sizeof(int) * (3 + nflags), s), "work list memset"));
    return cuda_check(cudaStreamSynchronize(s), "work list");
}

template <typename T>
static DslashArgs<T> pass_args(const tm_gauge *g, const tm_field *out, const tm_field *in, const tm_field *x,
                               int out_parity, int dagger, int epi, double coef, const Twist<T> &tw, int pidx)
{
    DslashArgs<T> a;
    memset(&a, 0, sizeof(a));
    fill_common(a, g, out, in, x, out_parity, pidx);
    a.epilogue = epi;
    a.sigma = dagger ? T(-1) : T(1);
    a.coef = (T)coef;
    a.tw_epi = tw;
    a.tw_pro = tw;
    return a;
}

// M_pc as one fused launch (FP64 / FP32, no clover, one right-hand side, not the adjoint of the
// symmetric operator): A = (tmp <- Ti_oo H_oe in), B = (out <- epilogue of H_eo tmp)
static tm_status fused_launch(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o,
                              int pc, int dagger, cudaStream_t s)
{
    const double k2 = g->p.kappa * g->p.kappa;
    const Twist<double> R = make_twist(g, TW_R, dagger), Ri = make_twist(g, TW_RINV, dagger);
    const int epiB = pc == TM_PC_ASYM ? EPI_TWX_AXPY : EPI_X_TWAXPY;
    const Twist<double> &twB = pc == TM_PC_ASYM ? R : Ri;
    // work counter, abort word and tile flags start at zero; the error word is kept until read
    TM_TRY(cuda_check(cudaMemsetAsync(g->fused_sync + 1, 0, sizeof(int) * (2 + fused_nflags(g->Vh)), s), "fused reset"));
    cudaError_t e;
    if (out_e->prec == TM_PREC_F64) {
        const DslashArgs<double> aA = pass_args<double>(g, tmp_o, in_e, nullptr, 1, dagger, EPI_TW, 1.0, Ri, 0);
        const DslashArgs<double> aB = pass_args<double>(g, out_e, tmp_o, in_e, 0, dagger, epiB, -k2, twB, 0);
        e = launch_fused_p64(aA, aB, g->nf, link_recon(g, 0), g->fused_items, g->fused_nitems, g->fused_sync, g->wait_limit_ns,
                             g->num_sms, s);
    } else {
        const DslashArgs<float> aA = pass_args<float>(g, tmp_o, in_e, nullptr, 1, dagger, EPI_TW, 1.0, to_float(Ri), 1);
        const DslashArgs<float> aB = pass_args<float>(g, out_e, tmp_o, in_e, 0, dagger, epiB, -k2, to_float(twB), 1);
        e = launch_fused_p32(aA, aB, g->nf, link_recon(g, 1), g->fused_items, g->fused_nitems, g->fused_sync, g->wait_limit_ns,
                             g->num_sms, s);
    }
    return cuda_check(e, "fused operator launch");
}

tm_status precond_core(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o, int pc,
                       int dagger, cudaStream_t s, const int *act, int nact)
{
    {
        const int pidx = prec_index(out_e->prec);
        if ((pidx == 0 || pidx == 1) && g->fused[pidx] && g->csw == 0.0 && act == nullptr && nact <= 1 &&
            out_e->nrhs == 1 && !(pc == TM_PC_SYM && dagger) && g->fused_sync && g->links[pidx])
            return fused_launch(g, out_e, in_e, tmp_o, pc, dagger, s);
    }
    const double k2 = g->p.kappa * g->p.kappa;
    const Twist<double> R = make_twist(g, TW_R, dagger), Ri = make_twist(g, TW_RINV, dagger);
    if (g->csw != 0.0 && (out_e->prec == TM_PREC_DF64 || act != nullptr || nact > 1)) {
        set_error("clover handles take single-RHS FP64 / FP32 / FP16 fields");
        return TM_ERR_ARG;
    }
    if (pc == TM_PC_ASYM) {
        // tmp = R^-1_oo H_oe in ;  out = R_ee in - kappa^2 H_eo tmp
        TM_TRY(dslash_launch(g, tmp_o, in_e, nullptr, 1, dagger, EPI_TW, 1.0, &Ri, nullptr, s, act, nact));
        return dslash_launch(g, out_e, tmp_o, in_e, 0, dagger, EPI_TWX_AXPY, -k2, &R, nullptr, s, act, nact);
    }
    if (!dagger) {
        // tmp = R^-1_oo H_oe in ;  out = in - kappa^2 R^-1_ee H_eo tmp
        TM_TRY(dslash_launch(g, tmp_o, in_e, nullptr, 1, 0, EPI_TW, 1.0, &Ri, nullptr, s, act, nact));
        return dslash_launch(g, out_e, tmp_o, in_e, 0, 0, EPI_X_TWAXPY, -k2, &Ri, nullptr, s, act, nact);
    }
    // adjoint of the symmetric operator: tmp = R^-dag_oo H^dag_oe R^-dag_ee in ; out = in - kappa^2 H^dag_eo tmp
    if (g->csw != 0.0) {
        // clover: L^-dag_ee as a pass into out_e (overwritten by the last launch)
        TM_TRY(cuda_check(launch_clover_apply(g, out_e, in_e, 0, true, clover_x(g, 1), s), "clover apply"));
        TM_TRY(dslash_launch(g, tmp_o, out_e, nullptr, 1, 1, EPI_TW, 1.0, &Ri, nullptr, s, act, nact));
        return dslash_launch(g, out_e, tmp_o, in_e, 0, 1, EPI_XPAY, -k2, nullptr, nullptr, s, act, nact);
    }
    if (out_e->prec == TM_PREC_DF64 || (out_e->prec == TM_PREC_F16 && g->nf == 2)) {
        // DF64, and the FP16 doublet: the input twist as its own launch into out_e (overwritten by
        // the last launch).  The FP16 doublet kernel is bound by the FMA pipe, and the prologue
        // would apply the flavour-mixing twist to all eight neighbours of every site; one
        // elementwise pass costs less (its one extra binary16 rounding of R^-dag in stays inside
        // the FP16 tolerance).
        TM_TRY(cuda_check(launch_twist_active(g, out_e, in_e, Ri, act, nact, s), "twist"));
        TM_TRY(dslash_launch(g, tmp_o, out_e, nullptr, 1, 1, EPI_TW, 1.0, &Ri, nullptr, s, act, nact));
        return dslash_launch(g, out_e, tmp_o, in_e, 0, 1, EPI_XPAY, -k2, nullptr, nullptr, s, act, nact);
    }
    TM_TRY(dslash_launch(g, tmp_o, in_e, nullptr, 1, 1, EPI_TW, 1.0, &Ri, &Ri, s, act, nact));
    return dslash_launch(g, out_e, tmp_o, in_e, 0, 1, EPI_XPAY, -k2, nullptr, nullptr, s, act, nact);
}

// Q = (R R^dag)^-1 per gamma5 block: a flavour matrix for the doublet,
// (1 + a^2 + b^2) + 2 b tau1 - 2 a b gamma5 tau2 inverted; a real number 1 / (1 + a^2) for one flavour
static Twist<double> rrdag_inverse(const tm_gauge *g)
{
    const Twist<double> R = make_twist(g, TW_R, 0);
    Twist<double> Q;
    memset(&Q, 0, sizeof(Q));
    for (int gi = 0; gi < 2; gi++) {
        const int n = g->nf;
        C<double> P[2][2] = {};
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                for (int k = 0; k < n; k++) {  // P = R R^dag
                    const C<double> r = R.m[gi][i][k], rc = {R.m[gi][j][k].r, -R.m[gi][j][k].i};
                    P[i][j].r += r.r * rc.r - r.i * rc.i;
                    P[i][j].i += r.r * rc.i + r.i * rc.r;
                }
        if (n == 1) {
            Q.m[gi][0][0] = {1.0 / P[0][0].r, 0.0};  // R R^dag = |r|^2 is real
        } else {
            const C<double> det = {P[0][0].r * P[1][1].r - P[0][0].i * P[1][1].i - (P[0][1].r * P[1][0].r - P[0][1].i * P[1][0].i),
                                   P[0][0].r * P[1][1].i + P[0][0].i * P[1][1].r - (P[0][1].r * P[1][0].i + P[0][1].i * P[1][0].r)};
            const double d2 = det.r * det.r + det.i * det.i;
            const C<double> inv = {det.r / d2, -det.i / d2};
            auto mul = [&](C<double> a, double sgn) { return C<double>{sgn * (a.r * inv.r - a.i * inv.i), sgn * (a.r * inv.i + a.i * inv.r)}; };
            Q.m[gi][0][0] = mul(P[1][1], 1.0);
            Q.m[gi][1][1] = mul(P[0][0], 1.0);
            Q.m[gi][0][1] = mul(P[0][1], -1.0);
            Q.m[gi][1][0] = mul(P[1][0], -1.0);
        }
    }
    return Q;
}

// Whether normal_core can fuse |A in|^2 into the epilogue of its second launch: single-RHS FP64 /
// FP32 / FP16 fields, no clover term, A = M_pc (no dagger), the handle's no-prologue launch form a
// staged one (variants 6 - 9), and room for one partial sum per block in the reduction scratch.
bool normal_red_supported(const tm_gauge *g, int prec, int dagger)
{
    const int pidx = prec_index(prec);
    if (pidx < 0 || pidx > 2 || dagger || g->csw != 0.0 || g->dd || !g->links[pidx]) return false;
    const int v = g->tune[pidx][0].variant;
    const size_t blocks = (size_t)(g->Vh + 127) / 128;  // four partial sums (warps) per block
    return v >= 6 && v <= 9 && 4 * blocks * sizeof(double) <= g->scratch_bytes - SCRATCH_PARTIALS_OFF;
}

// One staged launch with the fused reduction (red) and its fixed-order finish.
static tm_status red_launch(const tm_gauge *g, const tm_field *out, const tm_field *in, const tm_field *x, int dagger,
                            int epi, double coef, const Twist<double> &tw, const Twist<double> *q, const double *scal,
                            const RedArgs *red, cudaStream_t s)
{
    const int pidx = prec_index(in->prec);
    const int variant = g->tune[pidx][0].variant;
    cudaError_t e;
    if (pidx == 0) {
        DslashArgs<double> a = pass_args<double>(g, out, in, x, 0, dagger, epi, coef, tw, 0);
        if (q) a.tw_acc = *q;
        a.scal_in = scal;
        e = launch_dslash_red_p64(a, g->nf, link_recon(g, 0), variant, *red, s);
    } else {
        DslashArgs<float> a = pass_args<float>(g, out, in, x, 0, dagger, epi, coef, to_float(tw), pidx);
        if (q) a.tw_acc = to_float(*q);
        a.scal_in = scal;
        e = pidx == 1 ? launch_dslash_red_p32(a, g->nf, link_recon(g, pidx), variant, *red, s)
                      : launch_dslash_red_p16(a, g->nf, link_recon(g, pidx), variant, *red, s);
    }
    TM_TRY(cuda_check(e, "fused-reduction launch"));
    return cuda_check(launch_finish_partials(red->partials, 4L * ((g->Vh + 127) / 128), *red, s), "reduction finish");
}

// The first half of the normal operator with |A in|^2 = <in, A^dag A in> (CG's <p, A^dag A p>) from
// the epilogue of its second launch: te = M_asym in and |te|^2 for the asymmetric operator; for the
// symmetric one te = Q u with u = M_asym in and Q = (R R^dag)^-1, and the reduction Re<u, Q u>,
// since M_sym = R^-1 M_asym.
static tm_status normal_first_half_red(const tm_gauge *g, const tm_field *te_e, const tm_field *in_e,
                                       const tm_field *tmp_o, int pc, cudaStream_t s, const RedArgs *red)
{
    if (!normal_red_supported(g, in_e->prec, 0) || in_e->nrhs != 1) {
        set_error("internal: fused reduction not available for this operator");
        return TM_ERR_ARG;
    }
    const double k2 = g->p.kappa * g->p.kappa;
    const Twist<double> R = make_twist(g, TW_R, 0), Ri = make_twist(g, TW_RINV, 0), Q = rrdag_inverse(g);
    const bool sym = pc == TM_PC_SYM;
    TM_TRY(dslash_launch(g, tmp_o, in_e, nullptr, 1, 0, EPI_TW, 1.0, &Ri, nullptr, s, nullptr, 1));
    return red_launch(g, te_e, tmp_o, in_e, 0, sym ? EPI_TWX_AXPY_TW : EPI_TWX_AXPY, -k2, R, &Q, nullptr, red, s);
}

// CG's residual update without storing A^dag A p: launches 1 - 2 as normal_core with the fused
// |A p|^2 (red_a, whose finish leaves alpha = |r|^2 / |A p|^2 at *alpha_dev), launch 3 the first
// factor of M_asym^dag, launch 4 its second factor with r <- r - alpha (R^dag te - kappa^2
// H^dag_eo tmp) in place and |r|^2 summed in the same epilogue (red_r).
tm_status normal_rupd_core(const tm_gauge *g, const tm_field *r_e, const tm_field *p_e, const tm_field *te_e,
                           const tm_field *tmp_o, int pc, cudaStream_t s, const RedArgs *red_a, const RedArgs *red_r,
                           const double *alpha_dev)
{
    TM_TRY(normal_first_half_red(g, te_e, p_e, tmp_o, pc, s, red_a));
    const double k2 = g->p.kappa * g->p.kappa;
    const Twist<double> Rd = make_twist(g, TW_R, 1), Rid = make_twist(g, TW_RINV, 1);
    TM_TRY(dslash_launch(g, tmp_o, te_e, nullptr, 1, 1, EPI_TW, 1.0, &Rid, nullptr, s, nullptr, 1));
    return red_launch(g, r_e, tmp_o, te_e, 1, EPI_TWX_AXPY_RUPD, -k2, Rd, nullptr, alpha_dev, red_r, s);
}

// out = A^dag in with A = M_pc (A = M_pc^dag when dagger); in is overwritten.  For A = M_sym,
// A^dag = M_sym^dag = M_asym^dag R_ee^-dag (M_sym = R_ee^-1 M_asym): R_ee^-dag as a site pass on in,
// then M_asym^dag, which needs no input-twist prologue.
tm_status adjoint_core(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o, int pc,
                       int dagger, cudaStream_t s)
{
    if (pc == TM_PC_SYM && !dagger && g->csw == 0.0) {
        const Twist<double> Rid = make_twist(g, TW_RINV, 1);
        TM_TRY(cuda_check(launch_twist_active(g, in_e, in_e, Rid, nullptr, 1, s), "twist"));
        return precond_core(g, out_e, in_e, tmp_o, TM_PC_ASYM, 1, s, nullptr, 1);
    }
    return precond_core(g, out_e, in_e, tmp_o, pc, !dagger, s, nullptr, 1);
}

// out = A^dag A in with A = M_pc, or A = M_pc^dag when dagger (tm_normal_op).  For the symmetric
// operator (no dagger, no clover term) M_sym = R_ee^-1 M_asym gives
//   M_sym^dag M_sym = M_asym^dag (R_ee R_ee^dag)^-1 M_asym,
// four launches without the input-twist prologue: M_asym with Q = (R R^dag)^-1 applied in the
// epilogue of its second launch, then M_asym^dag.  te_e is overwritten with that intermediate.
tm_status normal_core(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *te_e,
                      const tm_field *tmp_o, int pc, int dagger, cudaStream_t s, const int *act, int nact,
                      const RedArgs *red)
{
    if (red) {
        if (dagger || act || nact > 1) {
            set_error("internal: fused reduction not available for this operator");
            return TM_ERR_ARG;
        }
        TM_TRY(normal_first_half_red(g, te_e, in_e, tmp_o, pc, s, red));
        return precond_core(g, out_e, te_e, tmp_o, TM_PC_ASYM, 1, s, nullptr, 1);
    }
    if (pc == TM_PC_SYM && !dagger && g->csw == 0.0) {
        const double k2 = g->p.kappa * g->p.kappa;
        const Twist<double> R = make_twist(g, TW_R, 0), Ri = make_twist(g, TW_RINV, 0), Q = rrdag_inverse(g);
        TM_TRY(dslash_launch(g, tmp_o, in_e, nullptr, 1, 0, EPI_TW, 1.0, &Ri, nullptr, s, act, nact));
        TM_TRY(dslash_launch(g, te_e, tmp_o, in_e, 0, 0, EPI_TWX_AXPY_TW, -k2, &R, nullptr, s, act, nact, 0, 0, &Q));
        return precond_core(g, out_e, te_e, tmp_o, TM_PC_ASYM, 1, s, act, nact);
    }
    TM_TRY(precond_core(g, te_e, in_e, tmp_o, pc, dagger, s, act, nact));
    return precond_core(g, out_e, te_e, tmp_o, pc, !dagger, s, act, nact);
}

// The kernel epilogue, coefficient and local operator of a tm_epilogue code (tm_dslash's mapping)
static tm_status epilogue_of(const tm_gauge *g, int epilogue, int dagger, int *epi, double *coef, Twist<double> *tw,
                             bool *has_tw)
{
    const double k = g->p.kappa;
    *has_tw = true;
    switch (epilogue) {
    case TM_EPI_NONE: *epi = EPI_SCALE; *coef = 1.0; *has_tw = false; break;
    case TM_EPI_TWINV: *epi = EPI_TW; *coef = 1.0; *tw = make_twist(g, TW_RINV, dagger); break;
    case TM_EPI_TWXPAY_ASYM: *epi = EPI_TWX_AXPY; *coef = -k * k; *tw = make_twist(g, TW_R, dagger); break;
    case TM_EPI_TWXPAY_SYM: *epi = EPI_X_TWAXPY; *coef = -k * k; *tw = make_twist(g, TW_RINV, dagger); break;
    case TM_EPI_XPAY: *epi = EPI_XPAY; *coef = k; *has_tw = false; break;
    case TM_EPI_XMAY_K2: *epi = EPI_XPAY; *coef = -k * k; *has_tw = false; break;
    case TM_EPI_TWINV_XPAY: *epi = EPI_TW_XPAY; *coef = k; *tw = make_twist(g, TW_RINV, dagger); break;
    default: set_error("unknown epilogue %d", epilogue); return TM_ERR_ARG;
    }
    return TM_OK;
}

static tm_status check_dd(const tm_gauge *g, const tm_field *f, const char *what)
{
    if (!g->dd) { set_error("%s: the handle holds no slab (tm_gauge_set_partition)", what); return TM_ERR_ARG; }
    if (f->prec == TM_PREC_DF64 || f->nrhs != 1) {
        set_error("%s: decomposed operators take single-RHS FP64 / FP32 / FP16 fields", what);
        return TM_ERR_ARG;
    }
    return TM_OK;
}


// face pack (ghost == NULL) or boundary-slice launch of a slab
template <typename T>
static cudaError_t dd_launch_t(const tm_gauge *g, DslashArgs<T> &a, const DDArgs<T> *dd, void *fp, void *fn, bool pro,
                               int pidx, cudaStream_t s)
{
    if constexpr (std::is_same<T, double>::value) return launch_dd_p64(a, dd, fp, fn, g->nf, link_recon(g, 0), pro, s);
    else return pidx == 1 ? launch_dd_p32(a, dd, fp, fn, g->nf, link_recon(g, pidx), pro, s)
                          : launch_dd_p16(a, dd, fp, fn, g->nf, link_recon(g, pidx), pro, s);
}

template <typename T>
static tm_status dd_call(const tm_gauge *g, const tm_field *out, const tm_field *in, const tm_field *x, int out_parity,
                         int dagger, int epi, double coef, const Twist<double> &tw_epi, const Twist<double> *tw_pro,
                         const void *ghost_prev, const void *ghost_next, void *face_prev, void *face_next, cudaStream_t s)
{
    const int pidx = prec_index(in->prec);
    TM_TRY(need_links(g, in->prec));
    DslashArgs<T> a;
    memset(&a, 0, sizeof(a));
    fill_common(a, g, out ? out : in, in, x, out_parity, pidx);
    a.epilogue = epi;
    a.sigma = dagger ? T(-1) : T(1);
    a.coef = (T)coef;
    Twist<double> z;
    memset(&z, 0, sizeof(z));
    if constexpr (std::is_same<T, double>::value) {
        a.tw_epi = tw_epi;
        a.tw_pro = tw_pro ? *tw_pro : z;
    } else {
        a.tw_epi = to_float(tw_epi);
        a.tw_pro = to_float(tw_pro ? *tw_pro : z);
    }
    if (!ghost_prev && !ghost_next) return cuda_check(dd_launch_t<T>(g, a, nullptr, face_prev, face_next, tw_pro != nullptr, pidx, s), "tm_dd_pack_faces");
    DDArgs<T> dd;
    dd.ghost_b = ghost_prev;
    dd.ghost_f = ghost_next;
    dd.st = g->X1h * g->p.L[1] * g->p.L[2];
    dd.sign_b = (T)g->dd_sign_b;
    dd.sign_f = (T)g->dd_sign_f;
    return cuda_check(dd_launch_t<T>(g, a, &dd, nullptr, nullptr, tw_pro != nullptr, pidx, s), "tm_dd_dslash boundary");
}

}  // namespace tmk

using namespace tmk;

// =============================================================================== C ABI
extern "C" {

const char *tm_version(void) { return "libtm 0.1 (sm_103a)"; }

tm_status tm_last_error(char *buf, size_t n)
{
    if (!buf || n == 0) return TM_ERR_ARG;
    snprintf(buf, n, "%s", g_err);
    return TM_OK;
}

tm_status tm_gauge_create(const tm_params *p, const void *U_canon, void *stream, tm_gauge **out)
{
    return tm_gauge_create_ex(p, U_canon, 0, stream, out);
}

tm_status tm_gauge_create_ex(const tm_params *p, const void *U_canon, int prec_mask, void *stream, tm_gauge **out)
{
    TM_NVTX("tm_gauge_create");
    if (prec_mask < 0 || prec_mask > 31) { set_error("tm_gauge_create_ex: prec_mask must be in [0, 31]"); return TM_ERR_ARG; }
    const bool f64_full = (prec_mask & TM_GAUGE_F64_FULL_LINKS) != 0;
    prec_mask &= 15;
    if (prec_mask == 0) prec_mask = 15;
    TM_TRY(check_params(p));
    if (!U_canon || !out) { set_error("tm_gauge_create: null pointer"); return TM_ERR_ARG; }
    *out = nullptr;
    tm_gauge *g = new tm_gauge;
    memset(g, 0, sizeof(*g));
    g->p = *p;
    g->nf = (p->flavor == TM_NDEG_DOUBLET) ? 2 : 1;
    const long V = (long)p->L[0] * p->L[1] * p->L[2] * p->L[3];
    g->Vh = (int)(V / 2);
    g->X1h = p->L[0] / 2;
    // link format per storage form: the handle's recon, except 18 reals for FP64 on request and at
    // least 12 for DF64 (no 8-real DF64 kernels)
    g->recon[0] = f64_full ? 18 : p->recon;
    g->recon[1] = g->recon[2] = p->recon;
    g->recon[3] = p->recon == 8 ? 12 : p->recon;
    for (int i = 0; i < 4; i++) {
        // measured on GB300 at 32^3x64: the register cap (3) for FP64; for FP32 and FP16 the
        // shared-memory staged pipeline with the paired hop: the doublet's flavours paired (FP32
        // 2 buffers, 8; FP16 3 buffers, 9), one flavour's spin rows paired (3 buffers, 9) except
        // with 18-real links, where the register cap stays ahead
        for (int j = 0; j < 2; j++) g->tune[i][j] = tm_tune_entry{3, 128};
        const bool nd = p->flavor == TM_NDEG_DOUBLET;
        if ((i == 1 || i == 2) && (nd || p->recon != 18))
            for (int j = 0; j < 2; j++) g->tune[i][j] = tm_tune_entry{(nd && i == 1) ? 8 : 9, 128};
        // multi-RHS shape, measured at 32^3x64 on 16 sources: the staged form with 4 sources per block
        // in group-major order for the binary32 / binary16 doublet, paired sources for one flavour
        // (group-major for FP32); FP64 the register form, 4
        g->multi_rpb[i] = (i == 1 || i == 2) ? (nd ? 34 : (i == 1 ? 36 : 16)) : 4;
        // measured on GB300 at 32^3x64: FP32 one flavour 4, doublet 3; FP16 3; FP64 insensitive
        if (i < 3) g->clov_minb[i] = i == 0 ? 1 : ((i == 1 && p->flavor != TM_NDEG_DOUBLET) ? 4 : 3);
    }
    cudaStream_t s = (cudaStream_t)stream;
    void *Ud = nullptr;
    tm_status st = resolve_canon(U_canon, &Ud, "tm_gauge_create");
    if (st != TM_OK) {
        delete g;
        return st;
    }
    U_canon = Ud;
    st = cuda_check(cudaGetDevice(&g->device), "cudaGetDevice");
    if (st == TM_OK) st = cuda_check(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device),
                                     "cudaDeviceGetAttribute");
    const int precs[4] = {TM_PREC_F64, TM_PREC_F32, TM_PREC_F16, TM_PREC_DF64};
    for (int i = 0; i < 4 && st == TM_OK; i++) {
        if (!(prec_mask & (1 << i))) continue;  // this storage form is not packed: its operators are refused
        const int recon_i = g->recon[i];
        const size_t per_link = (size_t)recon_i * real_bytes(precs[i]);
        const size_t chunks = per_link / link_chunk_bytes(precs[i], recon_i);
        g->link_bytes[i] = 8ull * g->Vh * chunks * link_chunk_bytes(precs[i], recon_i);
        if (cudaMalloc(&g->links[i], g->link_bytes[i]) != cudaSuccess) {
            set_error("tm_gauge_create: cudaMalloc of %zu bytes failed", g->link_bytes[i]);
            st = TM_ERR_NOMEM;
            break;
        }
        st = cuda_check(launch_pack_gauge(g, i, g->links[i], U_canon, s), "pack gauge");
    }
    if (st == TM_OK) {
        g->scratch_bytes = 1 << 20;
        if (cudaMalloc((void **)&g->scratch, g->scratch_bytes) != cudaSuccess) {
            set_error("tm_gauge_create: scratch allocation failed");
            st = TM_ERR_NOMEM;
        } else {
            st = cuda_check(cudaMemsetAsync(g->scratch, 0, g->scratch_bytes, s), "scratch memset");
        }
    }
    if (st == TM_OK && cudaHostAlloc((void **)&g->host_scalars, 4096, cudaHostAllocDefault) != cudaSuccess) {
        set_error("tm_gauge_create: pinned host allocation failed");
        st = TM_ERR_NOMEM;
    }
    if (st == TM_OK) st = build_fused_work(g, s);
    if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "tm_gauge_create sync");
    if (st != TM_OK) {
        tm_gauge_destroy(g);
        return st;
    }
    *out = g;
    return TM_OK;
}

tm_status tm_gauge_destroy(tm_gauge *g)
{
    if (!g) return TM_OK;
    cudaDeviceSynchronize();
    for (int i = 0; i < 4; i++)
        if (g->links[i]) cudaFree(g->links[i]);
    clover_free(g);
    if (g->fused_items) cudaFree(g->fused_items);
    if (g->fused_sync) cudaFree(g->fused_sync);
    if (g->scratch) cudaFree(g->scratch);
    if (g->host_scalars) cudaFreeHost(g->host_scalars);
    delete g;
    return TM_OK;
}

tm_status tm_field_bytes(const tm_gauge *g, int prec, int nrhs, size_t *data_bytes, size_t *norm_bytes)
{
    if (!g || !data_bytes || !norm_bytes) { set_error("tm_field_bytes: null pointer"); return TM_ERR_ARG; }
    if (prec_index(prec) < 0 || nrhs < 1) { set_error("tm_field_bytes: bad prec or nrhs"); return TM_ERR_ARG; }
    const size_t sites = (size_t)g->Vh * g->nf * nrhs;
    *data_bytes = sites * 24 * real_bytes(prec);
    *norm_bytes = (prec == TM_PREC_F16) ? sites * sizeof(float) : 0;
    return TM_OK;
}

// host <-> device copies of a field in the library's own layout: the bytes of data (and of the
// FP16 norm array) are moved unchanged, one cudaMemcpyAsync per array
static tm_status field_copy(const tm_gauge *g, const tm_field *f, void *data_dst, const void *data_src, void *norm_dst,
                            const void *norm_src, cudaMemcpyKind kind, cudaStream_t s, const char *what)
{
    size_t db = 0, nb = 0;
    TM_TRY(tm_field_bytes(g, f->prec, f->nrhs, &db, &nb));
    if (!data_dst || !data_src || (nb && (!norm_dst || !norm_src))) {
        set_error("%s: null pointer", what);
        return TM_ERR_ARG;
    }
    TM_TRY(cuda_check(cudaMemcpyAsync(data_dst, data_src, db, kind, s), what));
    if (nb) TM_TRY(cuda_check(cudaMemcpyAsync(norm_dst, norm_src, nb, kind, s), what));
    return TM_OK;
}

tm_status tm_field_upload(const tm_gauge *g, const tm_field *dev, const void *host_data, const void *host_norm,
                          void *stream)
{
    TM_NVTX("tm_field_upload");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, dev, "dev"));
    return field_copy(g, dev, dev->data, host_data, dev->norm, host_norm, cudaMemcpyHostToDevice,
                      (cudaStream_t)stream, "tm_field_upload");
}

tm_status tm_field_download(const tm_gauge *g, void *host_data, void *host_norm, const tm_field *dev, void *stream)
{
    TM_NVTX("tm_field_download");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, dev, "dev"));
    return field_copy(g, dev, host_data, dev->data, host_norm, dev->norm, cudaMemcpyDeviceToHost,
                      (cudaStream_t)stream, "tm_field_download");
}

tm_status tm_pack(const tm_gauge *g, const tm_field *out, const void *canon, int canon_type, int parity, void *stream)
{
    TM_NVTX("tm_pack");
    if (!g || !canon) { set_error("tm_pack: null pointer"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, out, "out"));
    if (parity != 0 && parity != 1) { set_error("parity must be 0 or 1"); return TM_ERR_ARG; }
    if (canon_type != TM_C128 && canon_type != TM_C64) { set_error("unknown canon_type"); return TM_ERR_ARG; }
    void *cd = nullptr;
    TM_TRY(resolve_canon(canon, &cd, "tm_pack"));
    return cuda_check(launch_pack_spinor(g, out, cd, canon_type, parity, (cudaStream_t)stream), "tm_pack");
}

tm_status tm_unpack(const tm_gauge *g, void *canon, int canon_type, const tm_field *in, int parity, void *stream)
{
    TM_NVTX("tm_unpack");
    if (!g || !canon) { set_error("tm_unpack: null pointer"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, in, "in"));
    if (parity != 0 && parity != 1) { set_error("parity must be 0 or 1"); return TM_ERR_ARG; }
    if (canon_type != TM_C128 && canon_type != TM_C64) { set_error("unknown canon_type"); return TM_ERR_ARG; }
    void *cd = nullptr;
    TM_TRY(resolve_canon(canon, &cd, "tm_unpack"));
    return cuda_check(launch_unpack_spinor(g, cd, canon_type, in, parity, (cudaStream_t)stream), "tm_unpack");
}

tm_status tm_noise_z2(const tm_gauge *g, const tm_field *out, int parity, unsigned long long seed, void *stream)
{
    TM_NVTX("tm_noise_z2");
    if (!g) { set_error("tm_noise_z2: null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, out, "out"));
    if (parity != 0 && parity != 1) { set_error("parity must be 0 or 1"); return TM_ERR_ARG; }
    return cuda_check(launch_noise_z2(g, out, parity, seed, (cudaStream_t)stream), "tm_noise_z2");
}

tm_status tm_dslash(const tm_gauge *g, const tm_field *out, const tm_field *in, int out_parity, int epilogue,
                    const tm_field *x, void *stream)
{
    TM_NVTX("tm_dslash");
    return dslash_api(g, out, in, out_parity, epilogue, x, stream, 0);
}

tm_status tm_dslash_dagger(const tm_gauge *g, const tm_field *out, const tm_field *in, int out_parity, int epilogue,
                           const tm_field *x, void *stream)
{
    TM_NVTX("tm_dslash_dagger");
    return dslash_api(g, out, in, out_parity, epilogue, x, stream, 1);
}

tm_status tm_precond_op(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o, int pc,
                        int dagger, void *stream)
{
    TM_NVTX("tm_precond_op");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(refuse_slab(g, "tm_precond_op"));
    TM_TRY(check_field(g, out_e, "out_e"));
    TM_TRY(check_field(g, in_e, "in_e"));
    TM_TRY(check_field(g, tmp_o, "tmp_o"));
    TM_TRY(same_prec(out_e, in_e, "tm_precond_op"));
    TM_TRY(same_prec(out_e, tmp_o, "tm_precond_op"));
    if (out_e->nrhs > TM_MAX_RHS_API) { set_error("tm_precond_op: at most %d right-hand sides", TM_MAX_RHS_API); return TM_ERR_ARG; }
    if (pc != TM_PC_ASYM && pc != TM_PC_SYM) { set_error("unknown pc %d", pc); return TM_ERR_ARG; }
    if (out_e->data == in_e->data || tmp_o->data == in_e->data || tmp_o->data == out_e->data) {
        set_error("tm_precond_op: out_e, in_e and tmp_o must be distinct");
        return TM_ERR_ARG;
    }
    return precond_core(g, out_e, in_e, tmp_o, pc, dagger, (cudaStream_t)stream, nullptr, out_e->nrhs);
}

tm_status tm_precond_op_active(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o,
                               int pc, int dagger, const int *active_dev, int nactive, void *stream)
{
    TM_NVTX("tm_precond_op_active");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(refuse_slab(g, "tm_precond_op_active"));
    TM_TRY(check_field(g, out_e, "out_e"));
    TM_TRY(check_field(g, in_e, "in_e"));
    TM_TRY(check_field(g, tmp_o, "tmp_o"));
    TM_TRY(same_prec(out_e, in_e, "tm_precond_op_active"));
    TM_TRY(same_prec(out_e, tmp_o, "tm_precond_op_active"));
    if (pc != TM_PC_ASYM && pc != TM_PC_SYM) { set_error("unknown pc %d", pc); return TM_ERR_ARG; }
    if (!active_dev || nactive < 1 || nactive > out_e->nrhs) {
        set_error("tm_precond_op_active: need 1 <= nactive <= nrhs (%d) and a device index list", out_e->nrhs);
        return TM_ERR_ARG;
    }
    if (out_e->data == in_e->data || tmp_o->data == in_e->data || tmp_o->data == out_e->data) {
        set_error("tm_precond_op_active: out_e, in_e and tmp_o must be distinct");
        return TM_ERR_ARG;
    }
    return precond_core(g, out_e, in_e, tmp_o, pc, dagger, (cudaStream_t)stream, active_dev, nactive);
}

tm_status tm_normal_op(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_e,
                       const tm_field *tmp_o, int pc, int dagger, void *stream)
{
    TM_NVTX("tm_normal_op");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(refuse_slab(g, "tm_normal_op"));
    TM_TRY(check_field(g, out_e, "out_e"));
    TM_TRY(check_field(g, in_e, "in_e"));
    TM_TRY(check_field(g, tmp_e, "tmp_e"));
    TM_TRY(check_field(g, tmp_o, "tmp_o"));
    TM_TRY(same_prec(out_e, in_e, "tm_normal_op"));
    TM_TRY(same_prec(out_e, tmp_e, "tm_normal_op"));
    TM_TRY(same_prec(out_e, tmp_o, "tm_normal_op"));
    if (out_e->nrhs > TM_MAX_RHS_API) { set_error("tm_normal_op: at most %d right-hand sides", TM_MAX_RHS_API); return TM_ERR_ARG; }
    if (pc != TM_PC_ASYM && pc != TM_PC_SYM) { set_error("unknown pc %d", pc); return TM_ERR_ARG; }
    const void *d[4] = {out_e->data, in_e->data, tmp_e->data, tmp_o->data};
    for (int i = 0; i < 4; i++)
        for (int j = i + 1; j < 4; j++)
            if (d[i] == d[j]) { set_error("tm_normal_op: out_e, in_e, tmp_e and tmp_o must be distinct"); return TM_ERR_ARG; }
    return normal_core(g, out_e, in_e, tmp_e, tmp_o, pc, dagger, (cudaStream_t)stream, nullptr, out_e->nrhs, nullptr);
}

tm_status tm_mat(const tm_gauge *g, const tm_field *out_e, const tm_field *out_o, const tm_field *in_e,
                 const tm_field *in_o, int dagger, void *stream)
{
    TM_NVTX("tm_mat");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(refuse_slab(g, "tm_mat"));
    TM_TRY(check_field(g, out_e, "out_e"));
    TM_TRY(check_field(g, out_o, "out_o"));
    TM_TRY(check_field(g, in_e, "in_e"));
    TM_TRY(check_field(g, in_o, "in_o"));
    TM_TRY(same_prec(out_e, in_e, "tm_mat"));
    TM_TRY(same_prec(out_o, in_o, "tm_mat"));
    TM_TRY(same_prec(out_e, out_o, "tm_mat"));
    if (out_e->data == in_e->data || out_e->data == in_o->data || out_o->data == in_e->data ||
        out_o->data == in_o->data) {
        set_error("tm_mat: outputs must not alias inputs");
        return TM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Twist<double> R = make_twist(g, TW_R, dagger);
    const double k = g->p.kappa;
    // out_p = R in_p - kappa H_{p,1-p} in_{1-p}
    TM_TRY(dslash_launch(g, out_e, in_o, in_e, 0, dagger, EPI_TWX_AXPY, -k, &R, nullptr, s));
    return dslash_launch(g, out_o, in_e, in_o, 1, dagger, EPI_TWX_AXPY, -k, &R, nullptr, s);
}

tm_status tm_prepare_rhs(const tm_gauge *g, const tm_field *bprime_e, const tm_field *b_e, const tm_field *b_o, int pc,
                         int dagger, void *stream)
{
    TM_NVTX("tm_prepare_rhs");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(refuse_slab(g, "tm_prepare_rhs"));
    TM_TRY(check_field(g, bprime_e, "bprime_e"));
    TM_TRY(check_field(g, b_e, "b_e"));
    TM_TRY(check_field(g, b_o, "b_o"));
    TM_TRY(same_prec(bprime_e, b_e, "tm_prepare_rhs"));
    TM_TRY(same_prec(bprime_e, b_o, "tm_prepare_rhs"));
    if (pc != TM_PC_ASYM && pc != TM_PC_SYM) { set_error("unknown pc %d", pc); return TM_ERR_ARG; }
    if (bprime_e->data == b_o->data) { set_error("tm_prepare_rhs: bprime_e must not alias b_o"); return TM_ERR_ARG; }
    if (bprime_e->prec == TM_PREC_DF64) { set_error("tm_prepare_rhs: use FP64 fields (no DF64 form)"); return TM_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const Twist<double> Ri = make_twist(g, TW_RINV, dagger);
    const double k = g->p.kappa;
    if (g->csw != 0.0) {
        // clover: t_o = L^-1_oo b_o in a temporary from the stream-ordered pool, then
        // b' = b_e + kappa H_eo t_o (sym: L^-1_ee of that)
        if (b_o->nrhs != 1) { set_error("clover handles take single-RHS fields (nrhs = 1)"); return TM_ERR_ARG; }
        size_t db = 0, nb = 0;
        TM_TRY(tm_field_bytes(g, b_o->prec, 1, &db, &nb));
        void *tbuf = nullptr;
        const size_t dpad = (db + 255) & ~(size_t)255;
        if (cudaMallocAsync(&tbuf, dpad + nb, s) != cudaSuccess) {
            cudaGetLastError();
            set_error("tm_prepare_rhs: temporary allocation failed");
            return TM_ERR_NOMEM;
        }
        tm_field t;
        t.data = tbuf;
        t.norm = nb ? (float *)((char *)tbuf + dpad) : nullptr;
        t.prec = b_o->prec;
        t.nrhs = 1;
        tm_status st = cuda_check(launch_clover_apply(g, &t, b_o, 1, true, clover_x(g, dagger), s), "clover apply");
        if (st == TM_OK) {
            if (pc == TM_PC_SYM && !dagger) st = dslash_launch(g, bprime_e, &t, b_e, 0, 0, EPI_TW_XPAY, k, &Ri, nullptr, s);
            else st = dslash_launch(g, bprime_e, &t, b_e, 0, dagger, EPI_XPAY, k, nullptr, nullptr, s);
        }
        cudaFreeAsync(tbuf, s);
        return st;
    }
    // b' = b_e + kappa H_eo (R^-1_oo b_o)   [the R^-1 twist is the prologue on every neighbour]
    if (pc == TM_PC_SYM && !dagger)
        return dslash_launch(g, bprime_e, b_o, b_e, 0, 0, EPI_TW_XPAY, k, &Ri, &Ri, s);
    return dslash_launch(g, bprime_e, b_o, b_e, 0, dagger, EPI_XPAY, k, nullptr, &Ri, s);
}

tm_status tm_reconstruct_odd(const tm_gauge *g, const tm_field *psi_o, const tm_field *b_o, const tm_field *psi_e,
                             int dagger, void *stream)
{
    TM_NVTX("tm_reconstruct_odd");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(refuse_slab(g, "tm_reconstruct_odd"));
    TM_TRY(check_field(g, psi_o, "psi_o"));
    TM_TRY(check_field(g, b_o, "b_o"));
    TM_TRY(check_field(g, psi_e, "psi_e"));
    TM_TRY(same_prec(psi_o, b_o, "tm_reconstruct_odd"));
    TM_TRY(same_prec(psi_o, psi_e, "tm_reconstruct_odd"));
    if (psi_o->data == psi_e->data) { set_error("tm_reconstruct_odd: psi_o must not alias psi_e"); return TM_ERR_ARG; }
    const Twist<double> Ri = make_twist(g, TW_RINV, dagger);
    return dslash_launch(g, psi_o, psi_e, b_o, 1, dagger, EPI_TW_XPAY, g->p.kappa, &Ri, nullptr, (cudaStream_t)stream);
}

tm_status tm_autotune(tm_gauge *g0, void *stream)
{
    TM_NVTX("tm_autotune");
    if (!g0) { set_error("null gauge handle"); return TM_ERR_ARG; }
    // the tune table chooses among the twisted-mass kernels; a clover handle's kernels have one
    // launch form, so the table is tuned on a shallow copy of the handle without the clover term
    tm_gauge gcopy = *g0;
    gcopy.csw = 0.0;
    tm_gauge *g = &gcopy;
    struct CopyBack {
        tm_gauge *dst;
        const tm_gauge *src;
        ~CopyBack()
        {
            memcpy(dst->tune, src->tune, sizeof(dst->tune));
            memcpy(dst->multi_rpb, src->multi_rpb, sizeof(dst->multi_rpb));
            memcpy(dst->fused, src->fused, sizeof(dst->fused));
        }
    } copy_back{g0, g};
    cudaStream_t s = (cudaStream_t)stream;
    const int precs[3] = {TM_PREC_F64, TM_PREC_F32, TM_PREC_F16};
    const int blocks[4] = {64, 128, 192, 256};
    tm_status st = TM_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void *buf = nullptr;
    size_t d, n;
    tm_field_bytes(g, TM_PREC_F64, 1, &d, &n);
    const size_t fb = (d + 255) & ~(size_t)255;
    if (cudaMalloc(&buf, 3 * fb) != cudaSuccess) { set_error("tm_autotune: allocation failed"); return TM_ERR_NOMEM; }
    st = cuda_check(cudaMemsetAsync(buf, 0, 3 * fb, s), "tm_autotune memset");
    if (st == TM_OK) st = cuda_check(cudaEventCreate(&e0), "event");
    if (st == TM_OK) st = cuda_check(cudaEventCreate(&e1), "event");
    for (int pi = 0; pi < 3 && st == TM_OK; pi++) {
        if (!g->links[pi]) continue;  // not packed on this handle
        // one FP64-sized buffer per field holds any precision; FP16 norms sit in the tail
        tm_field_bytes(g, precs[pi], 1, &d, &n);
        tm_field f[3];
        for (int k = 0; k < 3; k++) {
            f[k].data = (char *)buf + k * fb;
            f[k].norm = n ? (float *)((char *)buf + k * fb + ((d + 255) & ~(size_t)255)) : nullptr;
            f[k].prec = precs[pi];
            f[k].nrhs = 1;
        }
        const Twist<double> Ri = make_twist(g, TW_RINV, 0);
        for (int pro = 0; pro < 2 && st == TM_OK; pro++) {
            float best = 1e30f;
            tm_tune_entry bestc = g->tune[pi][pro];
            const int variants[9] = {0, 2, 3, 4, 5, 6, 7, 8, 9};
            for (int vi = 0; vi < 9; vi++) {
                const int variant = variants[vi];
                if (pro && variant == 2) continue;  // the register pipeline has no prologue
                if (variant >= 8 && pi == 0) continue;  // paired forms: binary32 only
                for (int bi = 0; bi < 4 && st == TM_OK; bi++) {
                    if (variant >= 3 && blocks[bi] != 128) continue;  // capped forms fix their own block
                    g->tune[pi][pro] = tm_tune_entry{variant, blocks[bi]};
                    float ms = 0;
                    for (int rep = 0; rep < 4 && st == TM_OK; rep++) {
                        st = cuda_check(cudaEventRecord(e0, s), "event");
                        if (st == TM_OK)
                            st = dslash_launch(g, &f[0], &f[1], &f[2], 0, 0, EPI_TWX_AXPY, -0.01, &Ri, pro ? &Ri : nullptr, s);
                        if (st == TM_OK) st = cuda_check(cudaEventRecord(e1, s), "event");
                        if (st == TM_OK) st = cuda_check(cudaEventSynchronize(e1), "event sync");
                        float t = 0;
                        if (st == TM_OK) cudaEventElapsedTime(&t, e0, e1);
                        if (rep > 0) ms += t;  // first repetition warms up
                    }
                    if (st == TM_OK && ms < best) {
                        best = ms;
                        bestc = g->tune[pi][pro];
                    }
                }
            }
            g->tune[pi][pro] = bestc;
        }
        if (g0->csw != 0.0 && st == TM_OK) {
            // clover kernel occupancy, timed on the heavier launch (the inverse L^-1 epilogue)
            const int minbs[4] = {1, 3, 4, 6};
            float best = 1e30f;
            int bestm = g0->clov_minb[pi];
            for (int mi = 0; mi < 4 && st == TM_OK; mi++) {
                g0->clov_minb[pi] = minbs[mi];
                float ms = 0;
                for (int rep = 0; rep < 4 && st == TM_OK; rep++) {
                    st = cuda_check(cudaEventRecord(e0, s), "event");
                    if (st == TM_OK) st = dslash_launch(g0, &f[0], &f[1], nullptr, 1, 0, EPI_TW, 1.0, &Ri, nullptr, s);
                    if (st == TM_OK) st = cuda_check(cudaEventRecord(e1, s), "event");
                    if (st == TM_OK) st = cuda_check(cudaEventSynchronize(e1), "event sync");
                    float t = 0;
                    if (st == TM_OK) cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0) ms += t;
                }
                if (st == TM_OK && ms < best) {
                    best = ms;
                    bestm = minbs[mi];
                }
            }
            g0->clov_minb[pi] = bestm;
        }
    }
    // fused operator or two launches, timed on the asymmetric operator (FP64, FP32)
    for (int pi = 0; pi < 2 && st == TM_OK; pi++) {
        if (!g->links[pi]) continue;
        tm_field_bytes(g, precs[pi], 1, &d, &n);
        tm_field f[3];
        for (int k = 0; k < 3; k++) {
            f[k].data = (char *)buf + k * fb;
            f[k].norm = nullptr;
            f[k].prec = precs[pi];
            f[k].nrhs = 1;
        }
        float best = 1e30f;
        int bestf = 0;
        for (int fz = 0; fz < 2 && st == TM_OK; fz++) {
            g->fused[pi] = fz;
            float ms = 0;
            for (int rep = 0; rep < 4 && st == TM_OK; rep++) {
                st = cuda_check(cudaEventRecord(e0, s), "event");
                if (st == TM_OK) st = precond_core(g, &f[0], &f[1], &f[2], TM_PC_ASYM, 0, s, nullptr, 1);
                if (st == TM_OK) st = cuda_check(cudaEventRecord(e1, s), "event");
                if (st == TM_OK) st = cuda_check(cudaEventSynchronize(e1), "event sync");
                float t = 0;
                if (st == TM_OK) cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms += t;
            }
            if (st == TM_OK && ms < best) {
                best = ms;
                bestf = fz;
            }
        }
        g->fused[pi] = bestf;
    }
    // multi-RHS block shape (right-hand sides per block), timed on 16 right-hand sides (8 in FP64)
    // of the single-RHS buffers' size each -- the block order's trade-off between link and spinor
    // reuse depends on the batch, so the shape is chosen at a typical batch size; the fields are
    // carved from one allocation of 3 x nr fields
    for (int pi = 0; pi < 3 && st == TM_OK; pi++) {
        if (!g->links[pi]) continue;
        const int nr = pi == 0 ? 8 : 16;
        tm_field_bytes(g, precs[pi], nr, &d, &n);
        const size_t fbm = ((d + 255) & ~(size_t)255) + ((n + 255) & ~(size_t)255);
        void *mbuf = nullptr;
        if (cudaMalloc(&mbuf, 3 * fbm) != cudaSuccess) {
            cudaGetLastError();
            break;  // not enough memory for the multi-RHS timing: keep the default shape
        }
        st = cuda_check(cudaMemsetAsync(mbuf, 0, 3 * fbm, s), "tm_autotune memset");
        tm_field f[3];
        for (int k = 0; k < 3; k++) {
            f[k].data = (char *)mbuf + k * fbm;
            f[k].norm = n ? (float *)((char *)mbuf + k * fbm + ((d + 255) & ~(size_t)255)) : nullptr;
            f[k].prec = precs[pi];
            f[k].nrhs = nr;
        }
        const Twist<double> Ri = make_twist(g, TW_RINV, 0);
        // the paired forms only for one flavour, the three-buffer staged forms only for the FP16 doublet
        const int rpbs[13] = {2, 4, 8, 12, 14, 32, 34, 16, 36, 13, 15, 33, 35};
        float best = 1e30f;
        int bestr = g->multi_rpb[pi];
        for (int ri = 0; ri < 13 && st == TM_OK; ri++) {
            if (ri >= 7 && ri < 9 && g->nf != 1) continue;
            if (ri >= 9 && (g->nf != 2 || pi != 2)) continue;
            g->multi_rpb[pi] = rpbs[ri];
            float ms = 1e30f;  // the fastest of four timed launches (the first warms up)
            for (int rep = 0; rep < 5 && st == TM_OK; rep++) {
                st = cuda_check(cudaEventRecord(e0, s), "event");
                if (st == TM_OK)
                    st = dslash_launch(g, &f[0], &f[1], &f[2], 0, 0, EPI_TWX_AXPY, -0.01, &Ri, nullptr, s, nullptr, nr);
                if (st == TM_OK) st = cuda_check(cudaEventRecord(e1, s), "event");
                if (st == TM_OK) st = cuda_check(cudaEventSynchronize(e1), "event sync");
                float t = 0;
                if (st == TM_OK) cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < ms) ms = t;
            }
            if (st == TM_OK && ms < best) {
                best = ms;
                bestr = rpbs[ri];
            }
        }
        g->multi_rpb[pi] = bestr;
        cudaStreamSynchronize(s);
        cudaFree(mbuf);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    return st;
}

tm_status tm_tune_export(const tm_gauge *g, char *buf, size_t n)
{
    if (!g || !buf || n == 0) { set_error("tm_tune_export: null argument"); return TM_ERR_ARG; }
    const char *names[3] = {"f64", "f32", "f16"};
    size_t off = 0;
    buf[0] = 0;
    for (int pi = 0; pi < 3; pi++)
        for (int pro = 0; pro < 2; pro++) {
            int w = snprintf(buf + off, n - off, "%s%s:%d:%d:%d", off ? " " : "", names[pi], pro,
                             g->tune[pi][pro].variant, g->tune[pi][pro].block);
            if (w < 0 || (size_t)w >= n - off) { set_error("tm_tune_export: buffer too small"); return TM_ERR_ARG; }
            off += (size_t)w;
        }
    for (int pi = 0; pi < 3; pi++) {
        int w = snprintf(buf + off, n - off, " %s:m:%d", names[pi], g->multi_rpb[pi]);
        if (w < 0 || (size_t)w >= n - off) { set_error("tm_tune_export: buffer too small"); return TM_ERR_ARG; }
        off += (size_t)w;
    }
    for (int pi = 0; pi < 3; pi++) {
        int w = snprintf(buf + off, n - off, " %s:c:%d", names[pi], g->clov_minb[pi]);
        if (w < 0 || (size_t)w >= n - off) { set_error("tm_tune_export: buffer too small"); return TM_ERR_ARG; }
        off += (size_t)w;
    }
    for (int pi = 0; pi < 2; pi++) {
        int w = snprintf(buf + off, n - off, " %s:p:%d", names[pi], g->fused[pi]);
        if (w < 0 || (size_t)w >= n - off) { set_error("tm_tune_export: buffer too small"); return TM_ERR_ARG; }
        off += (size_t)w;
    }
    return TM_OK;
}

tm_status tm_tune_import(tm_gauge *g, const char *text)
{
    if (!g || !text) { set_error("tm_tune_import: null argument"); return TM_ERR_ARG; }
    tm_tune_entry t[3][2];
    int mr[3], cm[3], fu[3];
    memcpy(t, g->tune, sizeof(t));
    memcpy(mr, g->multi_rpb, sizeof(mr));
    memcpy(cm, g->clov_minb, sizeof(cm));
    memcpy(fu, g->fused, sizeof(fu));
    const char *p = text;
    while (*p) {
        while (*p == ' ') p++;
        if (!*p) break;
        char name[8] = {0};
        int pro, variant, block, used = 0;
        if (sscanf(p, "%3[a-z0-9]:m:%d%n", name, &block, &used) == 2 && used > 0) {
            // multi-RHS entry "<prec>:m:<right-hand sides per block>"
            const int pi = !strcmp(name, "f64") ? 0 : (!strcmp(name, "f32") ? 1 : (!strcmp(name, "f16") ? 2 : -1));
            const bool okm = block == 2 || block == 4 || block == 8 || block == 12 || block == 14 || block == 16 ||
                             block == 32 || block == 34 || block == 36 ||
                             (pi == 2 && (block == 13 || block == 15 || block == 33 || block == 35));
            if (pi < 0 || !okm) {
                set_error("tm_tune_import: invalid entry '%.32s'", p);
                return TM_ERR_ARG;
            }
            mr[pi] = block;
            p += used;
            continue;
        }
        used = 0;
        if (sscanf(p, "%3[a-z0-9]:p:%d%n", name, &block, &used) == 2 && used > 0) {
            // fused-operator entry "<prec>:p:<0|1>" (FP64 / FP32)
            const int pi = !strcmp(name, "f64") ? 0 : (!strcmp(name, "f32") ? 1 : -1);
            if (pi < 0 || (block != 0 && block != 1)) {
                set_error("tm_tune_import: invalid entry '%.32s'", p);
                return TM_ERR_ARG;
            }
            fu[pi] = block;
            p += used;
            continue;
        }
        used = 0;
        if (sscanf(p, "%3[a-z0-9]:c:%d%n", name, &block, &used) == 2 && used > 0) {
            // clover entry "<prec>:c:<resident blocks per SM>"
            const int pi = !strcmp(name, "f64") ? 0 : (!strcmp(name, "f32") ? 1 : (!strcmp(name, "f16") ? 2 : -1));
            if (pi < 0 || (block != 1 && block != 3 && block != 4 && block != 6)) {
                set_error("tm_tune_import: invalid entry '%.32s'", p);
                return TM_ERR_ARG;
            }
            cm[pi] = block;
            p += used;
            continue;
        }
        used = 0;
        if (sscanf(p, "%3[a-z0-9]:%d:%d:%d%n", name, &pro, &variant, &block, &used) != 4 || used == 0) {
            set_error("tm_tune_import: cannot parse '%.32s'", p);
            return TM_ERR_ARG;
        }
        const int pi = !strcmp(name, "f64") ? 0 : (!strcmp(name, "f32") ? 1 : (!strcmp(name, "f16") ? 2 : -1));
        if (pi < 0 || (pro != 0 && pro != 1) || variant < 0 || variant == 1 || variant > 9 || block < 32 || block > 256 ||
            block % 32) {
            set_error("tm_tune_import: invalid entry '%.32s'", p);
            return TM_ERR_ARG;
        }
        t[pi][pro] = tm_tune_entry{variant, block};
        p += used;
    }
    memcpy(g->tune, t, sizeof(t));
    memcpy(g->multi_rpb, mr, sizeof(mr));
    memcpy(g->clov_minb, cm, sizeof(cm));
    memcpy(g->fused, fu, sizeof(fu));
    return TM_OK;
}

tm_status tm_twist(const tm_gauge *g, const tm_field *out, const tm_field *in, int inverse, int dagger, void *stream)
{
    TM_NVTX("tm_twist");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, out, "out"));
    TM_TRY(check_field(g, in, "in"));
    TM_TRY(same_prec(out, in, "tm_twist"));
    if (g->csw != 0.0) {
        set_error("tm_twist: a clover handle's local operator depends on the site; use tm_local_op");
        return TM_ERR_ARG;
    }
    const Twist<double> T = make_twist(g, inverse ? TW_RINV : TW_R, dagger);
    return cuda_check(launch_twist(g, out, in, T, (cudaStream_t)stream), "tm_twist");
}

tm_status tm_local_op(const tm_gauge *g, const tm_field *out, const tm_field *in, int parity, int inverse, int dagger,
                      void *stream)
{
    TM_NVTX("tm_local_op");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, out, "out"));
    TM_TRY(check_field(g, in, "in"));
    TM_TRY(same_prec(out, in, "tm_local_op"));
    if (parity != 0 && parity != 1) { set_error("tm_local_op: parity must be 0 or 1"); return TM_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (g->csw == 0.0) {
        const Twist<double> T = make_twist(g, inverse ? TW_RINV : TW_R, dagger);
        return cuda_check(launch_twist(g, out, in, T, s), "tm_local_op");
    }
    if (in->prec == TM_PREC_DF64 || in->nrhs != 1) {
        set_error("tm_local_op: clover handles take single-RHS FP64 / FP32 / FP16 fields");
        return TM_ERR_ARG;
    }
    return cuda_check(launch_clover_apply(g, out, in, parity, inverse != 0, clover_x(g, dagger), s), "tm_local_op");
}

int tm_fused_work_list(const int L[4], int num_sms, int *items, int capacity)
{
    if (!L) return -1;
    for (int m = 0; m < 4; m++)
        if (L[m] < 2 || (L[m] & 1)) return -1;
    const std::vector<int> v = fused_items(L, num_sms);
    if (items) {
        if (capacity < (int)v.size()) return -1;
        memcpy(items, v.data(), sizeof(int) * v.size());
    }
    return (int)v.size();
}

tm_status tm_fused_set_work_list(tm_gauge *g, const int *items, int nitems, unsigned long long wait_limit_ns,
                                 void *stream)
{
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    if (!g->fused_items) { set_error("tm_fused_set_work_list: the handle has no work list"); return TM_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> v;
    if (items) {
        // every entry names a group of the lattice and a pass; nothing else is checked, so a list
        // may omit work (the waits that depend on it then give up at the limit)
        const int ngroups = (int)(fused_nflags(g->Vh) / FUSED_GROUP);
        if (nitems < 1 || nitems > g->fused_capacity) {
            set_error("tm_fused_set_work_list: need 1 <= nitems <= %d", g->fused_capacity);
            return TM_ERR_ARG;
        }
        for (int i = 0; i < nitems; i++)
            if (items[i] < 0 || (items[i] >> 1) >= ngroups) {
                set_error("tm_fused_set_work_list: entry %d = %d names no group (%d groups)", i, items[i], ngroups);
                return TM_ERR_ARG;
            }
        v.assign(items, items + nitems);
    } else {
        v = fused_items(g->p.L, g->num_sms);
    }
    if (wait_limit_ns < 1000000ull || wait_limit_ns > 60000000000ull) {
        set_error("tm_fused_set_work_list: wait limit must be 1 ms ... 60 s");
        return TM_ERR_ARG;
    }
    TM_TRY(cuda_check(cudaStreamSynchronize(s), "tm_fused_set_work_list sync"));
    TM_TRY(cuda_check(cudaMemcpyAsync(g->fused_items, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s),
                      "work list copy"));
    TM_TRY(cuda_check(cudaStreamSynchronize(s), "tm_fused_set_work_list sync"));
    g->fused_nitems = (int)v.size();
    g->wait_limit_ns = wait_limit_ns;
    return TM_OK;
}

tm_status tm_device_status(const tm_gauge *g, void *stream)
{
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    int err = 0;
    TM_TRY(cuda_check(cudaMemcpyAsync(&err, g->fused_sync, sizeof(int), cudaMemcpyDeviceToHost, s), "status read"));
    TM_TRY(cuda_check(cudaStreamSynchronize(s), "status sync"));
    if (err) {
        TM_TRY(cuda_check(cudaMemsetAsync(g->fused_sync, 0, sizeof(int), s), "status reset"));
        TM_TRY(cuda_check(cudaStreamSynchronize(s), "status sync"));
        set_error("a bounded device-side wait gave up (the fused operator's output is incomplete)");
        return TM_ERR_TIMEOUT;
    }
    return TM_OK;
}

tm_status tm_gauge_set_clover(tm_gauge *g, double csw, void *stream)
{
    TM_NVTX("tm_gauge_set_clover");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    if (!isfinite(csw)) { set_error("tm_gauge_set_clover: c_sw must be finite"); return TM_ERR_ARG; }
    if (csw == 0.0) {
        cudaDeviceSynchronize();
        clover_free(g);
        return TM_OK;
    }
    return clover_build(g, csw, (cudaStream_t)stream);
}


/* ------------------------------------------------------------------ domain decomposition in t */
tm_status tm_gauge_set_partition(tm_gauge *g, int t_offset, int Lt_global)
{
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    if (Lt_global == 0) {
        g->dd = 0;
        return TM_OK;
    }
    const int Lt = g->p.L[3];
    if (g->csw != 0.0) { set_error("tm_gauge_set_partition: no decomposed clover operator"); return TM_ERR_ARG; }
    if (t_offset < 0 || (t_offset & 1) || Lt_global < Lt || (Lt_global & 1) || t_offset + Lt > Lt_global) {
        set_error("tm_gauge_set_partition: need an even offset t0 >= 0 and t0 + %d <= Lt_global (even)", Lt);
        return TM_ERR_ARG;
    }
    g->dd = 1;
    g->dd_t0 = t_offset;
    g->dd_Lt = Lt_global;
    g->dd_sign_b = (t_offset == 0 && g->p.t_antiperiodic) ? -1.0 : 1.0;
    g->dd_sign_f = (t_offset + Lt == Lt_global && g->p.t_antiperiodic) ? -1.0 : 1.0;
    return TM_OK;
}

tm_status tm_dd_face_bytes(const tm_gauge *g, int prec, size_t *bytes)
{
    if (!g || !bytes) { set_error("tm_dd_face_bytes: null argument"); return TM_ERR_ARG; }
    const size_t b = dd_face_bytes(prec, g->nf, g->X1h * g->p.L[1] * g->p.L[2]);
    if (!b) { set_error("tm_dd_face_bytes: faces exist for FP64, FP32 and FP16 fields"); return TM_ERR_ARG; }
    *bytes = b;
    return TM_OK;
}

tm_status tm_dd_pack_faces(const tm_gauge *g, void *face_prev, void *face_next, const tm_field *in, int out_parity,
                           int dagger, int twist_in, void *stream)
{
    TM_NVTX("tm_dd_pack_faces");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, in, "in"));
    TM_TRY(check_dd(g, in, "tm_dd_pack_faces"));
    if (!face_prev || !face_next || ((uintptr_t)face_prev & 15) || ((uintptr_t)face_next & 15)) {
        set_error("tm_dd_pack_faces: faces must be 16-byte aligned device buffers");
        return TM_ERR_ARG;
    }
    if (out_parity != 0 && out_parity != 1) { set_error("out_parity must be 0 or 1"); return TM_ERR_ARG; }
    const Twist<double> Ri = make_twist(g, TW_RINV, dagger);
    const Twist<double> *pro = twist_in ? &Ri : nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (in->prec == TM_PREC_F64)
        return dd_call<double>(g, nullptr, in, nullptr, out_parity, dagger, EPI_SCALE, 1.0, Ri, pro, nullptr, nullptr,
                               face_prev, face_next, s);
    return dd_call<float>(g, nullptr, in, nullptr, out_parity, dagger, EPI_SCALE, 1.0, Ri, pro, nullptr, nullptr, face_prev,
                          face_next, s);
}

tm_status tm_dd_dslash(const tm_gauge *g, const tm_field *out, const tm_field *in, int out_parity, int epilogue,
                       const tm_field *x, int dagger, int twist_in, const void *ghost_prev, const void *ghost_next,
                       int region, void *stream)
{
    TM_NVTX("tm_dd_dslash");
    if (!g) { set_error("null gauge handle"); return TM_ERR_ARG; }
    TM_TRY(check_field(g, out, "out"));
    TM_TRY(check_field(g, in, "in"));
    TM_TRY(same_prec(out, in, "tm_dd_dslash"));
    TM_TRY(check_dd(g, in, "tm_dd_dslash"));
    if (out_parity != 0 && out_parity != 1) { set_error("out_parity must be 0 or 1"); return TM_ERR_ARG; }
    if (out->data == in->data) { set_error("tm_dd_dslash: out must not alias in"); return TM_ERR_ARG; }
    if (region < TM_DD_ALL || region > TM_DD_BOUNDARY) { set_error("tm_dd_dslash: unknown region %d", region); return TM_ERR_ARG; }
    if (region != TM_DD_INTERIOR && (!ghost_prev || !ghost_next)) {
        set_error("tm_dd_dslash: the boundary slices need both received faces");
        return TM_ERR_ARG;
    }
    int epi;
    double coef;
    Twist<double> tw;
    bool has_tw;
    TM_TRY(epilogue_of(g, epilogue, dagger, &epi, &coef, &tw, &has_tw));
    if (epilogue >= TM_EPI_TWXPAY_ASYM) {
        TM_TRY(check_field(g, x, "x"));
        TM_TRY(same_prec(out, x, "tm_dd_dslash"));
    } else {
        x = nullptr;
    }
    if (!has_tw) memset(&tw, 0, sizeof(tw));
    const Twist<double> Ri = make_twist(g, TW_RINV, dagger);
    const Twist<double> *pro = twist_in ? &Ri : nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const int st = g->X1h * g->p.L[1] * g->p.L[2], Lt = g->p.L[3];
    if (region != TM_DD_BOUNDARY && Lt > 2)  // interior slices: the handle's tuned launch form over a site range
        TM_TRY(dslash_launch(g, out, in, x, out_parity, dagger, epi, coef, has_tw ? &tw : nullptr, pro, s, nullptr, 1,
                             st, (Lt - 2) * st));
    if (region == TM_DD_INTERIOR) return TM_OK;
    if (in->prec == TM_PREC_F64)
        return dd_call<double>(g, out, in, x, out_parity, dagger, epi, coef, tw, pro, ghost_prev, ghost_next, nullptr,
                               nullptr, s);
    return dd_call<float>(g, out, in, x, out_parity, dagger, epi, coef, tw, pro, ghost_prev, ghost_next, nullptr, nullptr, s);
}

}  // extern "C"

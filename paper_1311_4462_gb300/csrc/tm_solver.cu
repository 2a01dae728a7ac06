// tm_solver.cu -- CG on the normal equations of the even-even operator (sec. 2.2:
// DIRECT_PC solve with NORMOP CG), in FP64, and the mixed-precision reliable-update CG
// (the double-single / double-half solver of sec. 3): the sloppy iteration runs the fused
// operator and BLAS in FP32 or FP16 storage; the solution accumulation, the true residual
// and the stopping test run in FP64.
//
// Scalars (alpha, beta, |r|^2) live in the handle's device scalar table and are produced by
// the reductions' last block, so an iteration enqueues without host round trips; the host
// reads |r|^2 once per iteration to decide convergence and reliable updates.
#include <math.h>
#include <string.h>

#include <chrono>

#include "tm_blas.cuh"
#include "tm_internal.h"

namespace tmk {

__global__ void k_scalar_beta(double *S, int nrhs, const int *active)
{
    const int c = threadIdx.x;
    if (c >= nrhs) return;
    if (active && !active[c]) return;
    const double rr = S[SL_RR * TM_MAX_RHS + c], rn = S[SL_RRNEW * TM_MAX_RHS + c];
    S[SL_BETA * TM_MAX_RHS + c] = rr != 0.0 ? rn / rr : 0.0;
    S[SL_RR * TM_MAX_RHS + c] = rn;
}

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

struct Carve {
    char *base;
    size_t off, cap;
    bool ok = true;
    tm_field take(const tm_gauge *g, int prec)
    {
        tm_field f;
        memset(&f, 0, sizeof(f));
        size_t d, n;
        tm_field_bytes(g, prec, 1, &d, &n);
        f.prec = prec;
        f.nrhs = 1;
        f.data = base ? base + off : nullptr;
        off += align256(d);
        if (n) {
            f.norm = base ? reinterpret_cast<float *>(base + off) : nullptr;
            off += align256(n);
        }
        if (off > cap) ok = false;
        return f;
    }
};

static int true_prec_of(const tm_solver_params *sp)
{
    return sp->true_prec == TM_PREC_DF64 ? TM_PREC_DF64 : TM_PREC_F64;
}

static size_t workspace_need(const tm_gauge *g, const tm_solver_params *sp)
{
    Carve c{nullptr, 0, (size_t)-1};
    const int tp = true_prec_of(sp);
    for (int i = 0; i < 6; i++) c.take(g, tp);
    if (tp == TM_PREC_DF64)
        for (int i = 0; i < 2; i++) c.take(g, tp);  // x and b in DF64
    if (sp->solver == TM_SOLVER_MIXED_CG) {
        for (int i = 0; i < 5; i++) c.take(g, sp->sloppy_prec);
        c.take(g, TM_PREC_F32);
    }
    return c.off;
}

class Solver {
  public:
    const tm_gauge *g;
    const tm_solver_params *sp;
    cudaStream_t s;
    double *S;  // device scalar table
    double *H;  // pinned host mirror

    tm_status site(int op, FieldRef A, FieldRef B, FieldRef C, FieldRef D, SVal ca, SVal cb, int reduce, int fin,
                   int slot)
    {
        SiteOpArgs a;
        memset(&a, 0, sizeof(a));
        a.op = op;
        a.reduce = reduce;
        a.A = A;
        a.B = B;
        a.C = C;
        a.D = D;
        a.ca = ca;
        a.cb = cb;
        a.red.scalars = S;
        a.red.fin = fin;
        a.red.slot = slot;
        return cuda_check(launch_site_op(g, a, 1, s), "site op");
    }
    tm_status norm2(const tm_field *x, int slot)
    {
        return site(OP_NORM, fref(x), fnone(), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, slot);
    }
    tm_status copy(const tm_field *dst, const tm_field *src)
    {
        return site(OP_COPY, fref(src), fnone(), fref(dst), fnone(), sv(1), sv(0), 0, 0, 0);
    }
    // C = ca A + cb B
    tm_status axpby(const tm_field *C, SVal ca, const tm_field *A, SVal cb, const tm_field *B, int reduce = 0,
                    int fin = FIN_STORE, int slot = SL_TMP0)
    {
        return site(OP_AXPBY, fref(A), B ? fref(B) : fnone(), fref(C), fnone(), ca, cb, reduce, fin, slot);
    }
    tm_status read(int slot, double *v)
    {
        tm_status st = cuda_check(cudaMemcpyAsync(H, S + slot * TM_MAX_RHS, sizeof(double), cudaMemcpyDeviceToHost, s),
                                  "scalar readback");
        if (st != TM_OK) return st;
        st = cuda_check(cudaStreamSynchronize(s), "solver sync");
        *v = H[0];
        return st;
    }
    tm_status zero(const tm_field *f)
    {
        size_t d, n;
        tm_field_bytes(g, f->prec, 1, &d, &n);
        tm_status st = cuda_check(cudaMemsetAsync(f->data, 0, d, s), "memset");
        if (st == TM_OK && n) st = cuda_check(cudaMemsetAsync(f->norm, 0, n, s), "memset");
        return st;
    }
    // r = A^dag (b - A x) and |r|^2 in `slot`, in the precision of the fields (A = M_pc, or M_pc^dag
    // when dagger): the residual of the normal equations A^dag A x = A^dag b without their
    // right-hand side, two operator applications like A^dag A x itself; te is overwritten.
    tm_status true_residual(const tm_field *r, const tm_field *x, const tm_field *b, const tm_field *te,
                            const tm_field *to, int slot)
    {
        tm_status st = precond_core(g, te, x, to, sp->pc, sp->dagger, s, nullptr, 1);  // te = A x
        if (st == TM_OK) st = axpby(te, sv(1.0), b, sv(-1.0), te);                      // te = b - A x
        if (st == TM_OK) st = adjoint_core(g, r, te, to, sp->pc, sp->dagger, s);        // r = A^dag te
        if (st == TM_OK) st = norm2(r, slot);
        return st;
    }
    // out = A^dag A in with A = M_pc (or M_pc^dag when dagger)
    tm_status normal_op(const tm_field *out, const tm_field *in, const tm_field *te, const tm_field *to)
    {
        return normal_core(g, out, in, te, to, sp->pc, sp->dagger, s, nullptr, 1);
    }
    // out = A^dag A p and alpha = |r|^2 / <p, A^dag A p> in the scalar table.  Where the operator's
    // launch form allows it, <p, A^dag A p> = |A p|^2 is summed in the epilogue of the launch that
    // writes A p (sec. 2.1's local operations merged into the dslash kernels), which saves the
    // separate pass over p and A^dag A p.
    tm_status normal_op_alpha(const tm_field *out, const tm_field *p, const tm_field *te, const tm_field *to)
    {
        if (!normal_red_supported(g, p->prec, sp->dagger)) {
            tm_status st = normal_op(out, p, te, to);
            if (st != TM_OK) return st;
            return site(OP_DOT, fref(p), fref(out), fnone(), fnone(), sv(0), sv(0), 1, FIN_ALPHA, 0);
        }
        RedArgs r = red_args(FIN_ALPHA, 0);
        return normal_core(g, out, p, te, to, sp->pc, sp->dagger, s, nullptr, 1, &r);
    }
    // r -= alpha A^dag A p with alpha = |r|^2 / |A p|^2 and |r|^2 in SL_RRNEW, A^dag A p never stored:
    // the update and its norm are computed in the epilogue of the launch that produces A^dag A p
    // (normal_rupd_core).  Available where normal_op_alpha fuses its reduction, for A = M_pc.
    bool rupd_supported(int prec) const { return !sp->dagger && normal_red_supported(g, prec, 0); }
    tm_status normal_rupd(const tm_field *r, const tm_field *p, const tm_field *te, const tm_field *to)
    {
        RedArgs ra = red_args(FIN_ALPHA, 0), rr = red_args(FIN_STORE, SL_RRNEW);
        return normal_rupd_core(g, r, p, te, to, sp->pc, s, &ra, &rr, S + SL_ALPHA * TM_MAX_RHS);
    }
    RedArgs red_args(int fin, int slot) const
    {
        RedArgs r;
        memset(&r, 0, sizeof(r));
        r.partials = reinterpret_cast<double *>(reinterpret_cast<char *>(g->scratch) + SCRATCH_PARTIALS_OFF);
        r.counter = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(g->scratch) + SCRATCH_COUNTER_OFF);
        r.scalars = S;
        r.fin = fin;
        r.slot = slot;
        return r;
    }
};

static tm_status check_solver_params(const tm_gauge *g, const tm_solver_params *sp)
{
    if (!g || !sp) { set_error("tm_solve: null handle or params"); return TM_ERR_ARG; }
    if (sp->solver != TM_SOLVER_CG && sp->solver != TM_SOLVER_MIXED_CG) { set_error("unknown solver"); return TM_ERR_ARG; }
    if (sp->solution != TM_SOLUTION_MAT && sp->solution != TM_SOLUTION_MATDAG_MAT) {
        set_error("unknown solution type");
        return TM_ERR_ARG;
    }
    if (sp->pc != TM_PC_ASYM && sp->pc != TM_PC_SYM) { set_error("unknown pc"); return TM_ERR_ARG; }
    if (!(sp->tol > 0.0) || sp->maxiter < 1) { set_error("tol must be > 0 and maxiter >= 1"); return TM_ERR_ARG; }
    if (sp->true_prec != 0 && sp->true_prec != TM_PREC_F64 && sp->true_prec != TM_PREC_DF64) {
        set_error("true_prec must be TM_PREC_F64 or TM_PREC_DF64");
        return TM_ERR_ARG;
    }
    if (sp->solver == TM_SOLVER_MIXED_CG) {
        if (sp->sloppy_prec != TM_PREC_F32 && sp->sloppy_prec != TM_PREC_F16) {
            set_error("sloppy_prec must be TM_PREC_F32 or TM_PREC_F16");
            return TM_ERR_ARG;
        }
        if (!(sp->delta > 0.0 && sp->delta < 1.0)) { set_error("delta must be in (0, 1)"); return TM_ERR_ARG; }
    }
    return TM_OK;
}

#define TRY(x)                      \
    do {                            \
        st = (x);                   \
        if (st != TM_OK) goto done; \
    } while (0)

static tm_status solve(const tm_gauge *g, const tm_field *x, const tm_field *b, const tm_solver_params *sp,
                       tm_solver_stats *stats, void *ws, size_t ws_bytes, cudaStream_t s)
{
    auto t0 = std::chrono::steady_clock::now();
    tm_status st = TM_OK;
    Solver sv_;
    sv_.g = g;
    sv_.sp = sp;
    sv_.s = s;
    sv_.S = g->scratch;
    sv_.H = g->host_scalars;
    Solver &V = sv_;
    Carve c{reinterpret_cast<char *>(ws), 0, ws_bytes};
    const int tp = true_prec_of(sp);
    tm_field r = c.take(g, tp), p = c.take(g, tp), Ap = c.take(g, tp);
    tm_field te = c.take(g, tp), to = c.take(g, tp), bh = c.take(g, tp);
    tm_field xt{}, bt{};
    if (tp == TM_PREC_DF64) {
        xt = c.take(g, tp);
        bt = c.take(g, tp);
    }
    const bool mixed = sp->solver == TM_SOLVER_MIXED_CG;
    // The mixed solver with b on the right of M_pc x = b recomputes its true residuals as
    // A^dag (b - A x), so A^dag b only starts the sloppy iteration and normalises the stopping test;
    // with binary32 sloppy fields it is computed in binary32 (the norm to about 1e-7 relative, which
    // moves the stopping threshold by that fraction of itself), two FP64 launches fewer per solve.
    const bool mat_mixed = mixed && sp->solution == TM_SOLUTION_MAT;
    const bool sloppy_src = mat_mixed && sp->sloppy_prec == TM_PREC_F32;
    tm_field rs{}, ps{}, Aps{}, tes{}, tos{}, xs{};
    if (mixed) {
        rs = c.take(g, sp->sloppy_prec);
        ps = c.take(g, sp->sloppy_prec);
        Aps = c.take(g, sp->sloppy_prec);
        tes = c.take(g, sp->sloppy_prec);
        tos = c.take(g, sp->sloppy_prec);
        xs = c.take(g, TM_PREC_F32);
    }
    if (!c.ok) {
        set_error("tm_solve: workspace of %zu bytes is smaller than the %zu needed", ws_bytes, c.off);
        return TM_ERR_NOMEM;
    }
    double bb = 0, rr = 0, r2 = 0;
    int it = 0, nrel = 0;
    const double tol2 = sp->tol * sp->tol;
    const tm_field *x_user = x;
    const tm_field *bhat = nullptr;
    if (tp == TM_PREC_DF64) {
        // the iteration works on DF64 copies of b and x; x is converted back at the end
        TRY(V.copy(&bt, b));
        if (sp->use_x0) TRY(V.copy(&xt, x));
        b = &bt;
        x = &xt;
    }
    bhat = b;
    // right-hand side of the normal equations
    if (sloppy_src) {
        TRY(V.copy(&tes, b));
        TRY(adjoint_core(g, &rs, &tes, &tos, sp->pc, sp->dagger, s));  // rs = A^dag b in binary32
        TRY(V.norm2(&rs, SL_TMP0));
    } else {
        if (sp->solution == TM_SOLUTION_MAT) {
            TRY(tm_precond_op(g, &bh, b, &to, sp->pc, !sp->dagger, s));  // bhat = A^dag b
            bhat = &bh;
        }
        TRY(V.norm2(bhat, SL_TMP0));
    }
    TRY(V.read(SL_TMP0, &bb));
    if (!isfinite(bb)) { set_error("tm_solve: non-finite source"); st = TM_ERR_NAN; goto done; }
    if (bb == 0.0) {
        TRY(V.zero(x));
        goto done;
    }
    // r = bhat - A^dag A x
    if (sp->use_x0) {
        if (mat_mixed) {
            TRY(V.true_residual(&r, x, b, &te, &to, SL_RR));
        } else {
            TRY(V.normal_op(&Ap, x, &te, &to));
            TRY(V.axpby(&r, sv(1.0), bhat, sv(-1.0), &Ap, 1, FIN_STORE, SL_RR));
        }
        TRY(V.read(SL_RR, &r2));
    } else {
        TRY(V.zero(x));
        if (sloppy_src) {
            r2 = bb;  // r = A^dag b, held in binary32 by rs
        } else {
            TRY(V.copy(&r, bhat));
            TRY(V.norm2(&r, SL_RR));
            TRY(V.read(SL_RR, &r2));
        }
    }

    if (!mixed) {
        // CG on the recursively updated residual; when it reaches tol the true residual is
        // recomputed, and CG restarts from it (at most 4 times) if rounding left it above tol.
        for (int restart = 0; restart < 5 && r2 > tol2 * bb && it < sp->maxiter; restart++) {
            if (restart > 0) nrel++;
            TRY(V.copy(&p, &r));
            rr = r2;
            while (rr > tol2 * bb && it < sp->maxiter) {
                TRY(V.normal_op_alpha(&Ap, &p, &te, &to));
                TRY(V.site(OP_CG_UPDATE, fref(&p), fref(&r), fref(x), fref(&Ap), sslot(SL_ALPHA, 1.0), sv(0), 1,
                           FIN_BETA, 0));
                TRY(V.read(SL_RRNEW, &rr));
                it++;
                if (!isfinite(rr)) {
                    set_error("tm_solve: non-finite residual at iteration %d", it);
                    st = TM_ERR_NAN;
                    goto done;
                }
                if (rr <= tol2 * bb) break;
                TRY(V.axpby(&p, sv(1.0), &r, sslot(SL_BETA, 1.0), &p));  // p = r + beta p
            }
            // true residual r = bhat - A^dag A x, FP64; SL_RR = |r|^2 for the next restart
            TRY(V.normal_op(&Ap, x, &te, &to));
            TRY(V.axpby(&r, sv(1.0), bhat, sv(-1.0), &Ap, 1, FIN_STORE, SL_RR));
            TRY(V.read(SL_RR, &r2));
        }
    } else {
        // sloppy copies: rs = r (already in place when the source was computed in binary32), p = rs,
        // xs = 0; SL_RR = |rs|^2
        if (!sloppy_src || sp->use_x0) TRY(V.copy(&rs, &r));
        TRY(V.copy(&ps, &rs));
        TRY(V.zero(&xs));
        TRY(V.norm2(&rs, SL_RR));
        double maxr = sqrt(r2);
        bool converged = r2 <= tol2 * bb;
        const bool rupd = V.rupd_supported(sp->sloppy_prec);
        while (!converged && it < sp->maxiter) {
            // r_s -= alpha A p with |r_s|^2, in the epilogue of the last hopping launch where the
            // launch form allows it (A p is then never stored), else as a pass of its own; the
            // increment x_s += alpha p waits for beta and shares the pass of the search-direction
            // update (one field pass fewer per iteration)
            if (rupd) {
                TRY(V.normal_rupd(&rs, &ps, &tes, &tos));
            } else {
                TRY(V.normal_op_alpha(&Aps, &ps, &tes, &tos));
                TRY(V.site(OP_R_UPDATE, fref(&rs), fref(&rs), fnone(), fref(&Aps), sslot(SL_ALPHA, 1.0), sv(0), 1,
                           FIN_STORE, SL_RRNEW));
            }
            TRY(V.read(SL_RRNEW, &rr));
            it++;
            if (!isfinite(rr)) { set_error("tm_solve: non-finite residual at iteration %d", it); st = TM_ERR_NAN; goto done; }
            const double rn = sqrt(rr);
            if (rn > maxr) maxr = rn;
            const bool update = rn < sp->delta * maxr || rr <= tol2 * bb || it == sp->maxiter;
            if (!update) {
                k_scalar_beta<<<1, 32, 0, s>>>(V.S, 1, nullptr);
                TRY(cuda_check(cudaGetLastError(), "beta"));
                // x_s += alpha p ; p = r_s + beta p
                TRY(V.site(OP_XP_UPDATE, fref(&ps), fnone(), fref(&xs), fref(&rs), sslot(SL_ALPHA, 1.0),
                           sslot(SL_BETA, 1.0), 0, 0, 0));
                continue;
            }
            TRY(V.axpby(&xs, sslot(SL_ALPHA, 1.0), &ps, sv(1.0), &xs));  // x_s += alpha p
            {
                // reliable update: fold the sloppy solution into x, recompute the true residual in FP64
                TRY(V.axpby(x, sv(1.0), &xs, sv(1.0), x));
                TRY(V.zero(&xs));
                if (mat_mixed) {
                    TRY(V.true_residual(&r, x, b, &te, &to, SL_TMP0));
                } else {
                    TRY(V.normal_op(&Ap, x, &te, &to));
                    TRY(V.axpby(&r, sv(1.0), bhat, sv(-1.0), &Ap, 1, FIN_STORE, SL_TMP0));
                }
                TRY(V.read(SL_TMP0, &r2));
                nrel++;
                if (!isfinite(r2)) { set_error("tm_solve: non-finite true residual"); st = TM_ERR_NAN; goto done; }
                if (r2 <= tol2 * bb) { converged = true; break; }
                TRY(V.copy(&rs, &r));
                TRY(V.norm2(&rs, SL_RRNEW));
                maxr = sqrt(r2);
            }
            k_scalar_beta<<<1, 32, 0, s>>>(V.S, 1, nullptr);
            TRY(cuda_check(cudaGetLastError(), "beta"));
            TRY(V.axpby(&ps, sv(1.0), &rs, sslot(SL_BETA, 1.0), &ps));  // p = rs + beta p
        }
    }
    // r2 is the FP64 true residual of the final x on every path above (the FP64 loop ends with a
    // recomputation, the mixed loop with a reliable update), so it is not recomputed here.
    if (stats) {
        stats->true_residual = sqrt(r2 / bb);
        stats->pc_residual = -1.0;
    }
    if (stats && sp->want_pc_residual && sp->solution == TM_SOLUTION_MAT) {
        double b2, e2;
        TRY(tm_precond_op(g, &te, x, &to, sp->pc, sp->dagger, s));  // M_pc x
        TRY(V.axpby(&te, sv(1.0), b, sv(-1.0), &te, 1, FIN_STORE, SL_TMP0));
        TRY(V.read(SL_TMP0, &e2));
        TRY(V.norm2(b, SL_TMP1));
        TRY(V.read(SL_TMP1, &b2));
        stats->pc_residual = sqrt(e2 / b2);
    }
    if (r2 > tol2 * bb) {
        set_error("tm_solve: no convergence after %d iterations (true residual %.3e)", it, sqrt(r2 / bb));
        st = TM_ERR_NOCONV;
    }
done:
    if (x != x_user && (st == TM_OK || st == TM_ERR_NOCONV)) {
        const tm_status cst = V.copy(x_user, x);  // DF64 -> FP64
        if (st == TM_OK) st = cst;
    }
    if (st != TM_ERR_ARG && st != TM_ERR_NOMEM && st != TM_ERR_CUDA && g->fused_sync && (g->fused[0] || g->fused[1])) {
        // the fused operator may have run: a bounded wait that gave up left some output sites
        // unwritten, so the solution (and a residual computed from them) cannot be trusted
        const tm_status dst = tm_device_status(g, s);
        if (dst != TM_OK) st = dst;
    }
    if (stats) {
        stats->iterations = it;
        stats->reliable_updates = nrel;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return st;
}

}  // namespace tmk

using namespace tmk;

extern "C" {

tm_status tm_solve_workspace_bytes(const tm_gauge *g, const tm_solver_params *sp, size_t *bytes)
{
    tm_status st = check_solver_params(g, sp);
    if (st != TM_OK) return st;
    if (!bytes) { set_error("null output"); return TM_ERR_ARG; }
    *bytes = workspace_need(g, sp);
    return TM_OK;
}

tm_status tm_solve(const tm_gauge *g, const tm_field *x_e, const tm_field *b_e, const tm_solver_params *sp,
                   tm_solver_stats *stats, void *workspace, size_t workspace_bytes, void *stream)
{
    TM_NVTX("tm_solve");
    tm_status st = check_solver_params(g, sp);
    if (st != TM_OK) return st;
    if (!x_e || !b_e || !workspace) { set_error("tm_solve: null field or workspace"); return TM_ERR_ARG; }
    if (x_e->prec != TM_PREC_F64 || b_e->prec != TM_PREC_F64 || x_e->nrhs != 1 || b_e->nrhs != 1) {
        set_error("tm_solve: x and b must be single-RHS FP64 fields");
        return TM_ERR_ARG;
    }
    if (x_e->data == b_e->data) { set_error("tm_solve: x must not alias b"); return TM_ERR_ARG; }
    if (g->dd) { set_error("tm_solve: the handle holds one time slab of a decomposed lattice"); return TM_ERR_ARG; }
    if (((uintptr_t)workspace & 255) != 0) { set_error("tm_solve: workspace must be 256-byte aligned"); return TM_ERR_ARG; }
    if (stats) memset(stats, 0, sizeof(*stats));
    return solve(g, x_e, b_e, sp, stats, workspace, workspace_bytes, (cudaStream_t)stream);
}

tm_status tm_norm2(const tm_gauge *g, const tm_field *x, double *out, void *stream)
{
    TM_NVTX("tm_norm2");
    if (!g || !x || !x->data || !out) { set_error("tm_norm2: null argument"); return TM_ERR_ARG; }
    Solver V;
    V.g = g;
    V.sp = nullptr;
    V.s = (cudaStream_t)stream;
    V.S = g->scratch;
    V.H = g->host_scalars;
    tm_status st = V.site(OP_NORM, fref(x), fnone(), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, SL_TMP2);
    if (st != TM_OK) return st;
    return V.read(SL_TMP2, out);
}

tm_status tm_axpby(const tm_gauge *g, const tm_field *out, double a, const tm_field *x, double b, const tm_field *y,
                   void *stream)
{
    TM_NVTX("tm_axpby");
    if (!g || !out || !x || !out->data || !x->data) { set_error("tm_axpby: null argument"); return TM_ERR_ARG; }
    const bool hasy = y != nullptr;
    if (hasy && !y->data) { set_error("tm_axpby: null y data"); return TM_ERR_ARG; }
    if (prec_index(x->prec) < 0 || prec_index(out->prec) < 0 || (hasy && prec_index(y->prec) < 0)) {
        set_error("tm_axpby: unknown precision");
        return TM_ERR_ARG;
    }
    if ((out->prec == TM_PREC_F16 && !out->norm) || (x->prec == TM_PREC_F16 && !x->norm) ||
        (hasy && y->prec == TM_PREC_F16 && !y->norm)) {
        set_error("tm_axpby: FP16 fields need their norm arrays");
        return TM_ERR_ARG;
    }
    if (out->nrhs != x->nrhs || (hasy && y->nrhs != x->nrhs) || x->nrhs < 1 || x->nrhs > 65535) {
        set_error("tm_axpby: fields must share nrhs in [1, 65535]");
        return TM_ERR_ARG;
    }
    if (!isfinite(a) || !isfinite(b)) { set_error("tm_axpby: coefficients must be finite"); return TM_ERR_ARG; }
    SiteOpArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.op = OP_AXPBY;
    sa.A = fref(x);
    sa.B = hasy ? fref(y) : fnone();
    sa.C = fref(out);
    sa.ca = sv(a);
    sa.cb = sv(b);
    const cudaError_t e = launch_site_op(g, sa, x->nrhs, (cudaStream_t)stream);
    if (e == cudaErrorNotSupported) {
        set_error("tm_axpby: precision combination out %d, x %d, y %d is not offered", out->prec, x->prec,
                  hasy ? y->prec : x->prec);
        return TM_ERR_ARG;
    }
    return cuda_check(e, "tm_axpby");
}

tm_status tm_dot(const tm_gauge *g, const tm_field *a, const tm_field *b, double *re_out, void *stream)
{
    TM_NVTX("tm_dot");
    if (!g || !a || !b || !a->data || !b->data || !re_out) { set_error("tm_dot: null argument"); return TM_ERR_ARG; }
    Solver V;
    V.g = g;
    V.sp = nullptr;
    V.s = (cudaStream_t)stream;
    V.S = g->scratch;
    V.H = g->host_scalars;
    tm_status st = V.site(OP_DOT, fref(a), fref(b), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, SL_TMP2);
    if (st != TM_OK) return st;
    return V.read(SL_TMP2, re_out);
}

}  // extern "C"

// ============================================================================ multi-RHS CG
// All right-hand sides iterate together (one multi-RHS operator launch per factor, one BLAS
// launch per step with one column per source, per-source alpha/beta/|r|^2 in the scalar
// table).  Reliable updates are taken for all active sources at once when any source asks
// for one; a source whose FP64 true residual meets the tolerance is dropped from the active
// list, so later launches skip it.  With use_graph the sloppy iteration is captured once per
// active-set size as a CUDA graph on an internal stream and replayed.
namespace tmk {

static size_t multi_workspace_need(const tm_gauge *g, const tm_solver_params *sp, int nrhs)
{
    size_t need = 0, d, n;
    const int tp = true_prec_of(sp);
    const int ps = sp->solver == TM_SOLVER_MIXED_CG ? sp->sloppy_prec : tp;
    const int px = sp->solver == TM_SOLVER_MIXED_CG ? TM_PREC_F32 : tp;
    tm_field_bytes(g, tp, nrhs, &d, &n);
    need += (tp == TM_PREC_DF64 ? 7 : 5) * align256(d);
    tm_field_bytes(g, ps, nrhs, &d, &n);
    need += 5 * (align256(d) + align256(n));
    tm_field_bytes(g, px, nrhs, &d, &n);
    need += align256(d) + align256(n);
    need += 2 * align256(TM_MAX_RHS * sizeof(int));
    return need;
}

struct MultiCarve {
    char *base;
    size_t off;
    tm_field take(const tm_gauge *g, int prec, int nrhs)
    {
        tm_field f;
        memset(&f, 0, sizeof(f));
        size_t d, n;
        tm_field_bytes(g, prec, nrhs, &d, &n);
        f.prec = prec;
        f.nrhs = nrhs;
        f.data = base + off;
        off += align256(d);
        if (n) {
            f.norm = reinterpret_cast<float *>(base + off);
            off += align256(n);
        }
        return f;
    }
    int *ints()
    {
        int *p = reinterpret_cast<int *>(base + off);
        off += align256(TM_MAX_RHS * sizeof(int));
        return p;
    }
};

class MultiSolver {
  public:
    const tm_gauge *g;
    const tm_solver_params *sp;
    cudaStream_t s;
    int nrhs;
    double *S, *H;
    int *d_list, *d_mask, *h_ints;  // device active list / mask, pinned host staging

    tm_status site(int op, FieldRef A, FieldRef B, FieldRef C, FieldRef D, SVal ca, SVal cb, int reduce, int fin,
                   int slot, bool masked = true)
    {
        SiteOpArgs a;
        memset(&a, 0, sizeof(a));
        a.op = op;
        a.reduce = reduce;
        a.A = A;
        a.B = B;
        a.C = C;
        a.D = D;
        a.ca = ca;
        a.cb = cb;
        a.red.scalars = S;
        a.red.fin = fin;
        a.red.slot = slot;
        a.red.active = masked ? d_mask : nullptr;
        return cuda_check(launch_site_op(g, a, nrhs, s), "site op");
    }
    tm_status read_col(int slot, double *out)
    {
        tm_status st = cuda_check(
            cudaMemcpyAsync(H, S + slot * TM_MAX_RHS, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s), "readback");
        if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "sync");
        if (st == TM_OK) memcpy(out, H, nrhs * sizeof(double));
        return st;
    }
    // upload the active set: list of indices and a 0/1 mask
    tm_status set_active(const bool *act, int *nact)
    {
        int k = 0;
        for (int r = 0; r < nrhs; r++)
            if (act[r]) h_ints[k++] = r;
        for (int r = 0; r < nrhs; r++) h_ints[TM_MAX_RHS + r] = act[r] ? 1 : 0;
        *nact = k;
        tm_status st = cuda_check(cudaMemcpyAsync(d_list, h_ints, TM_MAX_RHS * sizeof(int), cudaMemcpyHostToDevice, s),
                                  "active list");
        if (st == TM_OK)
            st = cuda_check(cudaMemcpyAsync(d_mask, h_ints + TM_MAX_RHS, TM_MAX_RHS * sizeof(int),
                                            cudaMemcpyHostToDevice, s), "active mask");
        // the staging buffer is reused: wait until both copies have read it
        if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "sync");
        return st;
    }
    tm_status normal_op(const tm_field *out, const tm_field *in, const tm_field *te, const tm_field *to, int nact)
    {
        // every source active: no list (the operator may then pair sources, tune entry m:16)
        return normal_core(g, out, in, te, to, sp->pc, sp->dagger, s, nact == nrhs ? nullptr : d_list, nact);
    }
};

#define MTRY(x)                      \
    do {                             \
        st = (x);                    \
        if (st != TM_OK) goto mdone; \
    } while (0)

static tm_status solve_multi(const tm_gauge *g, const tm_field *x, const tm_field *b, const tm_solver_params *sp,
                             tm_solver_stats *stats, void *ws, cudaStream_t user_stream)
{
    auto t0 = std::chrono::steady_clock::now();
    const int nrhs = x->nrhs;
    const bool mixed = sp->solver == TM_SOLVER_MIXED_CG;
    const int tp = true_prec_of(sp);
    const int ps = mixed ? sp->sloppy_prec : tp;
    const int px = mixed ? TM_PREC_F32 : tp;
    MultiCarve c{reinterpret_cast<char *>(ws), 0};
    tm_field r = c.take(g, tp, nrhs), Ap = c.take(g, tp, nrhs), te = c.take(g, tp, nrhs);
    tm_field to = c.take(g, tp, nrhs), bh = c.take(g, tp, nrhs);
    tm_field xt{}, bt{};
    if (tp == TM_PREC_DF64) {
        xt = c.take(g, tp, nrhs);
        bt = c.take(g, tp, nrhs);
    }
    const tm_field *x_user = x;
    tm_field rs = c.take(g, ps, nrhs), pp = c.take(g, ps, nrhs), Aps = c.take(g, ps, nrhs);
    tm_field tes = c.take(g, ps, nrhs), tos = c.take(g, ps, nrhs), xs = c.take(g, px, nrhs);
    MultiSolver V;
    V.g = g;
    V.sp = sp;
    V.nrhs = nrhs;
    V.S = g->scratch;
    V.H = g->host_scalars;
    V.h_ints = reinterpret_cast<int *>(g->host_scalars + 256);
    V.d_list = c.ints();
    V.d_mask = c.ints();
    // work on a private stream (graph capture needs one), ordered after the caller's work
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_nact = -1;
    tm_status st = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    if (st != TM_OK) return st;
    V.s = s;
    double bb[TM_MAX_RHS], r2[TM_MAX_RHS], rr[TM_MAX_RHS], maxr[TM_MAX_RHS];
    bool act[TM_MAX_RHS];
    int conv_it[TM_MAX_RHS], nact = 0, it = 0, nrel = 0;
    const double tol2 = sp->tol * sp->tol;
    const double delta = mixed ? sp->delta : 0.0;
    const tm_field *bhat = b;
    for (int k = 0; k < nrhs; k++) {
        act[k] = true;
        conv_it[k] = -1;
    }
    MTRY(cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event"));
    MTRY(cuda_check(cudaEventRecord(ev, user_stream), "event"));
    MTRY(cuda_check(cudaStreamWaitEvent(s, ev, 0), "event wait"));
    MTRY(V.set_active(act, &nact));
    if (tp == TM_PREC_DF64) {
        // DF64 copies of b (and the initial x); x is converted back at the end
        MTRY(V.site(OP_COPY, fref(b), fnone(), fref(&bt), fnone(), sv(1), sv(0), 0, 0, 0, false));
        if (sp->use_x0) MTRY(V.site(OP_COPY, fref(x), fnone(), fref(&xt), fnone(), sv(1), sv(0), 0, 0, 0, false));
        b = &bt;
        x = &xt;
        bhat = b;
    }
    if (sp->solution == TM_SOLUTION_MAT) {
        MTRY(precond_core(g, &bh, b, &to, sp->pc, !sp->dagger, s, V.d_list, nact));  // bhat = A^dag b
        bhat = &bh;
    }
    MTRY(V.site(OP_NORM, fref(bhat), fnone(), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, SL_TMP0, false));
    MTRY(V.read_col(SL_TMP0, bb));
    for (int k = 0; k < nrhs; k++) {
        if (!isfinite(bb[k])) { set_error("tm_solve_multi: non-finite source %d", k); st = TM_ERR_NAN; goto mdone; }
        act[k] = bb[k] > 0.0;
        if (!act[k]) conv_it[k] = 0;  // a zero source has the zero solution
    }
    // x = 0 (or the given guess), r = bhat - A^dag A x
    if (sp->use_x0) {
        MTRY(V.set_active(act, &nact));
        if (nact) MTRY(V.normal_op(&Ap, x, &te, &to, nact));
        MTRY(V.site(OP_AXPBY, fref(bhat), fref(&Ap), fref(&r), fnone(), sv(1.0), sv(-1.0), 1, FIN_STORE, SL_TMP0,
                    false));
    } else {
        size_t d, n;
        tm_field_bytes(g, tp, nrhs, &d, &n);
        MTRY(cuda_check(cudaMemsetAsync(x->data, 0, d, s), "memset"));
        MTRY(V.site(OP_COPY, fref(bhat), fnone(), fref(&r), fnone(), sv(1), sv(0), 0, 0, 0, false));
        MTRY(V.site(OP_NORM, fref(&r), fnone(), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, SL_TMP0, false));
    }
    MTRY(V.read_col(SL_TMP0, r2));
    for (int k = 0; k < nrhs; k++) {
        if (act[k] && r2[k] <= tol2 * bb[k]) {
            act[k] = false;
            conv_it[k] = 0;
        }
        maxr[k] = sqrt(r2[k]);
    }
    MTRY(V.set_active(act, &nact));
    if (nact) {
        {
            size_t d, n;
            tm_field_bytes(g, px, nrhs, &d, &n);
            MTRY(cuda_check(cudaMemsetAsync(xs.data, 0, d, s), "memset"));
        }
        MTRY(V.site(OP_COPY, fref(&r), fnone(), fref(&rs), fnone(), sv(1), sv(0), 0, 0, 0));
        MTRY(V.site(OP_COPY, fref(&rs), fnone(), fref(&pp), fnone(), sv(1), sv(0), 0, 0, 0));
        MTRY(V.site(OP_NORM, fref(&rs), fnone(), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, SL_RR));
    }
    while (nact > 0 && it < sp->maxiter) {
        // ---- sloppy iteration (optionally one replayed graph): Ap = A p, alpha, x += a p, r -= a Ap, |r|^2
        if (sp->use_graph) {
            if (graph_nact != nact) {
                if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
                if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
                MTRY(cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture"));
                tm_status cst = V.normal_op(&Aps, &pp, &tes, &tos, nact);
                if (cst == TM_OK)
                    cst = V.site(OP_DOT, fref(&pp), fref(&Aps), fnone(), fnone(), sv(0), sv(0), 1, FIN_ALPHA, 0);
                if (cst == TM_OK)
                    cst = V.site(OP_CG_UPDATE, fref(&pp), fref(&rs), fref(&xs), fref(&Aps), sslot(SL_ALPHA, 1.0), sv(0),
                                 1, FIN_STORE, SL_RRNEW);
                cudaError_t ce = cudaStreamEndCapture(s, &graph);
                MTRY(cst);
                MTRY(cuda_check(ce, "end capture"));
                MTRY(cuda_check(cudaGraphInstantiate(&gexec, graph, 0), "graph instantiate"));
                graph_nact = nact;
            }
            MTRY(cuda_check(cudaGraphLaunch(gexec, s), "graph launch"));
        } else {
            MTRY(V.normal_op(&Aps, &pp, &tes, &tos, nact));
            MTRY(V.site(OP_DOT, fref(&pp), fref(&Aps), fnone(), fnone(), sv(0), sv(0), 1, FIN_ALPHA, 0));
            MTRY(V.site(OP_CG_UPDATE, fref(&pp), fref(&rs), fref(&xs), fref(&Aps), sslot(SL_ALPHA, 1.0), sv(0), 1,
                        FIN_STORE, SL_RRNEW));
        }
        MTRY(V.read_col(SL_RRNEW, rr));
        it++;
        bool update = (it == sp->maxiter);
        for (int k = 0; k < nrhs; k++) {
            if (!act[k]) continue;
            if (!isfinite(rr[k])) {
                set_error("tm_solve_multi: non-finite residual for source %d at iteration %d", k, it);
                st = TM_ERR_NAN;
                goto mdone;
            }
            const double rn = sqrt(rr[k]);
            if (rn > maxr[k]) maxr[k] = rn;
            if (rn < delta * maxr[k] || rr[k] <= tol2 * bb[k]) update = true;
        }
        if (update) {
            // fold the sloppy solutions of every active source into x, true residual in FP64
            MTRY(V.site(OP_AXPBY, fref(&xs), fref(x), fref(x), fnone(), sv(1.0), sv(1.0), 0, 0, 0));
            MTRY(V.site(OP_AXPBY, fref(&xs), fnone(), fref(&xs), fnone(), sv(0.0), sv(0.0), 0, 0, 0));
            MTRY(V.normal_op(&Ap, x, &te, &to, nact));
            MTRY(V.site(OP_AXPBY, fref(bhat), fref(&Ap), fref(&r), fnone(), sv(1.0), sv(-1.0), 1, FIN_STORE,
                        SL_TMP0));
            MTRY(V.read_col(SL_TMP0, r2));
            nrel++;
            bool changed = false;
            for (int k = 0; k < nrhs; k++) {
                if (!act[k]) continue;
                if (r2[k] <= tol2 * bb[k]) {
                    act[k] = false;
                    conv_it[k] = it;
                    changed = true;
                }
                maxr[k] = sqrt(r2[k]);
            }
            if (changed) MTRY(V.set_active(act, &nact));
            if (nact == 0) break;
            MTRY(V.site(OP_COPY, fref(&r), fnone(), fref(&rs), fnone(), sv(1), sv(0), 0, 0, 0));
            MTRY(V.site(OP_NORM, fref(&rs), fnone(), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, SL_RRNEW));
        }
        k_scalar_beta<<<1, TM_MAX_RHS, 0, s>>>(V.S, nrhs, V.d_mask);
        MTRY(cuda_check(cudaGetLastError(), "beta"));
        MTRY(V.site(OP_AXPBY, fref(&rs), fref(&pp), fref(&pp), fnone(), sv(1.0), sslot(SL_BETA, 1.0), 0, 0, 0));
    }
    if (nact > 0) {
        set_error("tm_solve_multi: %d source(s) not converged after %d iterations", nact, it);
        st = TM_ERR_NOCONV;
    }
mdone:
    if (x != x_user && (st == TM_OK || st == TM_ERR_NOCONV)) {
        const tm_status cst = V.site(OP_COPY, fref(x), fnone(), fref(x_user), fnone(), sv(1), sv(0), 0, 0, 0, false);
        if (st == TM_OK) st = cst;
    }
    if (stats) {
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int k = 0; k < nrhs; k++) {
            stats[k].iterations = conv_it[k] >= 0 ? conv_it[k] : it;
            stats[k].reliable_updates = nrel;
            stats[k].true_residual = bb[k] > 0 ? sqrt(r2[k] / bb[k]) : 0.0;
            stats[k].pc_residual = -1.0;
            stats[k].seconds = secs;
        }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (s) {
        cudaEvent_t done = nullptr;
        if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(done, s);
            cudaStreamWaitEvent(user_stream, done, 0);
            cudaEventDestroy(done);
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (ev) cudaEventDestroy(ev);
    return st;
}

}  // namespace tmk

extern "C" {

tm_status tm_g5dot(const tm_gauge *g, const tm_field *a, const tm_field *b, double *re_out, double *im_out,
                   void *stream)
{
    TM_NVTX("tm_g5dot");
    if (!g || !a || !b || !a->data || !b->data || !re_out || !im_out) { set_error("tm_g5dot: null argument"); return TM_ERR_ARG; }
    if (a->nrhs != b->nrhs || a->nrhs < 1 || a->nrhs > TM_MAX_RHS) {
        set_error("tm_g5dot: fields must share nrhs in [1, %d]", TM_MAX_RHS);
        return TM_ERR_ARG;
    }
    if ((a->prec == TM_PREC_F16 && !a->norm) || (b->prec == TM_PREC_F16 && !b->norm)) {
        set_error("tm_g5dot: FP16 field needs its norm array");
        return TM_ERR_ARG;
    }
    MultiSolver V;
    V.g = g;
    V.sp = nullptr;
    V.s = (cudaStream_t)stream;
    V.nrhs = a->nrhs;
    V.S = g->scratch;
    V.H = g->host_scalars;
    V.d_mask = nullptr;
    tm_status st = V.site(OP_G5DOT_RE, fref(a), fref(b), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, SL_TMP0, false);
    if (st == TM_OK) st = V.read_col(SL_TMP0, re_out);
    if (st == TM_OK) st = V.site(OP_G5DOT_IM, fref(a), fref(b), fnone(), fnone(), sv(0), sv(0), 1, FIN_STORE, SL_TMP0, false);
    if (st == TM_OK) st = V.read_col(SL_TMP0, im_out);
    return st;
}

tm_status tm_solve_multi_workspace_bytes(const tm_gauge *g, const tm_solver_params *sp, int nrhs, size_t *bytes)
{
    tm_status st = check_solver_params(g, sp);
    if (st != TM_OK) return st;
    if (!bytes || nrhs < 1 || nrhs > TM_MAX_RHS) {
        set_error("tm_solve_multi_workspace_bytes: need 1 <= nrhs <= %d", TM_MAX_RHS);
        return TM_ERR_ARG;
    }
    *bytes = multi_workspace_need(g, sp, nrhs);
    return TM_OK;
}

tm_status tm_solve_multi(const tm_gauge *g, const tm_field *x_e, const tm_field *b_e, const tm_solver_params *sp,
                         tm_solver_stats *stats, void *workspace, size_t workspace_bytes, void *stream)
{
    TM_NVTX("tm_solve_multi");
    tm_status st = check_solver_params(g, sp);
    if (st != TM_OK) return st;
    if (!x_e || !b_e || !workspace || !x_e->data || !b_e->data) {
        set_error("tm_solve_multi: null field or workspace");
        return TM_ERR_ARG;
    }
    if (x_e->prec != TM_PREC_F64 || b_e->prec != TM_PREC_F64 || x_e->nrhs != b_e->nrhs || x_e->nrhs < 1 ||
        x_e->nrhs > TM_MAX_RHS) {
        set_error("tm_solve_multi: x and b must be FP64 fields with the same nrhs in [1, %d]", TM_MAX_RHS);
        return TM_ERR_ARG;
    }
    if (x_e->data == b_e->data) { set_error("tm_solve_multi: x must not alias b"); return TM_ERR_ARG; }
    if (g->dd) { set_error("tm_solve_multi: the handle holds one time slab of a decomposed lattice"); return TM_ERR_ARG; }
    if (((uintptr_t)workspace & 255) != 0) { set_error("tm_solve_multi: workspace must be 256-byte aligned"); return TM_ERR_ARG; }
    const size_t need = multi_workspace_need(g, sp, x_e->nrhs);
    if (workspace_bytes < need) {
        set_error("tm_solve_multi: workspace of %zu bytes is smaller than the %zu needed", workspace_bytes, need);
        return TM_ERR_NOMEM;
    }
    if (stats) memset(stats, 0, sizeof(*stats) * x_e->nrhs);
    return solve_multi(g, x_e, b_e, sp, stats, workspace, (cudaStream_t)stream);
}

}  // extern "C"

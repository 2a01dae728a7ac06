/*
 * tm.h -- C ABI of libtm: the even-odd preconditioned Wilson twisted-mass operator
 * (degenerate and non-degenerate doublet) on one NVIDIA GB300 GPU (sm_103a).
 *
 * Operator (eq. 2.1, kappa normalisation, DeGrand-Rossi gamma matrices, mu = x,y,z,t):
 *   M psi(x) = R psi(x) - kappa (H psi)(x)
 *   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)
 *   R = 1 + 2 i kappa mu gamma5 tau3 + 2 kappa epsilon tau1       (doublet, tau on flavour)
 *   R = 1 + 2 i kappa mu (+-1) gamma5                            (one flavour, tau3 = +-1)
 * Periodic in x, y, z; hops across the time boundary carry -1 when t_antiperiodic != 0.
 * H^dag is H with the two projectors exchanged; R^dag = R(-mu, epsilon).
 * The even-odd blocks are H_eo (odd -> even) and H_oe (even -> odd); the paper's D_eo is read
 * as H_eo, which makes the left-hand sides of eq. 2.2 and 2.3 the exact Schur complements.
 *
 * Conventions shared by every call:
 *  - Operator calls (tm_dslash*, tm_precond_op, tm_mat, tm_prepare_rhs, tm_reconstruct_odd,
 *    tm_twist) accept fields with nrhs >= 1 (all operands sharing nrhs): every right-hand side
 *    is processed in one launch that reads each link once per site for all of them.
 *  - Field data (tm_field) are DEVICE pointers (cudaMalloc'd or from an allocator such as
 *    torch).  Canonical buffers (tm_gauge_create, tm_pack, tm_unpack) may also be pinned host
 *    memory, which the kernels read or write in place over the CPU-GPU link; pageable host
 *    memory is rejected with TM_ERR_ARG.  The caller owns every buffer; the library never
 *    frees one.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call except
 *    tm_gauge_create / tm_gauge_destroy / tm_solve / tm_solve_multi only enqueues work on
 *    `stream` and returns; errors found on the host are reported before anything is enqueued.
 *  - Every call returns a tm_status; nothing throws across the ABI.  tm_last_error() gives a
 *    one-line message for the last failing call on the calling host thread.
 *  - Calls that share one tm_gauge use its small reduction scratch area and must therefore be
 *    ordered on one stream (calls on different streams that overlap on the GPU race).
 *
 * Field storage (tm_field): one parity of a spinor field in structure-of-arrays form,
 *   data: [nrhs][nf][chunk][Vh] with the 24 reals of a site, ordered (spin*3 + colour)*2 + re/im,
 *         cut into 16-byte chunks (FP64: 12, FP32: 6, FP16: 3 chunks per site and flavour);
 *   norm: FP16 only, float [nrhs][nf][Vh], the site's max |real| (stored half = value / norm);
 *   DF64: 12 chunks per site and flavour, each (hi, lo, hi, lo) of two consecutive reals.
 * Vh = Lx Ly Lz Lt / 2; even sites have (x+y+z+t) even; site index within a parity is
 * (x + Lx (y + Ly (z + Lz t))) / 2.  tm_field_bytes() gives the sizes to allocate.
 *
 * Canonical (user) layout, complex128 or complex64, x fastest:
 *   spinor [Lt][Lz][Ly][Lx][nf][4][3],  gauge [4][Lt][Lz][Ly][Lx][3][3] (row-major 3x3).
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TM_OK = 0,
    TM_ERR_ARG = -1,     /* invalid argument (null pointer, odd extent, singular twist, ...) */
    TM_ERR_CUDA = -2,    /* a CUDA call or kernel launch failed */
    TM_ERR_NOCONV = -3,  /* solver hit maxiter before reaching the tolerance */
    TM_ERR_NAN = -4,     /* solver saw a non-finite residual */
    TM_ERR_TIMEOUT = -5, /* a bounded device-side wait gave up */
    TM_ERR_NOMEM = -6    /* device allocation failed, or a workspace is too small */
} tm_status;

/* twist_flavor (sec. 2.2): one flavour with tau3 = +1 / -1, or the two-flavour doublet. */
typedef enum { TM_TWIST_PLUS = 1, TM_TWIST_MINUS = -1, TM_NDEG_DOUBLET = 2 } tm_flavor;
/* storage precision.  F64/F32/F16: value = bytes per real; FP16 carries a per-site float norm and
 * computes in FP32.  DF64: each real is a pair of floats hi + lo (8 bytes, 48-bit significand,
 * relative rounding ~3.6e-15) computed with error-free float transformations -- double-precision
 * class accuracy at FP32-pipe throughput, which GB300 issues far faster than FP64.  DF64 links
 * use 18 or 12 reals (recon 8 handles keep 12 for their DF64 copy). */
typedef enum { TM_PREC_F64 = 8, TM_PREC_F32 = 4, TM_PREC_F16 = 2, TM_PREC_DF64 = 16 } tm_prec;
/* gauge link storage (sec. 3): 18 reals, 2 rows (12 reals), or 8 reals. */
typedef enum { TM_RECON_18 = 18, TM_RECON_12 = 12, TM_RECON_8 = 8 } tm_recon;
/* even-odd preconditioning: asymmetric (eq. 2.2) or symmetric (eq. 2.3). */
typedef enum { TM_PC_ASYM = 0, TM_PC_SYM = 1 } tm_pc;
/* canonical element type */
typedef enum { TM_C128 = 0, TM_C64 = 1 } tm_canon;

/*
 * Fused local operation applied at the output site of tm_dslash (sec. 2.1, "all local
 * operators are merged into dslash kernels"); D = H or H^dag, t = the input, x = the extra
 * field argument, R / R^-1 daggered in tm_dslash_dagger:
 */
typedef enum {
    TM_EPI_NONE = 0,        /* out = D t                                                    */
    TM_EPI_TWINV = 1,       /* out = R^-1 D t             the fused R^-1_oo D_oe of sec. 2.1 */
    TM_EPI_TWXPAY_ASYM = 2, /* out = R x - kappa^2 D t    the fused R_ee - kappa^2 D_eo      */
    TM_EPI_TWXPAY_SYM = 3,  /* out = x - kappa^2 R^-1 D t (eq. 2.3)                         */
    TM_EPI_XPAY = 4,        /* out = x + kappa D t                                          */
    TM_EPI_TWINV_XPAY = 5,  /* out = R^-1 (x + kappa D t)  odd-site reconstruction          */
    TM_EPI_XMAY_K2 = 6      /* out = x - kappa^2 D t      second launch of the adjoint of eq. 2.3 */
} tm_epilogue;

typedef struct {
    int L[4];             /* Lx, Ly, Lz, Lt: each even and >= 2; Vh = Lx Ly Lz Lt / 2 < 2^31 / 24 */
    double kappa;         /* hopping parameter */
    double mu;            /* twisted mass mu (mu-bar for the doublet) */
    double epsilon;       /* epsilon-bar of the doublet; must be 0 for TM_TWIST_PLUS/MINUS */
    int flavor;           /* tm_flavor */
    int t_antiperiodic;   /* 1: antiperiodic in time, 0: periodic */
    int recon;            /* tm_recon, used for every precision of the gauge handle (but see
                             TM_GAUGE_F64_FULL_LINKS and the DF64 note above) */
} tm_params;

typedef struct {
    void *data;  /* device pointer, layout above */
    float *norm; /* device pointer, FP16 only (NULL otherwise) */
    int prec;    /* tm_prec */
    int nrhs;    /* right-hand sides stored back to back (1 for single fields) */
} tm_field;

typedef struct tm_gauge tm_gauge; /* opaque: packed links in FP64, FP32, FP16, DF64 + scratch */

/* Library version string. */
const char *tm_version(void);

/* Copy the message of the last failing call on this host thread into buf (NUL-terminated). */
tm_status tm_last_error(char *buf, size_t n);

/*
 * Create a gauge handle on the current CUDA device.  U_canon: device pointer to the canonical
 * complex128 gauge field (see above); it is read once and may be freed after the call
 * returns.  The handle allocates and owns device memory for the packed links in all three
 * precisions plus a reduction scratch area; it synchronises `stream` before returning.
 * Errors: TM_ERR_ARG (params, null pointers, 1 + (2 kappa mu)^2 - (2 kappa eps)^2 <= 0 with
 * a doublet), TM_ERR_NOMEM, TM_ERR_CUDA.
 */
tm_status tm_gauge_create(const tm_params *p, const void *U_canon, void *stream, tm_gauge **out);

/* tm_gauge_create packing only the link storage forms in prec_mask: bit 0 FP64, 1 FP32, 2 FP16,
 * 3 DF64 (bits 0-3 all clear = all four, as tm_gauge_create).  An operator, solver or force call on
 * fields of a storage form the handle did not pack returns TM_ERR_ARG; a clover term needs the
 * FP64 links.  32^3x64, recon 12: FP64 805 MB, FP32 403 MB, FP16 201 MB, DF64 805 MB.
 * Bit 4 (TM_GAUGE_F64_FULL_LINKS): the FP64 links keep all 18 reals whatever p->recon (1208 MB at
 * 32^3x64); the other storage forms follow p->recon.  The FP64 hopping kernels are bound by the
 * FP64 pipe, not by HBM, so rebuilding the third row costs them more than reading it: the FP64
 * doublet M_asym at 32^3x64 takes 7.3 ms with 18-real links against 8.2 ms with 12 (sec. 3's
 * trade of flops for bytes runs the other way at this precision).  Results differ from the
 * compressed form by rounding only. */
#define TM_GAUGE_F64_FULL_LINKS 16
tm_status tm_gauge_create_ex(const tm_params *p, const void *U_canon, int prec_mask, void *stream, tm_gauge **out);

/* Release a handle (NULL is accepted).  Waits for the device to finish using it. */
tm_status tm_gauge_destroy(tm_gauge *g);

/* Bytes to allocate for one parity field of `prec` with the handle's flavour count and nrhs. */
tm_status tm_field_bytes(const tm_gauge *g, int prec, int nrhs, size_t *data_bytes, size_t *norm_bytes);

/*
 * Copy a field between device memory and host memory in the library's own layout (the bytes of
 * data, and of norm for FP16, unchanged; tm_field_bytes() sizes), for clients that keep fields on
 * the host in this form between host-driven steps or for checkpoints, so that no conversion
 * pass runs.  The paper has no counterpart; this is a library-usage addition.  host_data /
 * host_norm are host pointers (page-locked memory for the copies to be asynchronous); host_norm
 * is ignored, and may be NULL, unless the field is FP16.  One cudaMemcpyAsync per array on
 * `stream`.  Errors: TM_ERR_ARG (null pointers, bad field), TM_ERR_CUDA.
 */
tm_status tm_field_upload(const tm_gauge *g, const tm_field *dev, const void *host_data, const void *host_norm,
                          void *stream);
tm_status tm_field_download(const tm_gauge *g, void *host_data, void *host_norm, const tm_field *dev, void *stream);

/*
 * Convert between the canonical full-lattice layout and one parity of a tm_field (the
 * "converting routines" between a client's layout and the internal one, sec. 2).  pack reads
 * the sites of `parity` from canon (canon_type = tm_canon); unpack writes only those sites of
 * canon and leaves the others untouched.  For nrhs > 1 canon holds nrhs fields back to back.
 */
tm_status tm_pack(const tm_gauge *g, const tm_field *out, const void *canon, int canon_type, int parity,
                  void *stream);
tm_status tm_unpack(const tm_gauge *g, void *canon, int canon_type, const tm_field *in, int parity,
                    void *stream);

/*
 * Z2 noise sources (+-1 +- i)/sqrt 2 for the stochastic estimator of disconnected loops (the
 * paper's production use, sec. 1 and 4), written straight into one parity of a field: element i
 * (flat canonical index) of right-hand side r takes bits 0 / 1 (real / imaginary sign) of
 * SplitMix64's output function at the counter state (seed + r + 1) G + (i + 1) G,
 * G = 0x9E3779B97F4A7C15 (Steele, Lea & Flood 2014).
 */
tm_status tm_noise_z2(const tm_gauge *g, const tm_field *out, int parity, unsigned long long seed, void *stream);

/*
 * One fused hopping kernel (sec. 2.1):  out(out_parity) = epilogue(H_{p,1-p} in), with
 * H^dag and daggered twists in tm_dslash_dagger.  `x` has the output parity and is used by
 * the XPAY epilogues (NULL otherwise).  out, in and x must share a precision; out must not
 * alias in.  Errors: TM_ERR_ARG, TM_ERR_CUDA.
 */
tm_status tm_dslash(const tm_gauge *g, const tm_field *out, const tm_field *in, int out_parity, int epilogue,
                    const tm_field *x, void *stream);
tm_status tm_dslash_dagger(const tm_gauge *g, const tm_field *out, const tm_field *in, int out_parity,
                           int epilogue, const tm_field *x, void *stream);

/*
 * Even-even preconditioned operator, two fused launches through the odd temporary tmp_o:
 *   TM_PC_ASYM:  out = (R_ee - kappa^2 H_eo R_oo^-1 H_oe) in               (eq. 2.2 LHS)
 *   TM_PC_SYM:   out = (1 - kappa^2 R_ee^-1 H_eo R_oo^-1 H_oe) in          (eq. 2.3 LHS)
 * dagger = 1 applies the adjoint (for SYM: 1 - kappa^2 H^dag_eo R_oo^-dag H^dag_oe R_ee^-dag,
 * whose first launch twists every neighbour before the projection; for DF64 and FP16 doublet
 * fields R_ee^-dag in is instead one elementwise launch into out_e).  Fields share one
 * precision; tmp_o is overwritten; out_e must not alias in_e or tmp_o.
 */
tm_status tm_precond_op(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o,
                        int pc, int dagger, void *stream);

/*
 * tm_precond_op restricted to the right-hand sides listed in active_dev (device array of
 * nactive indices into the fields' nrhs), for solvers that stop iterating converged sources;
 * the other right-hand sides of out_e and tmp_o are left untouched.  Listed indices outside
 * [0, nrhs) are skipped by the kernels.
 */
tm_status tm_precond_op_active(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o,
                               int pc, int dagger, const int *active_dev, int nactive, void *stream);

/*
 * Normal operator of the even-even system: out = A^dag A in with A = M_pc of tm_precond_op (pc),
 * or A = M_pc^dag when dagger = 1 -- the operator CG iterates with (sec. 2.2, NORMOP).  Four fused
 * launches.  For TM_PC_SYM without dagger (and no clover term) it is evaluated as
 *   M_sym^dag M_sym = M_asym^dag (R_ee R_ee^dag)^-1 M_asym
 * (M_sym = R_ee^-1 M_asym, eq. 2.2/2.3), so no launch needs the input-twist prologue that
 * M_sym^dag alone has: (R R^dag)^-1 = ((1 + a^2 + b^2) + 2 b tau1 - 2 a b gamma5 tau2)^-1 for the
 * doublet (a = 2 kappa mu, b = 2 kappa eps), 1 / (1 + a^2) for one flavour, is applied in the
 * epilogue of the first M_asym.  tmp_e and tmp_o are overwritten.  Fields share a precision and
 * nrhs (<= 64) and are distinct.  Errors: TM_ERR_ARG, TM_ERR_CUDA.
 */
tm_status tm_normal_op(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_e,
                       const tm_field *tmp_o, int pc, int dagger, void *stream);

/*
 * Full unpreconditioned operator (eq. 2.1) on both parities: out = M in (dagger = 0) or
 * M^dag in.  Two fused launches; out must not alias in.
 */
tm_status tm_mat(const tm_gauge *g, const tm_field *out_e, const tm_field *out_o, const tm_field *in_e,
                 const tm_field *in_o, int dagger, void *stream);

/*
 * Right-hand side of the even system from the full source b (eq. 2.2 / 2.3 RHS, derived by
 * block elimination of M psi = b; the printed RHS is read with the sign and kappa of that
 * elimination):
 *   ASYM:  b'_e = b_e + kappa H_eo R_oo^-1 b_o
 *   SYM:   b'_e = R_ee^-1 (b_e + kappa H_eo R_oo^-1 b_o)
 * dagger = 1 daggers every factor (source of M^dag psi = b).  For SYM with dagger = 1 the
 * system is preconditioned from the right, M_sym^dag y = b'_e with b'_e as for ASYM, and
 * psi_e = R_ee^-dag y.  One fused launch (input twist in the prologue).  FP64/FP32/FP16 fields
 * (DF64 is not offered here: the right-hand side is prepared once, in FP64).
 */
tm_status tm_prepare_rhs(const tm_gauge *g, const tm_field *bprime_e, const tm_field *b_e, const tm_field *b_o,
                         int pc, int dagger, void *stream);

/*
 * Odd half of the solution (eq. 2.4, read as the block elimination of M psi = b):
 *   psi_o = R_oo^-1 (b_o + kappa H_oe psi_e)        (daggered factors when dagger = 1)
 * One fused launch.
 */
tm_status tm_reconstruct_odd(const tm_gauge *g, const tm_field *psi_o, const tm_field *b_o, const tm_field *psi_e,
                             int dagger, void *stream);

/* Local twist on one parity: out = R in, R^-1 in (inverse = 1), daggered when dagger = 1.
 * A clover handle's local operator depends on the site: tm_twist returns TM_ERR_ARG there
 * (use tm_local_op). */
tm_status tm_twist(const tm_gauge *g, const tm_field *out, const tm_field *in, int inverse, int dagger,
                   void *stream);

/* ------------------------------------------------------------------------------- clover term */
/*
 * Clover-improved twisted mass (the combination the paper's Conclusion names as the next step).
 * After tm_gauge_set_clover(g, c_sw) every operator of the handle uses the local operator
 *   L(x) = 1 + T(x) + (R - 1),   T(x) = i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x)
 * in place of R (eq. 2.1-2.4 with R -> L):  M = L - kappa H,  M_asym = L_ee - kappa^2 H_eo
 * L_oo^-1 H_oe,  M_sym = 1 - kappa^2 L_ee^-1 H_eo L_oo^-1 H_oe, b'_e and psi_o likewise.
 * sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] (DeGrand-Rossi), F_{mu nu} = (Q - Q^dag)/8 with Q
 * the four plaquettes of the mu-nu plane that start and end at x (same sense, mu first).
 * The field is computed on the device from the handle's FP64 links and stored per parity as
 * C = 1 + T and (C^2 - X^2)^-1 per gamma5 block (X = R - 1) in FP64, FP32 and FP16 (about
 * 1.15 / 0.58 / 0.33 KB per site; 32^3x64: 2.4 / 1.2 / 0.7 GB).  c_sw = 0 removes the term.
 * Synchronises `stream`.  With a clover term: operator calls take nrhs = 1 FP64 / FP32 / FP16
 * fields (no DF64, no multi-RHS, no tm_solve_multi); tm_force returns TM_ERR_ARG (the link
 * derivative of T is not implemented); tm_prepare_rhs draws one odd temporary from CUDA's
 * stream-ordered pool (cudaMallocAsync / cudaFreeAsync on `stream`).
 * Errors: TM_ERR_ARG (non-finite c_sw; C^2 - X^2 numerically singular at some site: the
 * handle keeps its previous clover state), TM_ERR_NOMEM, TM_ERR_CUDA.
 */
tm_status tm_gauge_set_clover(tm_gauge *g, double csw, void *stream);

/* Local operator of one parity: out = L in (inverse = 0) or L^-1 in, daggered when dagger = 1,
 * on the sites of `parity` (0 even, 1 odd).  L is R without a clover term (then any nrhs and
 * precision) and 1 + T + (R - 1) with one (nrhs = 1, FP64 / FP32 / FP16). */
tm_status tm_local_op(const tm_gauge *g, const tm_field *out, const tm_field *in, int parity, int inverse, int dagger,
                      void *stream);

/* ------------------------------------------------------------------------------ solvers */
/* CG on the normal equations (sec. 2.2: solve_type NORMOP on the even-odd preconditioned
 * system), either all in FP64 or as the mixed-precision reliable-update CG the paper runs
 * in production (double-single / double-half, sec. 3 and ref. [Clark:2009wm]). */
typedef enum { TM_SOLVER_CG = 0, TM_SOLVER_MIXED_CG = 1 } tm_solver_type;
/* solution_type (sec. 2.2): MAT solves A x = b, MATDAG_MAT solves A^dag A x = b, where
 * A = M_pc of tm_precond_op (or its adjoint when dagger = 1). */
typedef enum { TM_SOLUTION_MAT = 0, TM_SOLUTION_MATDAG_MAT = 1 } tm_solution_type;

typedef struct {
    int solver;      /* tm_solver_type */
    int solution;    /* tm_solution_type */
    int pc;          /* tm_pc */
    int dagger;      /* 1: A = M_pc^dag */
    double tol;      /* stop when |bhat - A^dag A x| / |bhat| <= tol (FP64 true residual);
                        bhat = A^dag b (MAT) or b (MATDAG_MAT).  The mixed solver of a MAT
                        solution computes the residual as A^dag (b - A x) and, with FP32 sloppy
                        fields, |bhat| from A^dag b in binary32 (about 1e-7 relative): bhat then
                        never exists in FP64, saving two FP64 operator applications */
    int maxiter;     /* CG iterations (sloppy iterations for the mixed solver) */
    double delta;    /* mixed: reliable update when |r_sloppy| < delta * max |r| since the last one */
    int sloppy_prec; /* mixed: TM_PREC_F32 or TM_PREC_F16 storage for the inner iteration */
    int use_x0;      /* 1: x_e holds the initial guess on entry; 0: start from zero */
    int want_pc_residual; /* 1: also compute stats->pc_residual (one more FP64 operator application) */
    int use_graph;   /* tm_solve_multi: capture the sloppy iteration as a CUDA graph and replay it */
    int true_prec;   /* TM_PREC_F64 (default, 0 means F64) or TM_PREC_DF64: precision of the solution
                        accumulation, the true residual and (plain CG) the whole iteration; x and b
                        stay FP64 fields either way */
} tm_solver_params;

typedef struct {
    int iterations;
    int reliable_updates; /* mixed: reliable updates; FP64 CG: restarts from the true residual */
    double true_residual; /* |bhat - A^dag A x| / |bhat|, recomputed in FP64 at exit (|bhat| as
                             the stopping test takes it, see tol) */
    double pc_residual;   /* |A x - b| / |b| for MAT solutions when want_pc_residual, else -1 */
    double seconds;       /* host wall time of the call */
} tm_solver_stats;

/* Device workspace tm_solve needs for these parameters (caller allocates, 256-byte aligned). */
tm_status tm_solve_workspace_bytes(const tm_gauge *g, const tm_solver_params *sp, size_t *bytes);

/*
 * Solve on the even sites.  x_e (in/out) and b_e are FP64 single-RHS fields.  Blocks until
 * the solve ends (one scalar read per iteration).  Errors: TM_ERR_ARG, TM_ERR_NOMEM
 * (workspace too small), TM_ERR_NOCONV (maxiter reached; x_e holds the last iterate and the
 * stats are filled), TM_ERR_NAN (non-finite residual), TM_ERR_CUDA.
 */
tm_status tm_solve(const tm_gauge *g, const tm_field *x_e, const tm_field *b_e, const tm_solver_params *sp,
                   tm_solver_stats *stats, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Multi-RHS solve (batched stochastic sources): x_e and b_e hold nrhs <= 64 right-hand sides
 * (FP64).  All sources iterate together: every operator factor is one multi-RHS launch that
 * reads each link once per site for all active sources, and every BLAS step is one launch with
 * per-source alpha, beta and |r|^2.  The mixed solver takes its FP64 reliable updates for all
 * active sources at once when any of them asks for one; a source whose FP64 true residual meets
 * tol is dropped (later launches skip it) and its iteration count recorded.  use_graph captures
 * the sloppy iteration (two operator applications, the alpha reduction and the fused update)
 * as a CUDA graph, re-captured when the number of active sources changes.  The solve runs on an
 * internal stream ordered after `stream` and blocks until it ends.  stats: array of nrhs
 * entries.  Errors as tm_solve (TM_ERR_NOCONV when any source misses tol within maxiter).
 */
tm_status tm_solve_multi_workspace_bytes(const tm_gauge *g, const tm_solver_params *sp, int nrhs, size_t *bytes);
tm_status tm_solve_multi(const tm_gauge *g, const tm_field *x_e, const tm_field *b_e, const tm_solver_params *sp,
                         tm_solver_stats *stats, void *workspace, size_t workspace_bytes, void *stream);

/*
 * <a_r, gamma5 b_r> for every right-hand side r (complex, FP64 accumulation, blocking): the
 * per-source term of the stochastic estimator Tr[gamma5 M^-1] ~ (1/N) sum_n eta_n^dag gamma5 s_n
 * (s_n = M^-1 eta_n), evaluated per parity and summed by the caller.  re_out, im_out: host
 * arrays of nrhs doubles.  Operand precisions as for the solver's combinations (FP64 pairs).
 */
tm_status tm_g5dot(const tm_gauge *g, const tm_field *a, const tm_field *b, double *re_out, double *im_out,
                   void *stream);

/* FP64-accumulated reductions over one parity field (blocking): |x|^2 and Re<a, b>. */
tm_status tm_norm2(const tm_gauge *g, const tm_field *x, double *out, void *stream);
tm_status tm_dot(const tm_gauge *g, const tm_field *a, const tm_field *b, double *re_out, void *stream);

/*
 * out = a x + b y on one parity field (y = NULL: out = a x), every right-hand side, the solvers'
 * site-wise linear combination (sec. 2.2, the BLAS of CG) offered for callers that combine
 * solutions, e.g. the gradient 2 X of the pseudofermion action.  out, x, y share nrhs; out may
 * alias x or y.  Precisions: all equal, or the mixed combinations the solvers use (an FP64 or
 * DF64 out / y with an FP32 or FP16 x and the reverse conversions, e.g. out FP32 = x FP64, or
 * out FP64 = x FP32 + y FP64); others return TM_ERR_ARG.  Arithmetic in FP64 when a field is
 * FP64, double-float for DF64, FP32 otherwise.  Asynchronous on `stream`.
 * Errors: TM_ERR_ARG, TM_ERR_CUDA.
 */
tm_status tm_axpby(const tm_gauge *g, const tm_field *out, double a, const tm_field *x, double b, const tm_field *y,
                   void *stream);

/* ------------------------------------------------------------------------ differentiation */
/*
 * Link gradient of L(U) = Re <g, M(U) psi> for every link, in the convention
 * dL = Re sum_ij conj(F_ij) dU_ij (the gradient torch's autograd propagates for complex U):
 *   F_mu(x) = coef * (-kappa) * bc * sum_flavour [ sum_s ((1 - gamma_mu) g(x))_s psi(x+mu)_s^dag
 *                                                 + sum_s psi(x)_s ((1 + gamma_mu) g(x+mu))_s^dag ]
 * with bc = -1 on links across the antiperiodic time boundary (eq. 2.1 differentiated; R does
 * not depend on U).  project = 1 returns the su(3) tangent-space part TA(F U^dag) U, TA(Z) =
 * (Z - Z^dag)/2 - tr(Z - Z^dag)/6, which is what a gradient along SU(3) needs.  The pseudofermion
 * force of S = phi^dag (M^dag M)^-1 phi is the case psi = X = (M^dag M)^-1 phi, g = Y = M X,
 * coef = -2.  psi and g: FP64 or FP32 fields of both parities.  F_canon: device pointer to the
 * canonical gauge layout, complex128 (canon_type TM_C128) or complex64.
 */
tm_status tm_force(const tm_gauge *g, void *F_canon, int canon_type, const tm_field *psi_e, const tm_field *psi_o,
                   const tm_field *g_e, const tm_field *g_o, double coef, int project, void *stream);

/* ---------------------------------------------------------------------------- autotuning */
/*
 * Time every launch choice of the hopping kernel (thread per site with 64-256 threads per block,
 * the same with a two-stage load pipeline in registers or in shared memory, or with a
 * 128-register cap in three block shapes) for
 * each precision, with and without the input-twist prologue, and the multi-RHS form (the tune
 * entries below, timed on 16 right-hand sides, 8 in FP64), on this handle's lattice, and
 * keep the fastest; with a clover term also the clover kernel's form (1, 3 or 4 blocks per SM,
 * or the staged pipeline).  Allocates three single-RHS and three 16-RHS (FP64: 8-RHS) scratch fields for the duration of the call
 * (the multi-RHS shape keeps its default when the latter do not fit) and synchronises `stream`;
 * do not call it while capturing a graph.  Until it runs (or a table is imported) the handle
 * uses defaults (FP64 capped 128 x 4; FP32 and FP16 the shared-memory pipeline with the paired
 * hop: two buffers for the FP32 doublet (8), three otherwise (9), except one flavour with
 * 18-real links, capped; multi-RHS: for FP32 / FP16 the staged form with 4 right-hand sides
 * per block in group-major order (doublet, 34) or paired sources (one flavour: FP32 36, FP16
 * 16), the register form with 4 for FP64; clover 1 block per SM for FP64, 3 for FP16 and the FP32 doublet,
 * 4 for FP32 one flavour).
 */
tm_status tm_autotune(tm_gauge *g, void *stream);
/* The tuned table as text, and back.  Single-RHS entries "f32:0:3:128" = precision:prologue:
 * variant:block (variant 0 plain, 2 pipelined in registers, 3 / 4 / 5 capped at 128 registers with
 * 128 / 64 / 256-thread blocks, 6 / 7 pipelined through shared memory with cp.async, two / three
 * buffers, 8 / 9 the same as 6 / 7 with the hop in packed FMAs over register pairs: the two
 * flavours of an FP32 or FP16 doublet, the two projected spin rows of one flavour (as 6 / 7 in
 * FP64), with results bit-identical to 6 / 7; 2 has no prologue form); multi-RHS entries "f32:m:4" = precision:m:right-hand sides per block (2, 4
 * or 8) of the register form, or 12 / 14 for the staged form (the pipeline of 8 / 9 with links
 * copied through L1) with 2 / 4 right-hand sides per block, or 16 (one flavour): with every
 * right-hand side of an even count, two sources at a time through the doublet's staged kernels
 * (a one-flavour field with 2k sources has a doublet field's layout with k), else as 14; 32 / 34
 * / 36 = 12 / 14 / 16 with the blocks ordered group by group (one sweep over the sites per group
 * of sources) instead of interleaving the groups of a site block; for FP16 also 13 / 15 (33 / 35):
 * 12 / 14 (32 / 34) with three staging buffers, used for the doublet without the input prologue
 * (otherwise they run as 12 / 14); clover entries "f32:c:3" = precision:c:resident 128-thread blocks per SM the clover
 * kernel's register allocation allows (1, 3 or 4), or 6 for its shared-memory staged pipeline;
 * fused-operator entries "f32:p:1" = precision:p:1 when tm_precond_op runs as one fused launch
 * (FP64 and FP32; see tm_device_status).  Import accepts any subset of the entries; an
 * invalid entry leaves the table unchanged and returns TM_ERR_ARG. */
tm_status tm_tune_export(const tm_gauge *g, char *buf, size_t n);
tm_status tm_tune_import(tm_gauge *g, const char *text);

/*
 * Status of the handle's bounded device-side waits.  The fused form of tm_precond_op (tune entry
 * "<prec>:p:1": both passes of M_pc in one persistent launch whose second-pass tiles wait for the
 * first-pass tiles they read) bounds every wait in time: a wait that has not seen its flag after
 * the handle's limit (1 s by default, measured on the device's nanosecond clock) records the
 * failure in a device word instead of hanging, and every later wait of the same launch on an
 * unset flag gives up at once; the affected sites are left unwritten.  This call synchronises
 * `stream`, returns TM_ERR_TIMEOUT (and clears the word) if any wait gave up since the last call,
 * TM_OK otherwise.  tm_solve makes the same check before it returns.
 */
tm_status tm_device_status(const tm_gauge *g, void *stream);

/*
 * Replace the fused operator's work list of a handle (for tests of the bounded waits and for
 * experiments with the claim order): items as returned by tm_fused_work_list, 1 <= nitems <= the
 * length of the handle's own list, every entry naming a group of the lattice ((entry >> 1) below
 * the number of 512-site groups).  Nothing else is checked: a list that leaves out first-pass
 * work makes the second-pass waits on it give up after wait_limit_ns (1 ms ... 60 s) with
 * TM_ERR_TIMEOUT reported by tm_device_status, never a hang.  items = NULL restores the handle's
 * own list.  Synchronises `stream`.  Errors: TM_ERR_ARG, TM_ERR_CUDA.
 */
tm_status tm_fused_set_work_list(tm_gauge *g, const int *items, int nitems, unsigned long long wait_limit_ns,
                                 void *stream);

/*
 * The fused operator's work list for a lattice (host only, no GPU; for inspection and tests):
 * entries (group << 1) | pass, pass 0 = first pass (odd output), 1 = second pass (even output),
 * a group being 4 tiles of 128 consecutive checkerboard sites.  Every second-pass group appears
 * after the first-pass groups holding its sites' neighbours.  With items = NULL returns the
 * length; otherwise fills items (capacity entries) and returns the length, or -1 on odd or too
 * small extents or too small a capacity.
 */
int tm_fused_work_list(const int L[4], int num_sms, int *items, int capacity);

/* ------------------------------------------------------- domain decomposition in time (sec. 2.1) */
/*
 * The multi-GPU parallelisation of sec. 2.1 (Figs. 1-2): the lattice is cut into time slabs, one
 * per rank, and every hopping launch exchanges one face per neighbour: the spin-projected
 * half-spinors of the boundary slice (2 spin rows x 3 colours = 12 reals per site and flavour,
 * both flavours of the doublet in one message).  A rank holds its slab in an ordinary handle
 * (tm_gauge_create with L[3] = its slab's time extent, t_antiperiodic of the whole lattice, the
 * links of its own sites) and marks it with tm_gauge_set_partition.  A hopping launch then runs as
 *   1. tm_dd_pack_faces   the faces of the input field for the previous and the next slab;
 *   2. (the caller's transport) send them; receive the neighbours' faces;
 *   3. tm_dd_dslash       the interior slices (region TM_DD_INTERIOR, needs no face, may start
 *                         before the faces arrive) and the first and last slice (TM_DD_BOUNDARY).
 * The composed operators (eq. 2.2-2.4) are two such launches; reductions of a solver are sums of
 * the ranks' tm_dot / tm_norm2 (one FP64 allreduce each).  Faces are kept in the arithmetic
 * precision (FP64 fields: doubles, FP32 / FP16 fields: floats, FP16 with the input's site norm),
 * so a decomposed operator gives the same bits as the undecomposed one.  A slab handle refuses
 * the other hopping calls (tm_dslash, tm_precond_op, tm_mat, tm_prepare_rhs, tm_reconstruct_odd,
 * tm_solve, tm_solve_multi, tm_force) with TM_ERR_ARG; site-local calls work as before.
 * Decomposed operators take single-RHS FP64 / FP32 / FP16 fields and no clover term.
 */
typedef enum { TM_DD_ALL = 0, TM_DD_INTERIOR = 1, TM_DD_BOUNDARY = 2 } tm_dd_region;

/* Mark the handle as the slab of time slices [t_offset, t_offset + L[3]) of a lattice with
 * Lt_global slices (t_offset even, t_offset + L[3] <= Lt_global, Lt_global even); the faces that
 * cross the time boundary of the whole lattice take the antiperiodic sign.  Lt_global = 0 removes
 * the mark.  One slab covering the whole lattice (t_offset 0, Lt_global = L[3]) whose faces go
 * back to itself gives the undecomposed operator.  Host only.  Errors: TM_ERR_ARG. */
tm_status tm_gauge_set_partition(tm_gauge *g, int t_offset, int Lt_global);

/* Bytes of one face buffer for fields of `prec` (both flavours of a doublet). */
tm_status tm_dd_face_bytes(const tm_gauge *g, int prec, size_t *bytes);

/*
 * Pack the two faces of the input `in` of a hopping launch with output parity out_parity (in has
 * parity 1 - out_parity): face_prev (for the previous slab) = (1 - s gamma_4) in at the first
 * slice; face_next (for the next slab) = U_4^dag (1 + s gamma_4) in at the last slice; s = +1 for
 * H, -1 for H^dag (dagger = 1).  twist_in = 1 applies R^-1 (R^-dag when dagger) to in first, as
 * the input prologue of tm_dd_dslash does.  Device buffers of tm_dd_face_bytes, 16-byte aligned.
 * Asynchronous on `stream`.  Errors: TM_ERR_ARG, TM_ERR_CUDA.
 */
tm_status tm_dd_pack_faces(const tm_gauge *g, void *face_prev, void *face_next, const tm_field *in, int out_parity,
                           int dagger, int twist_in, void *stream);

/*
 * tm_dslash (dagger = 0) or tm_dslash_dagger (dagger = 1) on a slab: out(out_parity) =
 * epilogue(H in) with the epilogues of tm_dslash (x as there), twist_in = 1 applying R^-1 (R^-dag)
 * to every neighbour first.  ghost_prev / ghost_next: the faces received from the previous /
 * next slab (their face_next / face_prev), needed by TM_DD_ALL and TM_DD_BOUNDARY; TM_DD_INTERIOR
 * reads none (NULL allowed).  The interior slices run in the handle's tuned launch form, the
 * boundary slices in a register-capped form.  Asynchronous on `stream`.
 * Errors: TM_ERR_ARG, TM_ERR_CUDA.
 */
tm_status tm_dd_dslash(const tm_gauge *g, const tm_field *out, const tm_field *in, int out_parity, int epilogue,
                       const tm_field *x, int dagger, int twist_in, const void *ghost_prev, const void *ghost_next,
                       int region, void *stream);

/* --------------------------------------------------------------------- allocation-free variant */
/*
 * |x|^2 of each right-hand side of a parity field (the tm_norm2 reduction), for callers that
 * cannot allocate device memory: it needs no tm_gauge handle (creating one allocates) and calls
 * no allocating routine.  The paper has no counterpart; this is a library-usage addition.
 *   x:          field to reduce (any precision); Vh sites per parity, nf flavours (1 or 2),
 *               x->nrhs right-hand sides, at most 64.
 *   result_dev: device pointer to x->nrhs doubles, written with |x_rhs|^2 (FP64 accumulation).
 * The reduction's scratch (256 x 64 partial sums and a completion ticket, about 128 KB) is one
 * static device array per loaded copy of the library, kept on every GPU that uses it until the
 * process exits.  The first call on a device (with that device current) looks up the array's
 * device address and caches it; make that first call before any stream capture.  The cached
 * address belongs to the device's primary context: do not reset the device (cudaDeviceReset)
 * between calls while the library stays loaded.  Every call
 * shares the array: calls that overlap on the GPU (different streams, or different host threads
 * without ordering) race and give wrong results; calls ordered on one stream are safe.
 * Errors: TM_ERR_ARG (null pointers, nrhs > 64, nf not 1 or 2, bad Vh), TM_ERR_CUDA.
 */
tm_status tm_norm2_noalloc(const tm_field *x, int Vh, int nf, double *result_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TM_H */

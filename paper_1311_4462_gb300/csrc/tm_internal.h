// tm_internal.h -- declarations shared by the library's translation units (not installed).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>

#include "../../include/tm.h"

namespace tmk {

// NVTX range around a C-ABI call, named after the entry point (shown by Nsight tools; a push and a
// pop of a few nanoseconds when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
#define TM_NVTX(name) ::tmk::NvtxRange tm_nvtx_range_(name)

// kernel-level epilogue codes (see tm_dslash.cuh)
enum Epilogue {
    EPI_SCALE = 0,     // out = c acc
    EPI_TW = 1,        // out = T acc
    EPI_TWX_AXPY = 2,  // out = T x + c acc
    EPI_X_TWAXPY = 3,  // out = x + c T acc
    EPI_XPAY = 4,      // out = x + c acc
    EPI_TW_XPAY = 5,   // out = T (x + c acc)
    EPI_TWX_AXPY_TW = 6,  // out = Q (T x + c acc), Q a second constant local matrix
    EPI_TWX_AXPY_RUPD = 7  // out = out - s (T x + c acc), s = *scal_in: CG's residual update in place
                           // (staged launch forms with the fused reduction only)
};

// twist selector for host-built coefficient tables
enum TwistKind { TW_R = 0, TW_RINV = 1 };

// clover field of a handle (tm_clover.cu)
tm_status clover_build(tm_gauge *g, double csw, cudaStream_t s);
void clover_free(tm_gauge *g);
size_t clover_bytes(int pidx, long Vh);
// operator composition shared by the API and the solvers (tm_api.cu)
tm_status precond_core(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o, int pc,
                       int dagger, cudaStream_t s, const int *act, int nact);
struct RedArgs;
tm_status normal_core(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *te_e,
                      const tm_field *tmp_o, int pc, int dagger, cudaStream_t s, const int *act, int nact,
                      const RedArgs *red = nullptr);
bool normal_red_supported(const tm_gauge *g, int prec, int dagger);
tm_status adjoint_core(const tm_gauge *g, const tm_field *out_e, const tm_field *in_e, const tm_field *tmp_o, int pc,
                       int dagger, cudaStream_t s);
tm_status normal_rupd_core(const tm_gauge *g, const tm_field *r_e, const tm_field *p_e, const tm_field *te_e,
                           const tm_field *tmp_o, int pc, cudaStream_t s, const RedArgs *red_a, const RedArgs *red_r,
                           const double *alpha_dev);
}  // namespace tmk

// Launch choice of the hopping kernel for one (precision, prologue) pair.
struct tm_tune_entry {
    int variant;  // 0: one thread per site; 2: two-stage load pipeline; 3 / 4 / 5: register-capped
                  // (128 x 4, 64 x 8, 256 x 2 threads x blocks per SM)
    int block;    // threads per block
};

// The opaque handle behind tm_gauge*.
struct tm_gauge {
    tm_params p;
    int nf;
    int Vh, X1h;
    int device;
    int num_sms;
    void *links[4];     // packed links, index 0: FP64, 1: FP32, 2: FP16, 3: DF64
    size_t link_bytes[4];
    int recon[4];       // reals per stored link of each storage form (p.recon unless overridden)
    double *scratch;    // reduction partials + device scalars (library-owned)
    double *host_scalars;  // pinned mirror for scalar readback
    tm_tune_entry tune[4][2];  // [precision index][prologue]
    int multi_rpb[4];          // right-hand sides per block of the multi-RHS kernel (2, 4, 8)
    double csw;                // clover coefficient; 0: no clover term
    void *clov[3];             // per-site local clover operator, FP64 / FP32 / FP16 (tm_clover.cuh)
    float *clov_norm;          // FP16 block scales
    int clov_minb[3];          // clover kernel: resident blocks per SM its registers allow (1, 3, 4), 6: staged
    int fused[3];              // 1: the preconditioned operator as one fused launch (FP64 / FP32; FP16 unused)
    int *fused_items;          // device work list of the fused operator (2 x tiles entries)
    int fused_nitems;
    int fused_capacity;        // entries the device work list holds
    int *fused_sync;           // [0] error word, [1] work counter, [2] abort word, [3 + tile] A-tile flags
    unsigned long long wait_limit_ns;  // time limit of one bounded wait of the fused operator
    int dd;                    // 1: the handle holds the time slab [dd_t0, dd_t0 + L[3]) of a decomposed lattice
    int dd_t0, dd_Lt;          // slab offset and time extent of the whole lattice
    double dd_sign_b, dd_sign_f;  // boundary signs of the faces from the previous / next slab
    size_t scratch_bytes;
};

namespace tmk {
int prec_index(int prec);          // 0/1/2/3 for F64/F32/F16/DF64, -1 otherwise
size_t real_bytes(int prec);       // storage bytes per real
int spinor_chunks(int prec);       // 16-byte chunks per site and flavour
size_t chunk_bytes(int prec);      // always 16
void set_error(const char *fmt, ...);
tm_status cuda_check(cudaError_t e, const char *what);
tm_status need_links(const tm_gauge *g, int prec);  // TM_ERR_ARG when the handle did not pack prec
inline int link_recon(const tm_gauge *g, int pidx) { return g->recon[pidx]; }  // link format of a storage form
}  // namespace tmk

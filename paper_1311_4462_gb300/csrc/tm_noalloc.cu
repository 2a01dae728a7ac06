// tm_noalloc.cu -- |x|^2 of a spinor field for callers that cannot allocate device memory.
//
// Who needs it: code that owns no allocator of its own -- a host application that hands the
// library a fixed arena and forbids any other device allocation, a real-time or signal-safe
// loop where cudaMalloc's implicit synchronisation and possible failure are not acceptable,
// or a caller that does not want to create a tm_gauge handle (whose creation allocates the
// packed links and the reduction scratch) just to measure a field.  Such a caller passes its
// input field and a device buffer for the result; the reduction's per-block partial sums and
// its completion ticket live in the file-scope array below instead of in allocated memory.
#include <string.h>

#include <mutex>

#include "tm_blas.cuh"
#include "tm_internal.h"

namespace tmk {
cudaError_t launch_site_op_explicit(SiteOpArgs a, int Vh, int nf, int grid_x, int nrhs, cudaStream_t s);
}

namespace {

constexpr int NOALLOC_BLOCKS_PER_RHS = 256;  // grid.x of the reduction
constexpr size_t NOALLOC_PARTIALS = (size_t)NOALLOC_BLOCKS_PER_RHS * tmk::TM_MAX_RHS;
constexpr size_t NOALLOC_BYTES = NOALLOC_PARTIALS * sizeof(double) + 256;  // partials + ticket

// Reduction scratch shared by every call on a device; lives until the process exits.  The
// host never dereferences this name (in host code it is only a stand-in for the symbol); the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES];  // device address of g_noalloc_scratch per device (set up once)

tm_status scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) {
        tmk::set_error("tm_norm2_noalloc: device ordinal %d out of range", dev);
        return TM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return tmk::cuda_check(e, "tm_norm2_noalloc: cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return TM_OK;
}

}  // namespace

extern "C" tm_status tm_norm2_noalloc(const tm_field *x, int Vh, int nf, double *result_dev, void *stream)
{
    using namespace tmk;
    if (!x || !x->data || !result_dev) { set_error("tm_norm2_noalloc: null argument"); return TM_ERR_ARG; }
    if (prec_index(x->prec) < 0) { set_error("tm_norm2_noalloc: unknown precision %d", x->prec); return TM_ERR_ARG; }
    if (x->prec == TM_PREC_F16 && !x->norm) { set_error("tm_norm2_noalloc: FP16 field needs its norm array"); return TM_ERR_ARG; }
    if (nf != 1 && nf != 2) { set_error("tm_norm2_noalloc: nf must be 1 or 2"); return TM_ERR_ARG; }
    if (Vh < 1 || (long)Vh * nf > 0x7fffffffL) { set_error("tm_norm2_noalloc: Vh = %d out of range", Vh); return TM_ERR_ARG; }
    if (x->nrhs < 1 || x->nrhs > TM_MAX_RHS) {
        set_error("tm_norm2_noalloc: nrhs = %d exceeds the static scratch limit of %d right-hand sides", x->nrhs,
                  TM_MAX_RHS);
        return TM_ERR_ARG;
    }
    int dev = 0;
    tm_status st = cuda_check(cudaGetDevice(&dev), "tm_norm2_noalloc: cudaGetDevice");
    if (st != TM_OK) return st;
    void *base = nullptr;
    st = scratch_address(dev, &base);
    if (st != TM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = reinterpret_cast<double *>(base);
    unsigned *counter = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(base) + NOALLOC_PARTIALS * sizeof(double));
    // the completion ticket must start at zero (a failed earlier launch could have left it set)
    st = cuda_check(cudaMemsetAsync(counter, 0, sizeof(unsigned), s), "tm_norm2_noalloc: clear ticket");
    if (st != TM_OK) return st;
    SiteOpArgs a;
    memset(&a, 0, sizeof(a));
    a.op = OP_NORM;
    a.reduce = 1;
    a.A = fref(x);
    a.red.partials = partials;
    a.red.counter = counter;
    a.red.scalars = result_dev;  // column c of slot 0 is result_dev[c]
    a.red.fin = FIN_STORE;
    a.red.slot = 0;
    long gx = ((long)Vh * nf + 255) / 256;
    if (gx > NOALLOC_BLOCKS_PER_RHS) gx = NOALLOC_BLOCKS_PER_RHS;
    return cuda_check(launch_site_op_explicit(a, Vh, nf, (int)gx, x->nrhs, s), "tm_norm2_noalloc launch");
}

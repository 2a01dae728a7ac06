// Instantiations of the fused hopping kernels for DF64 storage (double-float arithmetic on the
// FP32 pipes): 2 flavour(s), 12-real links, thread-per-site and multi-RHS forms (no input-twist
// prologue: DF64 applies that twist as a separate launch).  One file per combination keeps
// each ptxas run short.
#include "tm_dslash.cuh"

namespace tmk {
cudaError_t launch_dslash_pdf_nf2_r12(const DslashArgs<df64> &a, int block, cudaStream_t s)
{
    const int grid = (a.Vh + block - 1) / block;
    k_dslash<PDF, 2, 12, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dslash_multi_pdf_nf2_r12(const DslashArgs<df64> &a, const int *act, int nact, int nrhs, cudaStream_t s)
{
    const unsigned grid = (unsigned)(((long)a.Vh + 31) / 32 * ((nact + 3) / 4));
    k_dslash_multi<PDF, 2, 12, false><<<grid, 128, 0, s>>>(a, act, nact, nrhs);
    return cudaGetLastError();
}
}  // namespace tmk

// Instantiations of the multi-RHS fused hopping kernel for FP64 storage (2, 4 and 8 right-hand
// sides per block; a translation unit of its own so it compiles in parallel with the rest).
#include "tm_dslash.cuh"

namespace tmk {
cudaError_t launch_dslash_multi_p64(const DslashArgs<double> &a, int nf, int recon, bool pro, const int *act, int nact,
                                    int nrhs, int rpb, cudaStream_t s)
{
    return launch_dslash_multi_impl<P64>(a, nf, recon, pro, act, nact, nrhs, rpb, s);
}
}  // namespace tmk

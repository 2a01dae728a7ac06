// Instantiations of the clover-twisted-mass hopping kernel for FP64 storage (a translation unit
// of its own so it compiles in parallel with the rest).
#include "tm_dslash.cuh"

namespace tmk {
cudaError_t launch_dslash_clov_p64(const DslashArgs<double> &a, int nf, int recon, int minb, cudaStream_t s)
{
    return launch_dslash_clov_impl<P64>(a, nf, recon, minb, s);
}
}  // namespace tmk

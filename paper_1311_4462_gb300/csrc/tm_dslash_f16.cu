// Instantiations of the single-RHS fused hopping kernels for FP16 storage (one translation unit per
// precision so the three compile in parallel).
#include "tm_dslash.cuh"

namespace tmk {
cudaError_t launch_dslash_p16(const DslashArgs<float> &a, int nf, int recon, bool pro, int variant, int block,
                              cudaStream_t s)
{
    return launch_dslash_impl<P16>(a, nf, recon, pro, variant, block, s);
}
cudaError_t launch_dslash_red_p16(const DslashArgs<float> &a, int nf, int recon, int variant, const RedArgs &red,
                                  cudaStream_t s)
{
    return launch_dslash_red_impl<P16>(a, nf, recon, variant, red, s);
}
}  // namespace tmk

// Instantiations of the fused preconditioned operator (both passes of M_pc in one persistent
// launch) for FP64 and FP32 storage.
#include "tm_dslash.cuh"

namespace tmk {
cudaError_t launch_fused_p64(const DslashArgs<double> &aA, const DslashArgs<double> &aB, int nf, int recon,
                             const int *items, int nitems, int *sync, unsigned long long limit_ns, int num_sms,
                             cudaStream_t s)
{
    return launch_fused_dispatch<P64>(aA, aB, nf, recon, items, nitems, sync, limit_ns, num_sms, s);
}
cudaError_t launch_fused_p32(const DslashArgs<float> &aA, const DslashArgs<float> &aB, int nf, int recon,
                             const int *items, int nitems, int *sync, unsigned long long limit_ns, int num_sms,
                             cudaStream_t s)
{
    return launch_fused_dispatch<P32>(aA, aB, nf, recon, items, nitems, sync, limit_ns, num_sms, s);
}
}  // namespace tmk

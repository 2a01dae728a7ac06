// Instantiations of the domain-decomposition kernels (face pack and the boundary-slice hopping
// launch of a slab, tm_dslash.cuh) for FP64, FP32 and FP16 storage.
#include "tm_dslash.cuh"

namespace tmk {
cudaError_t launch_dd_p64(const DslashArgs<double> &a, const DDArgs<double> *dd, void *face_prev, void *face_next,
                          int nf, int recon, bool pro, cudaStream_t s)
{
    return launch_dd_impl<P64>(a, dd, face_prev, face_next, nf, recon, pro, s);
}
cudaError_t launch_dd_p32(const DslashArgs<float> &a, const DDArgs<float> *dd, void *face_prev, void *face_next,
                          int nf, int recon, bool pro, cudaStream_t s)
{
    return launch_dd_impl<P32>(a, dd, face_prev, face_next, nf, recon, pro, s);
}
cudaError_t launch_dd_p16(const DslashArgs<float> &a, const DDArgs<float> *dd, void *face_prev, void *face_next,
                          int nf, int recon, bool pro, cudaStream_t s)
{
    return launch_dd_impl<P16>(a, dd, face_prev, face_next, nf, recon, pro, s);
}
size_t dd_face_bytes(int prec, int nf, int st)
{
    switch (prec) {
    case TM_PREC_F64: return FaceGeo<P64>::bytes(nf, st);
    case TM_PREC_F32: return FaceGeo<P32>::bytes(nf, st);
    case TM_PREC_F16: return FaceGeo<P16>::bytes(nf, st);
    default: return 0;
    }
}
}  // namespace tmk

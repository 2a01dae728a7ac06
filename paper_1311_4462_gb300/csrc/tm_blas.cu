// tm_blas.cu -- site-wise kernels on parity fields: the standalone local twist.
#include "tm_core.cuh"
#include "tm_internal.h"

namespace tmk {

// thread per (rhs, cb): both flavours of the site are twisted together (tau1 mixes them)
template <int PREC, int NF>
__global__ void k_twist(void *out, float *out_norm, const void *in, const float *in_norm, int Vh, int nrhs,
                        Twist<typename Traits<PREC>::real> tw)
{
    using T = typename Traits<PREC>::real;
    using SC = typename Traits<PREC>::schunk;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)Vh * nrhs) return;
    const int cb = (int)(id % Vh);
    const long rhs = id / Vh;
    const long fstride = (long)Traits<PREC>::SCHUNKS * Vh;
    T v[NF][24];
#pragma unroll
    for (int f = 0; f < NF; f++) {
        const long blk = rhs * NF + f;
        load_spinor<PREC>(reinterpret_cast<const SC *>(in) + blk * fstride, in_norm ? in_norm + blk * Vh : nullptr, cb,
                          Vh, v[f]);
    }
    apply_twist<T, NF>(tw, v);
#pragma unroll
    for (int f = 0; f < NF; f++) {
        const long blk = rhs * NF + f;
        store_spinor<PREC>(reinterpret_cast<SC *>(out) + blk * fstride, out_norm ? out_norm + blk * Vh : nullptr, cb,
                           Vh, v[f]);
    }
}

template <typename T>
static Twist<T> cast_twist(const Twist<double> &t)
{
    Twist<T> o;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            for (int k = 0; k < 2; k++) o.m[i][j][k] = {(T)t.m[i][j][k].r, (T)t.m[i][j][k].i};
    return o;
}

cudaError_t launch_twist(const tm_gauge *g, const tm_field *out, const tm_field *in, const Twist<double> &tw,
                         cudaStream_t s)
{
    const long n = (long)g->Vh * out->nrhs;
    const int block = 128;
    const long grid = (n + block - 1) / block;
#define TM_T(P, NF, TT) \
    k_twist<P, NF><<<grid, block, 0, s>>>(out->data, out->norm, in->data, in->norm, g->Vh, out->nrhs, cast_twist<TT>(tw))
    if (g->nf == 1) {
        if (in->prec == TM_PREC_F64) TM_T(P64, 1, double);
        else if (in->prec == TM_PREC_F32) TM_T(P32, 1, float);
        else TM_T(P16, 1, float);
    } else {
        if (in->prec == TM_PREC_F64) TM_T(P64, 2, double);
        else if (in->prec == TM_PREC_F32) TM_T(P32, 2, float);
        else TM_T(P16, 2, float);
    }
#undef TM_T
    return cudaGetLastError();
}

}  // namespace tmk

// 2D AD-LBR stencil construction, one thread per grid point (the per-point
// construction and its certification are in stencil2d.cuh).
#include "stencil2d.cuh"

namespace adlbr {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) build2d_kernel(int64_t N, const T *__restrict__ D,
                                                      short4 *__restrict__ offs, void *wbase,
                                                      adlbr_dtype wt, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    build_point2d<T>(D[i], D[N + i], D[2 * N + i], i, offs, wbase, wt, err);
}

}  // namespace

adlbr_status launch_build2d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st) {
    ADLBR_NVTX("build");
    stencils_changed(s);
    const int threads = 256;
    unsigned blocks = blocks_for(s->N, threads);
    if (D_t == ADLBR_F32)
        build2d_kernel<float><<<blocks, threads, 0, st>>>(s->N, (const float *)D, (short4 *)s->offs,
                                                          s->w, s->w_t, s->err);
    else
        build2d_kernel<double><<<blocks, threads, 0, st>>>(s->N, (const double *)D,
                                                           (short4 *)s->offs, s->w, s->w_t, s->err);
    ADLBR_CUDA(cudaGetLastError());
    s->built = 1;
    return ADLBR_OK;
}

}  // namespace adlbr

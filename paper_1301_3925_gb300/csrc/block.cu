// Block-vector kernels of the periodic spectral study (Sec. 4, Fig. Eigen).
// The block eigensolver over the operator's smallest eigenvalues needs,
// besides A X (the operator), the Gram matrices of its search blocks, linear
// combinations of their rows and the residual rows R = A X - theta X.
// Blocks are m rows of n FP64 values, row-major with row stride n.  FP64
// throughout; every sum is taken by one CTA in a fixed order, so the
// results do not depend on the launch.
#include "internal.cuh"

namespace adlbr {

namespace {

constexpr int BT = 256;
constexpr int kMaxRows = 64;     // rows of a block (the eigensolver uses 3 x its block size)
constexpr int kCombine = 8;      // output rows per pass of the combination kernel

// Sum over the CTA in a fixed order (warp shuffles, then the first warp);
// the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double part[BT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = lane < BT / 32 ? part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// G[i][j] = <A_i, B_j>, one CTA per (i, j)
__global__ void __launch_bounds__(BT) block_dot_kernel(const double *__restrict__ A, const double *__restrict__ B,
                                                       int mb, int64_t n, double *__restrict__ G) {
    const int i = blockIdx.x / mb, j = blockIdx.x - i * mb;
    const double *a = A + (int64_t)i * n, *b = B + (int64_t)j * n;
    double s = 0.0;
    for (int64_t p = threadIdx.x; p < n; p += BT) s = fma(a[p], b[p], s);
    s = block_sum(s);
    if (threadIdx.x == 0) G[blockIdx.x] = s;
}

// out_r = sum_i C[i][r] S_i for r < k, one thread per column p; the sum runs
// over i in order
__global__ void __launch_bounds__(BT) block_combine_kernel(const double *__restrict__ C, int m, int k,
                                                           const double *__restrict__ S, int64_t n,
                                                           double *__restrict__ out) {
    __shared__ double c[kMaxRows * kMaxRows];
    for (int t = threadIdx.x; t < m * k; t += BT) c[t] = C[t];
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (p >= n) return;
    for (int r0 = 0; r0 < k; r0 += kCombine) {
        double acc[kCombine];
#pragma unroll
        for (int q = 0; q < kCombine; ++q) acc[q] = 0.0;
        for (int i = 0; i < m; ++i) {
            const double s = S[(int64_t)i * n + p];
#pragma unroll
            for (int q = 0; q < kCombine; ++q)
                if (r0 + q < k) acc[q] = fma(c[i * k + r0 + q], s, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < kCombine; ++q)
            if (r0 + q < k) out[(int64_t)(r0 + q) * n + p] = acc[q];
    }
}

// R_i = AX_i - theta_i X_i and ||R_i||, one CTA per row (R may be AX: each
// element is read and then written by the same thread)
__global__ void __launch_bounds__(BT) block_residual_kernel(const double *AX, const double *__restrict__ X,
                                                            const double *__restrict__ theta, int64_t n,
                                                            double *R, double *__restrict__ rnorm) {
    const int64_t off = (int64_t)blockIdx.x * n;
    const double th = theta[blockIdx.x];
    double s = 0.0;
    for (int64_t p = threadIdx.x; p < n; p += BT) {
        const double r = fma(-th, X[off + p], AX[off + p]);
        R[off + p] = r;
        s = fma(r, r, s);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) rnorm[blockIdx.x] = sqrt(s);
}

}  // namespace

}  // namespace adlbr

using namespace adlbr;

adlbr_status adlbr_block_dot(const double *A, int ma, const double *B, int mb, int64_t n, double *G,
                             cudaStream_t stream) {
    ADLBR_NVTX("block_dot");
    if (!A || !B || !G || ma < 1 || mb < 1 || ma > kMaxRows || mb > kMaxRows || n < 1)
        return fail(ADLBR_E_ARG, "block_dot: bad argument");
    block_dot_kernel<<<ma * mb, BT, 0, stream>>>(A, B, mb, n, G);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status adlbr_block_combine(const double *C, int m, int k, const double *S, int64_t n, double *out,
                                 cudaStream_t stream) {
    ADLBR_NVTX("block_combine");
    if (!C || !S || !out || m < 1 || k < 1 || m > kMaxRows || k > kMaxRows || n < 1)
        return fail(ADLBR_E_ARG, "block_combine: bad argument");
    block_combine_kernel<<<blocks_for(n, BT), BT, 0, stream>>>(C, m, k, S, n, out);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status adlbr_block_residual(const double *AX, const double *X, const double *theta, int m, int64_t n,
                                  double *R, double *rnorm, cudaStream_t stream) {
    ADLBR_NVTX("block_residual");
    if (!AX || !X || !theta || !R || !rnorm || m < 1 || m > kMaxRows || n < 1)
        return fail(ADLBR_E_ARG, "block_residual: bad argument");
    block_residual_kernel<<<m, BT, 0, stream>>>(AX, X, theta, n, R, rnorm);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

// The 3D coherence-enhancing tensor (Sec. 5, 3D experiments, following the 2D
// definition of Sec. 4.4): u_sigma = K_sigma * u, J_rho = K_rho * (grad
// u_sigma grad u_sigma^T) with six channels (xx, yy, zz, xy, xz, yz), and
// D(J) with the eigenvectors of J and, for eigenvalues mu1 >= mu2 >= mu3,
//   lambda1 = alpha,
//   lambda2 = alpha + (1 - alpha) exp(-C / (mu1 - mu2)^2),
//   lambda3 = alpha + (1 - alpha) exp(-C / (mu1 - mu3)^2),
// exp(-C/0) = 0.  Readings as in 2D: standard deviations, truncation at
// int(3 s + 0.5), normalised taps, every stage reflects its own input.
//
// The edge-enhancing tensor of the 3D MRI experiment (Sec. 5) shares J_rho
// and the eigenvectors and takes
//   lambda1 = 1 - exp(-C / mu1^2), lambda2 = 1 - exp(-C / mu2^2), lambda3 = 1,
// with exp(-C/0) = 0 and 1 - exp(-x) evaluated as -expm1(-x).
//
// Kernels: one Gaussian pass per axis (x, y, z) on C channels, one thread per
// output (neighbours read from L1/L2; a warp covers consecutive x, so every
// axis reads coalesced rows), the gradient outer product, and the 3 x 3
// eigen-decomposition by cyclic Jacobi rotations in FP32 with the tensor
// assembled from it.  D is continuous in J at repeated eigenvalues (the
// lambdas of a repeated pair coincide), so the FP32 eigenvectors suffice.
#include "ced_common.cuh"

namespace adlbr {

using ced::kMaxR;
using ced::make_taps;
using ced::radius_of;
using ced::reflect;
using ced::Taps;

namespace {

constexpr int BT = 128;   // threads per block, along x

// out[c] = Gaussian of in[c] along AXIS (0 = x, 1 = y, 2 = z), reflected.
template <int C, int AXIS>
__global__ void __launch_bounds__(BT) blur3_kernel(int nx, int ny, int nz, int64_t N, int r, Taps tp,
                                                   const float *__restrict__ in, float *__restrict__ out) {
    const int x = blockIdx.x * BT + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t p = z * sz + y * sy + x;
    const int n = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
    const int c0 = AXIS == 0 ? x : (AXIS == 1 ? y : z);
    const int64_t st = AXIS == 0 ? sx : (AXIS == 1 ? sy : sz);
    const int64_t base = p - (int64_t)c0 * st;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *a = in + c * N + base;
        float acc = __fmul_rn(tp.t[0], a[(int64_t)c0 * st]);
        for (int k = 1; k <= r; ++k)
            acc = __fmaf_rn(tp.t[k],
                            __fadd_rn(a[(int64_t)reflect(c0 - k, n) * st], a[(int64_t)reflect(c0 + k, n) * st]),
                            acc);
        out[c * N + p] = acc;
    }
}

// (gx gx, gy gy, gz gz, gx gy, gx gz, gy gz) of the centred differences of us.
__global__ void __launch_bounds__(BT) grad_outer3_kernel(int nx, int ny, int nz, int64_t N,
                                                         const float *__restrict__ us, float *__restrict__ P) {
    const int x = blockIdx.x * BT + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t p = z * sz + y * sy + x;
    const float *row = us + z * sz + y * sy;
    const float gx = __fmul_rn(0.5f, __fsub_rn(row[reflect(x + 1, nx)], row[reflect(x - 1, nx)]));
    const float *col = us + z * sz + x;
    const float gy = __fmul_rn(0.5f, __fsub_rn(col[reflect(y + 1, ny) * sy], col[reflect(y - 1, ny) * sy]));
    const float *pil = us + y * sy + x;
    const float gz = __fmul_rn(0.5f, __fsub_rn(pil[reflect(z + 1, nz) * sz], pil[reflect(z - 1, nz) * sz]));
    P[p] = __fmul_rn(gx, gx);
    P[N + p] = __fmul_rn(gy, gy);
    P[2 * N + p] = __fmul_rn(gz, gz);
    P[3 * N + p] = __fmul_rn(gx, gy);
    P[4 * N + p] = __fmul_rn(gx, gz);
    P[5 * N + p] = __fmul_rn(gy, gz);
}

// One Jacobi rotation annihilating a[p][q] of the symmetric 3 x 3 matrix a,
// accumulated into the columns of v.
__device__ __forceinline__ void jacobi_rotate(float (&a)[3][3], float (&v)[3][3], int p, int q) {
    const float apq = a[p][q];
    if (apq == 0.f) return;
    const float theta = (a[q][q] - a[p][p]) / (2.f * apq);
    const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
    const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
    a[p][p] -= t * apq;
    a[q][q] += t * apq;
    a[p][q] = a[q][p] = 0.f;
    const int r = 3 - p - q;
    const float arp = a[r][p], arq = a[r][q];
    a[r][p] = a[p][r] = c * arp - s * arq;
    a[r][q] = a[q][r] = s * arp + c * arq;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
    }
}

__device__ __forceinline__ float lam_of(float d, float alpha, float C) {
    // alpha + (1 - alpha) exp(-C / d^2); exp(-C/0) = 0
    if (!(d > 0.f)) return alpha;
    return fmaf(1.f - alpha, expf(-C / (d * d)), alpha);
}

// lambda of the edge-enhancing tensor for the eigenvalue m of J
__device__ __forceinline__ float eed_lam(float m, float C) {
    const float q = m * m;
    return q > 0.f ? -expm1f(-C / q) : 1.f;
}

template <bool EED>
__global__ void __launch_bounds__(BT) tensor3_kernel(int64_t N, const float *__restrict__ J, float *__restrict__ D,
                                                     float alpha, float C) {
    const int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (i >= N) return;
    float a[3][3] = {{J[i], J[3 * N + i], J[4 * N + i]},
                     {J[3 * N + i], J[N + i], J[5 * N + i]},
                     {J[4 * N + i], J[5 * N + i], J[2 * N + i]}};
    float v[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
    const float scale = fabsf(a[0][0]) + fabsf(a[1][1]) + fabsf(a[2][2]) + fabsf(a[0][1]) + fabsf(a[0][2]) +
                        fabsf(a[1][2]);
    for (int sweep = 0; sweep < 8; ++sweep) {
        const float off = fabsf(a[0][1]) + fabsf(a[0][2]) + fabsf(a[1][2]);
        if (!(off > 1e-9f * scale)) break;
        jacobi_rotate(a, v, 0, 1);
        jacobi_rotate(a, v, 0, 2);
        jacobi_rotate(a, v, 1, 2);
    }
    // order: mu1 >= mu2 >= mu3
    int o[3] = {0, 1, 2};
    const float mu[3] = {a[0][0], a[1][1], a[2][2]};
    if (mu[o[0]] < mu[o[1]]) { const int t = o[0]; o[0] = o[1]; o[1] = t; }
    if (mu[o[1]] < mu[o[2]]) { const int t = o[1]; o[1] = o[2]; o[2] = t; }
    if (mu[o[0]] < mu[o[1]]) { const int t = o[0]; o[0] = o[1]; o[1] = t; }
    float l[3];
    if (EED) {
        l[0] = eed_lam(mu[o[0]], C);
        l[1] = eed_lam(mu[o[1]], C);
        l[2] = 1.f;
    } else {
        l[0] = alpha;
        l[1] = lam_of(mu[o[0]] - mu[o[1]], alpha, C);
        l[2] = lam_of(mu[o[0]] - mu[o[2]], alpha, C);
    }
    float d[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    constexpr int R[6] = {0, 1, 2, 0, 0, 1}, S[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int c = o[k];
#pragma unroll
        for (int e = 0; e < 6; ++e) d[e] = fmaf(l[k] * v[R[e]][c], v[S[e]][c], d[e]);
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) D[e * N + i] = d[e];
}

}  // namespace

size_t ced_tensor3d_scratch_bytes(int64_t N) { return (size_t)N * sizeof(float) * 12; }

namespace {

adlbr_status tensor3d(int nx, int ny, int nz, const float *u, float *D, double sigma, double rho, double alpha,
                      double C, bool eed, void *scratch, cudaStream_t st) {
    const int rs = radius_of(sigma), rr = radius_of(rho);
    if (rs > kMaxR || rr > kMaxR) return fail(ADLBR_E_ARG, "Gaussian radius above %d", kMaxR);
    const Taps ts = make_taps(sigma), tr = make_taps(rho);
    const int64_t N = (int64_t)nx * ny * nz;
    float *A = (float *)scratch, *B = A + 6 * N;
    const dim3 g(blocks_for(nx, BT), (unsigned)ny, (unsigned)nz);
    blur3_kernel<1, 0><<<g, BT, 0, st>>>(nx, ny, nz, N, rs, ts, u, A);
    blur3_kernel<1, 1><<<g, BT, 0, st>>>(nx, ny, nz, N, rs, ts, A, B);
    blur3_kernel<1, 2><<<g, BT, 0, st>>>(nx, ny, nz, N, rs, ts, B, A);
    grad_outer3_kernel<<<g, BT, 0, st>>>(nx, ny, nz, N, A, B);
    blur3_kernel<6, 0><<<g, BT, 0, st>>>(nx, ny, nz, N, rr, tr, B, A);
    blur3_kernel<6, 1><<<g, BT, 0, st>>>(nx, ny, nz, N, rr, tr, A, B);
    blur3_kernel<6, 2><<<g, BT, 0, st>>>(nx, ny, nz, N, rr, tr, B, A);
    if (eed)
        tensor3_kernel<true><<<blocks_for(N, BT), BT, 0, st>>>(N, A, D, 0.f, (float)C);
    else
        tensor3_kernel<false><<<blocks_for(N, BT), BT, 0, st>>>(N, A, D, (float)alpha, (float)C);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace

adlbr_status launch_ced_tensor3d(int nx, int ny, int nz, const float *u, float *D, double sigma, double rho,
                                 double alpha, double C, void *scratch, cudaStream_t st) {
    ADLBR_NVTX("tensor");
    if (!(sigma > 0) || !(rho > 0) || !(alpha > 0 && alpha <= 1) || !(C >= 0))
        return fail(ADLBR_E_ARG, "bad CED parameters");
    return tensor3d(nx, ny, nz, u, D, sigma, rho, alpha, C, false, scratch, st);
}

adlbr_status launch_eed_tensor3d(int nx, int ny, int nz, const float *u, float *D, double sigma, double rho,
                                 double C, void *scratch, cudaStream_t st) {
    ADLBR_NVTX("tensor");
    // C > 0: with C = 0 every direction of non-zero mu would get lambda = 0
    if (!(sigma > 0) || !(rho > 0) || !(C > 0) || !std::isfinite(C)) return fail(ADLBR_E_ARG, "bad EED parameters");
    return tensor3d(nx, ny, nz, u, D, sigma, rho, 0.0, C, true, scratch, st);
}

}  // namespace adlbr

// Coherence-enhancing diffusion (Sec. 4.4, Eq. parabolique): the tensor
// stage D(J_rho(grad u_sigma)),
//   u_sigma = K_sigma * u,  J_rho = K_rho * (grad u_sigma grad u_sigma^T),
//   D = alpha v1 v1^T + lambda2 v2 v2^T,
//   lambda2 = alpha + (1 - alpha) exp(-C / (mu1 - mu2)^2),
// followed (adlbr_ced_stencils) by the AD-LBR stencil construction of D.
//
// sigma and rho are standard deviations; kernels are truncated at
// int(3 s + 0.5) and normalised; every stage reflects its own input about the
// border (u(-1) = u(0)): the Gaussians and the centred-difference gradient.
//
// Kernels: separable Gaussian passes staged through shared memory (a row
// segment plus halo for the x pass, a column band plus halo for the y pass),
// the gradient and outer product in one pass, and the 2x2 eigen-
// decomposition fused into the epilogue of the last (y) pass.
#include "ced_common.cuh"
#include "stencil2d.cuh"

namespace adlbr {

using ced::d_from_j;
using ced::kMaxR;
using ced::make_taps;
using ced::radius_of;
using ced::reflect;
using ced::Taps;

namespace {

// Each thread produces RB consecutive outputs along the blur direction from
// RB + 2r staged values (register blocking), so a 25-tap pass reads about
// 7 values from shared memory per output instead of 25.
constexpr int RB = 4;
constexpr int TXT = 128;            // x pass: threads per block
constexpr int TX = TXT * RB;        // x pass: outputs per block (one row segment)

// out[c][y][x] = sum_k taps[|k|] in[c][y][reflect(x + k)]
template <int C>
__global__ void __launch_bounds__(TXT) blur_x_kernel(int nx, int ny, int64_t N, int r, Taps tp,
                                                     const float *__restrict__ in,
                                                     float *__restrict__ out) {
    extern __shared__ float smx[];  // C * (TX + 2r)
    const int x0 = blockIdx.x * TX, y = blockIdx.y;
    const int W = TX + 2 * r;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *row = in + c * N + (int64_t)y * nx;
        for (int j = threadIdx.x; j < W; j += TXT) smx[c * W + j] = row[reflect(x0 - r + j, nx)];
    }
    __syncthreads();
    const int xb = x0 + RB * threadIdx.x;
    if (xb >= nx) return;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *s = smx + c * W + RB * threadIdx.x + r;  // s[j] = in[xb + j]
        float acc[RB];
#pragma unroll
        for (int o = 0; o < RB; ++o) acc[o] = __fmul_rn(tp.t[0], s[o]);
        for (int k = 1; k <= r; ++k) {
            float lo[RB], hi[RB];
#pragma unroll
            for (int o = 0; o < RB; ++o) {
                lo[o] = s[o - k];
                hi[o] = s[o + k];
            }
#pragma unroll
            for (int o = 0; o < RB; ++o) acc[o] = __fmaf_rn(tp.t[k], __fadd_rn(lo[o], hi[o]), acc[o]);
        }
        float *dst = out + c * N + (int64_t)y * nx + xb;
#pragma unroll
        for (int o = 0; o < RB; ++o)
            if (xb + o < nx) dst[o] = acc[o];
    }
}

constexpr int BX = 32, BY = 32;  // y pass tile; 8 rows of threads, RB rows each

// y pass; EPI 0: plain store; EPI 1: the channels are (Jxx, Jxy, Jyy) and the
// epilogue writes D(J) (three planes) instead.
template <int C, int EPI>
__global__ void __launch_bounds__(BX * 8) blur_y_kernel(int nx, int ny, int64_t N, int r, Taps tp,
                                                        const float *__restrict__ in,
                                                        float *__restrict__ out, float alpha,
                                                        float Cc) {
    extern __shared__ float smy[];  // C * (BY + 2r) * BX
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int H = BY + 2 * r;
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int x = x0 + tx;
    const bool xin = x < nx;
#pragma unroll
    for (int c = 0; c < C; ++c)
        for (int j = ty; j < H; j += 8) {
            int yy = reflect(y0 - r + j, ny);
            smy[(c * H + j) * BX + tx] = xin ? in[c * N + (int64_t)yy * nx + x] : 0.f;
        }
    __syncthreads();
    if (!xin) return;
    const int oy0 = RB * ty;  // this thread's rows: oy0 .. oy0 + RB - 1
    float v[C][RB];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *s = smy + (c * H + oy0 + r) * BX + tx;  // s[j * BX] = row oy0 + j
#pragma unroll
        for (int o = 0; o < RB; ++o) v[c][o] = __fmul_rn(tp.t[0], s[o * BX]);
        for (int k = 1; k <= r; ++k) {
            float lo[RB], hi[RB];
#pragma unroll
            for (int o = 0; o < RB; ++o) {
                lo[o] = s[(o - k) * BX];
                hi[o] = s[(o + k) * BX];
            }
#pragma unroll
            for (int o = 0; o < RB; ++o) v[c][o] = __fmaf_rn(tp.t[k], __fadd_rn(lo[o], hi[o]), v[c][o]);
        }
    }
#pragma unroll
    for (int o = 0; o < RB; ++o) {
        const int y = y0 + oy0 + o;
        if (y >= ny) break;
        const int64_t z = (int64_t)y * nx + x;
        if (EPI == 0) {
#pragma unroll
            for (int c = 0; c < C; ++c) out[c * N + z] = v[c][o];
        } else {
            float dxx, dxy, dyy;
            d_from_j(v[0][o], v[1][o], v[2][o], alpha, Cc, dxx, dxy, dyy);
            out[z] = dxx;
            out[N + z] = dxy;
            out[2 * N + z] = dyy;
        }
    }
}

// (gx^2, gx gy, gy^2) of the centred differences of us, reflected border.
__global__ void grad_outer_kernel(int nx, int ny, int64_t N, const float *__restrict__ us,
                                  float *__restrict__ P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const float *row = us + (int64_t)y * nx;
    const float gx = __fmul_rn(0.5f, __fsub_rn(row[reflect(x + 1, nx)], row[reflect(x - 1, nx)]));
    const float gy = __fmul_rn(0.5f, __fsub_rn(us[(int64_t)reflect(y + 1, ny) * nx + x],
                                                us[(int64_t)reflect(y - 1, ny) * nx + x]));
    const int64_t z = (int64_t)y * nx + x;
    P[z] = __fmul_rn(gx, gx);
    P[N + z] = __fmul_rn(gx, gy);
    P[2 * N + z] = __fmul_rn(gy, gy);
}

adlbr_status separable_tensor(int nx, int ny, const float *u, float *D, int rs, int rr, const Taps &ts,
                             const Taps &tr, float alpha, float C, void *scratch, cudaStream_t st) {
    const int64_t N = (int64_t)nx * ny;
    float *A = (float *)scratch;  // 3N
    float *B = A + 3 * N;         // 3N
    dim3 gx(blocks_for(nx, TX), ny), gy(blocks_for(nx, BX), blocks_for(ny, BY));
    blur_x_kernel<1><<<gx, TXT, (TX + 2 * rs) * sizeof(float), st>>>(nx, ny, N, rs, ts, u, A);
    blur_y_kernel<1, 0><<<gy, BX * 8, (BY + 2 * rs) * BX * sizeof(float), st>>>(nx, ny, N, rs, ts, A,
                                                                                   B, 0.f, 0.f);
    grad_outer_kernel<<<dim3(blocks_for(nx, 256), ny), 256, 0, st>>>(nx, ny, N, B, A);
    blur_x_kernel<3><<<gx, TXT, 3 * (TX + 2 * rr) * sizeof(float), st>>>(nx, ny, N, rr, tr, A, B);
    size_t smy = 3 * (BY + 2 * rr) * BX * sizeof(float);
    ADLBR_CUDA(cudaFuncSetAttribute(blur_y_kernel<3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smy));
    blur_y_kernel<3, 1><<<gy, BX * 8, smy, st>>>(nx, ny, N, rr, tr, B, D, alpha, C);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status check_params(double sigma, double rho, double alpha, double C) {
    if (!(sigma > 0) || !(rho > 0) || !(alpha > 0 && alpha <= 1) || !(C >= 0))
        return fail(ADLBR_E_ARG, "bad CED parameters");
    if (radius_of(sigma) > kMaxR || radius_of(rho) > kMaxR)
        return fail(ADLBR_E_ARG, "Gaussian radius above %d", kMaxR);
    return ADLBR_OK;
}

}  // namespace

size_t ced_tensor_scratch_bytes(int64_t N) { return (size_t)N * sizeof(float) * 6; }

adlbr_status launch_ced_tensor(int nx, int ny, const float *u, float *D, double sigma, double rho,
                               double alpha, double C, void *scratch, cudaStream_t st) {
    if (adlbr_status e = check_params(sigma, rho, alpha, C)) return e;
    return separable_tensor(nx, ny, u, D, radius_of(sigma), radius_of(rho), make_taps(sigma),
                            make_taps(rho), (float)alpha, (float)C, scratch, st);
}

adlbr_status launch_ced_build(adlbr_stencils *s, const float *u, double sigma, double rho,
                              double alpha, double C, void *scratch, float *Dtmp, cudaStream_t st) {
    if (adlbr_status e = launch_ced_tensor((int)s->n[0], (int)s->n[1], u, Dtmp, sigma, rho, alpha, C,
                                           scratch, st))
        return e;
    return launch_build2d(s, Dtmp, ADLBR_F32, st);
}

}  // namespace adlbr

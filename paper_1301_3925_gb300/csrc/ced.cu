// Coherence-enhancing diffusion (Sec. 4.4, Eq. parabolique): the tensor
// stage D(J_rho(grad u_sigma)),
//   u_sigma = K_sigma * u,  J_rho = K_rho * (grad u_sigma grad u_sigma^T),
//   D = alpha v1 v1^T + lambda2 v2 v2^T,
//   lambda2 = alpha + (1 - alpha) exp(-C / (mu1 - mu2)^2),
// optionally fused with the AD-LBR stencil construction of D.
//
// sigma and rho are standard deviations; kernels are truncated at
// int(3 s + 0.5) and normalised; every stage reflects its own input about the
// border (u(-1) = u(0)): the Gaussians and the centred-difference gradient.
//
// Main kernel (streaming): a CTA owns a strip of SW output columns and a
// segment of rows and marches down the rows four at a time, keeping ring
// buffers of the intermediate rows (x-blurred u, u_sigma, x-blurred
// products) in shared memory.  Each intermediate row is computed once per
// strip (only the 2H-column halo is recomputed by the neighbouring strip and
// H + a few rows at each segment start), the x-blurs are register-blocked
// over 4 columns and the y-blurs over the 4 rows of a group, and the
// epilogue either writes D or builds the stencil from D in registers, so D
// never travels through HBM.  Supported radii are compiled in (sigma = 1 or
// 0.5 with rho = 4); other radii use the separable multi-kernel fallback.
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

// =================================================================== streaming
constexpr int G = 4;      // rows per group
constexpr int SW = 96;    // output columns per strip
constexpr int CT = 128;   // threads per CTA
constexpr int SH = 128;   // output rows per segment

struct StreamArgs {
    int nx, ny;
    float alpha, C;
    Taps ts, tr;
    const float *u;
    float *D;          // MODE 0
    short4 *offs;      // MODE 1
    void *wbase;
    adlbr_dtype wt;
    int *err;
};

template <int RS, int RR>
struct Geo {
    static constexpr int H = RR + 1 + RS;
    static constexpr int WU = SW + 2 * H;      // smem row width (global columns x0-H .. x0+SW+H)
    static constexpr int capB = 2 * RS + G;
    static constexpr int capS = 2 + G;
    static constexpr int capT = 2 * RR + G;
    static constexpr int oU = 0;
    static constexpr int oB = oU + G * WU;
    static constexpr int oS = oB + capB * WU;
    static constexpr int oP = oS + capS * WU;
    static constexpr int oT = oP + 3 * G * WU;
    static constexpr int total = oT + capT * 3 * SW;  // floats
    static_assert(WU <= CT, "a row must fit one pass of the CTA");
};

template <int RS, int RR, int MODE>
__global__ void __launch_bounds__(CT) ced_stream_kernel(StreamArgs A) {
    using GG = Geo<RS, RR>;
    extern __shared__ __align__(16) float sm[];
    float *Urow = sm + GG::oU;  // [G][WU]
    float *Bx = sm + GG::oB;    // [capB][WU]
    float *Us = sm + GG::oS;    // [capS][WU]
    float *Pr = sm + GG::oP;    // [G][3][WU]
    float *T3 = sm + GG::oT;    // [capT][3][SW]
    const int nx = A.nx, ny = A.ny;
    const int x0 = blockIdx.x * SW;
    const int cbase = x0 - GG::H;
    const int ys = blockIdx.y * SH, ye = min(ny, ys + SH);
    const int cu0 = max(0, x0 - GG::H), cu1 = min(nx, x0 + SW + GG::H);
    const int cs0 = max(0, x0 - RR - 1), cs1 = min(nx, x0 + SW + RR + 1);
    const int cp0 = max(0, x0 - RR), cp1 = min(nx, x0 + SW + RR);
    const int co1 = min(nx, x0 + SW);
    const int p_first = max(0, ys - RR), p_last = min(ny - 1, ye - 1 + RR);
    const int s_first = max(0, p_first - 1), s_last = min(ny - 1, p_last + 1);
    const int b_first = max(0, s_first - RS), b_last = min(ny - 1, s_last + RS);
    const int tid = threadIdx.x;

    for (int b0 = b_first; b0 - RS - 1 - RR <= ye - 1; b0 += G) {
        // ---- stage 1: u rows b0 .. b0+G-1 over [cu0, cu1)
        {
            const int g = tid >> 5, lane = tid & 31;
            const int row = b0 + g;
            if (row <= b_last)
                for (int c = cu0 + lane; c < cu1; c += 32)
                    Urow[g * GG::WU + c - cbase] = A.u[(int64_t)row * nx + c];
        }
        __syncthreads();
        // ---- stage 2: Bx = x-blur(sigma) of those rows over [cs0, cs1), 4 columns / thread
        {
            const int g = tid >> 5, lane = tid & 31;
            const int row = b0 + g;
            const int c0 = cs0 + 4 * lane;
            if (row <= b_last && c0 < cs1) {
                const float *U = Urow + g * GG::WU;
                float v[4 + 2 * RS];
#pragma unroll
                for (int j = 0; j < 4 + 2 * RS; ++j) v[j] = U[reflect(c0 - RS + j, nx) - cbase];
                float *dst = Bx + (row % GG::capB) * GG::WU;
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    if (c0 + o >= cs1) break;
                    float acc = __fmul_rn(A.ts.t[0], v[o + RS]);
#pragma unroll
                    for (int k = 1; k <= RS; ++k)
                        acc = __fmaf_rn(A.ts.t[k], __fadd_rn(v[o + RS - k], v[o + RS + k]), acc);
                    dst[c0 + o - cbase] = acc;
                }
            }
        }
        __syncthreads();
        // ---- stage 3: u_sigma rows s0 .. s0+3 (y-blur of Bx) over [cs0, cs1)
        const int s0 = b0 - RS;
        {
            const int c = cs0 + tid;
            if (c < cs1) {
                float col[G + 2 * RS];
#pragma unroll
                for (int j = 0; j < G + 2 * RS; ++j) {
                    const int r = reflect(s0 - RS + j, ny);
                    col[j] = Bx[(r % GG::capB) * GG::WU + c - cbase];
                }
#pragma unroll
                for (int o = 0; o < G; ++o) {
                    const int s = s0 + o;
                    if (s < s_first || s > s_last) continue;
                    float acc = __fmul_rn(A.ts.t[0], col[o + RS]);
#pragma unroll
                    for (int k = 1; k <= RS; ++k)
                        acc = __fmaf_rn(A.ts.t[k], __fadd_rn(col[o + RS - k], col[o + RS + k]), acc);
                    Us[(s % GG::capS) * GG::WU + c - cbase] = acc;
                }
            }
        }
        __syncthreads();
        // ---- stage 4a: gradient products of rows p0 .. p0+3 over [cp0, cp1)
        const int p0 = s0 - 1;
        {
            const int c = cp0 + tid;
            if (c < cp1) {
                const int cl = reflect(c - 1, nx) - cbase, cr = reflect(c + 1, nx) - cbase;
#pragma unroll
                for (int o = 0; o < G; ++o) {
                    const int p = p0 + o;
                    if (p < p_first || p > p_last) continue;
                    const float *um = Us + (reflect(p - 1, ny) % GG::capS) * GG::WU;
                    const float *u0 = Us + (p % GG::capS) * GG::WU;
                    const float *up = Us + (reflect(p + 1, ny) % GG::capS) * GG::WU;
                    const float gx = __fmul_rn(0.5f, __fsub_rn(u0[cr], u0[cl]));
                    const float gy = __fmul_rn(0.5f, __fsub_rn(up[c - cbase], um[c - cbase]));
                    float *P = Pr + o * 3 * GG::WU + c - cbase;
                    P[0] = __fmul_rn(gx, gx);
                    P[GG::WU] = __fmul_rn(gx, gy);
                    P[2 * GG::WU] = __fmul_rn(gy, gy);
                }
            }
        }
        __syncthreads();
        // ---- stage 4b: T3 = x-blur(rho) of the products, rows p0..p0+3, columns [x0, co1)
        if (tid < G * (SW / 4)) {
            const int g = tid / (SW / 4), q = tid % (SW / 4);
            const int p = p0 + g;
            const int c0 = x0 + 4 * q;
            if (p >= p_first && p <= p_last && c0 < co1) {
                float *dst = T3 + (p % GG::capT) * 3 * SW;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float *P = Pr + (g * 3 + ch) * GG::WU;
                    float v[4 + 2 * RR];
#pragma unroll
                    for (int j = 0; j < 4 + 2 * RR; ++j) v[j] = P[reflect(c0 - RR + j, nx) - cbase];
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        float acc = __fmul_rn(A.tr.t[0], v[o + RR]);
#pragma unroll
                        for (int k = 1; k <= RR; ++k)
                            acc = __fmaf_rn(A.tr.t[k], __fadd_rn(v[o + RR - k], v[o + RR + k]), acc);
                        if (c0 + o < co1) dst[ch * SW + c0 + o - x0] = acc;
                    }
                }
            }
        }
        __syncthreads();
        // ---- stage 5: J rows y0 .. y0+3 (y-blur of T3), D, epilogue
        const int y0 = p0 - RR;
        if (tid < SW && y0 + G - 1 >= ys && y0 < ye) {
            const int c = x0 + tid;
            if (c < co1) {
                float J[3][G];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float col[G + 2 * RR];
#pragma unroll
                    for (int j = 0; j < G + 2 * RR; ++j) {
                        const int r = reflect(y0 - RR + j, ny);
                        col[j] = T3[(r % GG::capT) * 3 * SW + ch * SW + tid];
                    }
#pragma unroll
                    for (int o = 0; o < G; ++o) {
                        float acc = __fmul_rn(A.tr.t[0], col[o + RR]);
#pragma unroll
                        for (int k = 1; k <= RR; ++k)
                            acc = __fmaf_rn(A.tr.t[k], __fadd_rn(col[o + RR - k], col[o + RR + k]), acc);
                        J[ch][o] = acc;
                    }
                }
#pragma unroll
                for (int o = 0; o < G; ++o) {
                    const int y = y0 + o;
                    if (y < ys || y >= ye) continue;
                    float dxx, dxy, dyy;
                    d_from_j(J[0][o], J[1][o], J[2][o], A.alpha, A.C, dxx, dxy, dyy);
                    const int64_t z = (int64_t)y * nx + c;
                    if (MODE == 0) {
                        const int64_t N = (int64_t)nx * ny;
                        A.D[z] = dxx;
                        A.D[N + z] = dxy;
                        A.D[2 * N + z] = dyy;
                    } else {
                        build_point2d_call(dxx, dxy, dyy, z, A.offs, A.wbase, A.wt, A.err);
                    }
                }
            }
        }
        // the barriers of the next group's stages 1-4 order these reads
        // before the ring slots they use are overwritten
    }
}

template <int RS, int RR, int MODE>
adlbr_status launch_stream(const StreamArgs &a, cudaStream_t st) {
    using GG = Geo<RS, RR>;
    const size_t smem = GG::total * sizeof(float);
    auto kern = ced_stream_kernel<RS, RR, MODE>;
    ADLBR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(blocks_for(a.nx, SW), blocks_for(a.ny, SH));
    kern<<<grid, CT, smem, st>>>(a);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

template <int MODE>
bool try_stream(int rs, int rr, const StreamArgs &a, cudaStream_t st, adlbr_status &out) {
    if (rr == 12 && rs == 3) {
        out = launch_stream<3, 12, MODE>(a, st);
        return true;
    }
    if (rr == 12 && rs == 2) {
        out = launch_stream<2, 12, MODE>(a, st);
        return true;
    }
    return false;
}

// =================================================================== fallback
constexpr int TX = 128;  // x pass: outputs per block

// out[c][y][x] = sum_k taps[|k|] in[c][y][reflect(x + k)]
template <int C>
__global__ void __launch_bounds__(TX) blur_x_kernel(int nx, int ny, int64_t N, int r, Taps tp,
                                                    const float *__restrict__ in,
                                                    float *__restrict__ out) {
    extern __shared__ float smx[];  // C * (TX + 2r)
    const int x0 = blockIdx.x * TX, y = blockIdx.y;
    const int W = TX + 2 * r;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *row = in + c * N + (int64_t)y * nx;
        for (int j = threadIdx.x; j < W; j += TX) smx[c * W + j] = row[reflect(x0 - r + j, nx)];
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= nx) return;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *s = smx + c * W + threadIdx.x + r;
        float acc = __fmul_rn(tp.t[0], s[0]);
        for (int k = 1; k <= r; ++k) acc = __fmaf_rn(tp.t[k], __fadd_rn(s[-k], s[k]), acc);
        out[c * N + (int64_t)y * nx + x] = acc;
    }
}

constexpr int BX = 32, BY = 32;  // y pass tile

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
    for (int oy = ty; oy < BY; oy += 8) {
        const int y = y0 + oy;
        if (y >= ny) break;
        float v[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float *s = smy + (c * H + oy + r) * BX + tx;
            float acc = __fmul_rn(tp.t[0], s[0]);
            for (int k = 1; k <= r; ++k) acc = __fmaf_rn(tp.t[k], __fadd_rn(s[-k * BX], s[k * BX]), acc);
            v[c] = acc;
        }
        const int64_t z = (int64_t)y * nx + x;
        if (EPI == 0) {
#pragma unroll
            for (int c = 0; c < C; ++c) out[c * N + z] = v[c];
        } else {
            float dxx, dxy, dyy;
            d_from_j(v[0], v[1], v[2], alpha, Cc, dxx, dxy, dyy);
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

adlbr_status fallback_tensor(int nx, int ny, const float *u, float *D, int rs, int rr, const Taps &ts,
                             const Taps &tr, float alpha, float C, void *scratch, cudaStream_t st) {
    const int64_t N = (int64_t)nx * ny;
    float *A = (float *)scratch;  // 3N
    float *B = A + 3 * N;         // 3N
    dim3 gx(blocks_for(nx, TX), ny), gy(blocks_for(nx, BX), blocks_for(ny, BY));
    blur_x_kernel<1><<<gx, TX, (TX + 2 * rs) * sizeof(float), st>>>(nx, ny, N, rs, ts, u, A);
    blur_y_kernel<1, 0><<<gy, BX * 8, (BY + 2 * rs) * BX * sizeof(float), st>>>(nx, ny, N, rs, ts, A,
                                                                                   B, 0.f, 0.f);
    grad_outer_kernel<<<dim3(blocks_for(nx, 256), ny), 256, 0, st>>>(nx, ny, N, B, A);
    blur_x_kernel<3><<<gx, TX, 3 * (TX + 2 * rr) * sizeof(float), st>>>(nx, ny, N, rr, tr, A, B);
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
    StreamArgs a = {};
    a.nx = nx;
    a.ny = ny;
    a.alpha = (float)alpha;
    a.C = (float)C;
    a.ts = make_taps(sigma);
    a.tr = make_taps(rho);
    a.u = u;
    a.D = D;
    adlbr_status out;
    if (try_stream<0>(radius_of(sigma), radius_of(rho), a, st, out)) return out;
    return fallback_tensor(nx, ny, u, D, radius_of(sigma), radius_of(rho), a.ts, a.tr, a.alpha, a.C,
                           scratch, st);
}

adlbr_status launch_ced_build(adlbr_stencils *s, const float *u, double sigma, double rho,
                              double alpha, double C, void *scratch, float *Dtmp, cudaStream_t st) {
    if (adlbr_status e = check_params(sigma, rho, alpha, C)) return e;
    StreamArgs a = {};
    a.nx = (int)s->n[0];
    a.ny = (int)s->n[1];
    a.alpha = (float)alpha;
    a.C = (float)C;
    a.ts = make_taps(sigma);
    a.tr = make_taps(rho);
    a.u = u;
    a.offs = (short4 *)s->offs;
    a.wbase = s->w;
    a.wt = s->w_t;
    a.err = s->err;
    adlbr_status out;
    if (try_stream<1>(radius_of(sigma), radius_of(rho), a, st, out)) return out;
    if (adlbr_status e = fallback_tensor(a.nx, a.ny, u, Dtmp, radius_of(sigma), radius_of(rho), a.ts,
                                         a.tr, a.alpha, a.C, scratch, st))
        return e;
    return launch_build2d(s, Dtmp, ADLBR_F32, st);
}

}  // namespace adlbr

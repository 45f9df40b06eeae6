// The learned preconditioner's network: a 3-level U-Net (not in the paper),
// forward and backward passes and an Adam step, FP32.
//
//   enc1: conv3x3(Cin->c1) ReLU, conv3x3(c1->c1) ReLU           -> s1 (H x W)
//   avgpool 2x2
//   enc2: conv3x3(c1->c2) ReLU, conv3x3(c2->c2) ReLU            -> s2 (H/2)
//   avgpool 2x2
//   mid : conv3x3(c2->c3) ReLU, conv3x3(c3->c3) ReLU                  (H/4)
//   nearest upsample x2, concat [up, s2]
//   dec2: conv3x3(c3+c2->c2) ReLU, conv3x3(c2->c2) ReLU               (H/2)
//   nearest upsample x2, concat [up, s1]
//   dec1: conv3x3(c2+c1->c1) ReLU, conv3x3(c1->c1) ReLU               (H)
//   out : conv1x1(c1->1)
// Convolutions are cross-correlations with zero padding.  Parameters are one
// flat FP32 vector: per layer, in the order above, weights [co][ci][ky][kx]
// then bias [co].  Tensors are [batch][channel][H][W].
//
// Kernels: direct 3x3 convolution (a CTA computes a 32 x 8 pixel tile for 16
// output channels, staging 8 input channels plus halo and their weights in
// shared memory per step); the data gradient is the same convolution with the
// weights transposed and flipped; the weight gradient is a per-CTA reduction
// over a pixel range with one FP32 atomic per weight per CTA.
#include <cmath>
#include <new>
#include <vector>

#include "internal.cuh"

struct adlbr_unet {
    int cin, c1, c2, c3, B, H, W;
    int device;
    // activations (post-ReLU) and work buffers, one allocation
    float *mem;
    size_t mem_floats;
    float *x, *a1a, *s1, *p1, *a2a, *s2, *p2, *a3a, *a3b, *cat2, *d2a, *d2b, *cat1, *d1a, *d1b;
    float *g0, *g1, *gcat;  // gradient work buffers (largest activation size)
    float *wt;              // transposed / flipped weights for the data gradient
    int64_t n_params;
    // inference on the tensor cores (unet_tc.cu): BF16 packed weights per
    // layer and BF16 channels-last activations (one allocation)
    int tensor_cores;
    int fwd_tc;             // the last forward ran on the tensor cores
    __nv_bfloat16 *wpack;
    size_t wpack_off[10];
    __nv_bfloat16 *hmem;
    __nv_bfloat16 *hx, *h1a, *h1b, *hp1, *h2a, *h2b, *hp2, *h3a, *h3b, *hu3, *hd2a, *hd2b, *hu2, *hd1a, *hd1b;
};

namespace adlbr {

namespace {

struct Layer {
    int co, ci, k;
    int64_t w_off, b_off;
};

void layer_table(const adlbr_unet *n, Layer (&L)[11]) {
    const int sh[11][3] = {{n->c1, n->cin, 3}, {n->c1, n->c1, 3}, {n->c2, n->c1, 3},
                           {n->c2, n->c2, 3},  {n->c3, n->c2, 3}, {n->c3, n->c3, 3},
                           {n->c2, n->c3 + n->c2, 3}, {n->c2, n->c2, 3},
                           {n->c1, n->c2 + n->c1, 3}, {n->c1, n->c1, 3}, {1, n->c1, 1}};
    int64_t o = 0;
    for (int l = 0; l < 11; ++l) {
        L[l].co = sh[l][0];
        L[l].ci = sh[l][1];
        L[l].k = sh[l][2];
        L[l].w_off = o;
        o += (int64_t)L[l].co * L[l].ci * L[l].k * L[l].k;
        L[l].b_off = o;
        o += L[l].co;
    }
}

// ---------------------------------------------------------------- conv3x3 fwd
constexpr int CTW = 32, CTH = 8, COB = 16, CIB = 8;

// y[b][co][p] = (bias[co]) + sum_ci sum_taps W[co][ci][ky][kx] x[b][ci][p + (ky-1, kx-1)]
template <bool RELU, bool BIAS>
__global__ void __launch_bounds__(CTW *CTH) conv3x3_kernel(int B, int Ci, int Co, int H, int W,
                                                           const float *__restrict__ x,
                                                           const float *__restrict__ w,
                                                           const float *__restrict__ bias,
                                                           float *__restrict__ y) {
    __shared__ float xs[CIB][CTH + 2][CTW + 2];
    __shared__ float ws[COB][CIB][9];
    const int nco = (Co + COB - 1) / COB;
    const int b = blockIdx.z / nco, co0 = (blockIdx.z % nco) * COB;
    const int tx = threadIdx.x % CTW, ty = threadIdx.x / CTW;
    const int px = blockIdx.x * CTW + tx, py = blockIdx.y * CTH + ty;
    float acc[COB];
#pragma unroll
    for (int o = 0; o < COB; ++o) acc[o] = (BIAS && co0 + o < Co) ? bias[co0 + o] : 0.f;
    const float *xb = x + (int64_t)b * Ci * H * W;
    for (int c0 = 0; c0 < Ci; c0 += CIB) {
        // stage CIB input channels with a 1-pixel halo
        for (int i = threadIdx.x; i < CIB * (CTH + 2) * (CTW + 2); i += CTW * CTH) {
            const int cc = i / ((CTH + 2) * (CTW + 2));
            const int rem = i % ((CTH + 2) * (CTW + 2));
            const int yy = rem / (CTW + 2), xx = rem % (CTW + 2);
            const int gy = blockIdx.y * CTH + yy - 1, gx = blockIdx.x * CTW + xx - 1;
            float v = 0.f;
            if (c0 + cc < Ci && gy >= 0 && gy < H && gx >= 0 && gx < W)
                v = xb[((int64_t)(c0 + cc) * H + gy) * W + gx];
            xs[cc][yy][xx] = v;
        }
        for (int i = threadIdx.x; i < COB * CIB * 9; i += CTW * CTH) {
            const int o = i / (CIB * 9), rem = i % (CIB * 9), cc = rem / 9, t = rem % 9;
            float v = 0.f;
            if (co0 + o < Co && c0 + cc < Ci) v = w[((int64_t)(co0 + o) * Ci + c0 + cc) * 9 + t];
            ws[o][cc][t] = v;
        }
        __syncthreads();
#pragma unroll 2
        for (int cc = 0; cc < CIB; ++cc) {
            float in[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) in[t] = xs[cc][ty + t / 3][tx + t % 3];
#pragma unroll
            for (int o = 0; o < COB; ++o)
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[o] = fmaf(ws[o][cc][t], in[t], acc[o]);
        }
        __syncthreads();
    }
    if (px >= W || py >= H) return;
#pragma unroll
    for (int o = 0; o < COB; ++o) {
        if (co0 + o >= Co) break;
        float v = acc[o];
        if (RELU) v = fmaxf(v, 0.f);
        y[(((int64_t)b * Co + co0 + o) * H + py) * W + px] = v;
    }
}

// 1x1 convolution to one output channel (the output layer)
__global__ void conv1x1_out_kernel(int B, int Ci, int HW, const float *__restrict__ x,
                                   const float *__restrict__ w, const float *__restrict__ bias,
                                   float *__restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * HW) return;
    const int b = (int)(i / HW);
    const int64_t p = i % HW;
    float acc = bias[0];
    for (int c = 0; c < Ci; ++c) acc = fmaf(w[c], x[((int64_t)b * Ci + c) * HW + p], acc);
    y[i] = acc;
}

// ---------------------------------------------------------------- reshaping
// y[b][c][h][w] = mean of the 2x2 block of x (x is 2H x 2W)
__global__ void pool2_kernel(int64_t n, int H, int W, const float *__restrict__ x, float *__restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int w = (int)(i % W);
    const int64_t r = i / W;
    const int h = (int)(r % H);
    const int64_t bc = r / H;
    const float *s = x + (bc * (2 * H) + 2 * h) * (2 * W) + 2 * w;
    y[i] = 0.25f * (s[0] + s[1] + s[2 * W] + s[2 * W + 1]);
}
// gx (2H x 2W) = 1/4 of gy broadcast over each block (+= when ACC)
template <bool ACC>
__global__ void pool2_bwd_kernel(int64_t n2, int H, int W, const float *__restrict__ gy,
                                 float *__restrict__ gx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // index into gx
    if (i >= n2) return;
    const int w2 = (int)(i % (2 * W));
    const int64_t r = i / (2 * W);
    const int h2 = (int)(r % (2 * H));
    const int64_t bc = r / (2 * H);
    const float v = 0.25f * gy[(bc * H + h2 / 2) * W + w2 / 2];
    gx[i] = ACC ? gx[i] + v : v;
}

// dst[b][c0 + c][2h + dy][2w + dx] = src[b][c][h][w]  (nearest upsample into a channel slice)
__global__ void up2_into_kernel(int B, int C, int H, int W, int Cdst, int c0,
                                const float *__restrict__ src, float *__restrict__ dst) {
    int64_t n = (int64_t)B * C * 4 * H * W;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int w2 = (int)(i % (2 * W));
    int64_t r = i / (2 * W);
    const int h2 = (int)(r % (2 * H));
    r /= (2 * H);
    const int c = (int)(r % C);
    const int b = (int)(r / C);
    dst[(((int64_t)b * Cdst + c0 + c) * 2 * H + h2) * 2 * W + w2] =
        src[(((int64_t)b * C + c) * H + h2 / 2) * W + w2 / 2];
}
// gsrc[b][c][h][w] = sum over the 2x2 block of gdst's channel slice
__global__ void up2_bwd_kernel(int B, int C, int H, int W, int Cdst, int c0,
                               const float *__restrict__ gdst, float *__restrict__ gsrc) {
    int64_t n = (int64_t)B * C * H * W;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int w = (int)(i % W);
    int64_t r = i / W;
    const int h = (int)(r % H);
    r /= H;
    const int c = (int)(r % C);
    const int b = (int)(r / C);
    const float *s = gdst + (((int64_t)b * Cdst + c0 + c) * 2 * H + 2 * h) * 2 * W + 2 * w;
    gsrc[i] = s[0] + s[1] + s[2 * W] + s[2 * W + 1];
}
// copy a [B][C][HW] tensor into / out of a channel slice of a [B][Cdst][HW] tensor
template <bool INTO, bool ACC>
__global__ void slice_kernel(int B, int C, int64_t HW, int Cdst, int c0, float *__restrict__ a,
                             float *__restrict__ big) {
    int64_t n = (int64_t)B * C * HW;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = i % HW;
    const int64_t r = i / HW;
    const int c = (int)(r % C), b = (int)(r / C);
    float *bp = big + ((int64_t)b * Cdst + c0 + c) * HW + p;
    if (INTO)
        *bp = a[i];
    else
        a[i] = ACC ? a[i] + *bp : *bp;
}

// g *= (a > 0)   (ReLU backward through the stored post-activation)
__global__ void relu_bwd_kernel(int64_t n, const float *__restrict__ a, float *__restrict__ g) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(a[i] > 0.f)) g[i] = 0.f;
}

// wt[ci][co][8 - t] = w[co][ci][t]
__global__ void transpose_flip_kernel(int Co, int Ci, const float *__restrict__ w, float *__restrict__ wt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)Co * Ci * 9) return;
    const int t = (int)(i % 9);
    const int64_t r = i / 9;
    const int ci = (int)(r % Ci), co = (int)(r / Ci);
    wt[((int64_t)ci * Co + co) * 9 + (8 - t)] = w[i];
}

// weight and bias gradients of a 3x3 layer:
// gw[co][ci][t] += sum_{b,p} gy[b][co][p] x[b][ci][p + d(t)],  gb[co] += sum gy[b][co][p]
constexpr int WG_THREADS = 256, WG_CI = 8;
__global__ void __launch_bounds__(WG_THREADS) conv3x3_wgrad_kernel(int B, int Ci, int Co, int H, int W,
                                                                   int64_t pix_per_cta,
                                                                   const float *__restrict__ x,
                                                                   const float *__restrict__ gy,
                                                                   float *__restrict__ gw,
                                                                   float *__restrict__ gb) {
    const int co = blockIdx.x, ci0 = blockIdx.y * WG_CI;
    const int64_t P = (int64_t)B * H * W;
    const int64_t p0 = (int64_t)blockIdx.z * pix_per_cta, p1 = min(P, p0 + pix_per_cta);
    float acc[WG_CI][9];
    float accb = 0.f;
#pragma unroll
    for (int c = 0; c < WG_CI; ++c)
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[c][t] = 0.f;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += WG_THREADS) {
        const int b = (int)(p / ((int64_t)H * W));
        const int rem = (int)(p % ((int64_t)H * W));
        const int py = rem / W, px = rem % W;
        const float g = gy[((int64_t)b * Co + co) * H * W + rem];
        accb += g;
#pragma unroll
        for (int c = 0; c < WG_CI; ++c) {
            if (ci0 + c >= Ci) break;
            const float *xc = x + ((int64_t)b * Ci + ci0 + c) * H * W;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int yy = py + t / 3 - 1, xx = px + t % 3 - 1;
                const float v = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? xc[yy * W + xx] : 0.f;
                acc[c][t] = fmaf(g, v, acc[c][t]);
            }
        }
    }
    // block reduction of the WG_CI * 9 + 1 sums
    __shared__ float red[WG_THREADS / 32][WG_CI * 9 + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < WG_CI; ++c)
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            float v = acc[c][t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[wid][c * 9 + t] = v;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) accb += __shfl_down_sync(0xffffffffu, accb, o);
    if (lane == 0) red[wid][WG_CI * 9] = accb;
    __syncthreads();
    for (int k = threadIdx.x; k < WG_CI * 9 + 1; k += WG_THREADS) {
        float s = 0.f;
        for (int q = 0; q < WG_THREADS / 32; ++q) s += red[q][k];
        if (k < WG_CI * 9) {
            const int c = k / 9, t = k % 9;
            if (ci0 + c < Ci) atomicAdd(gw + ((int64_t)co * Ci + ci0 + c) * 9 + t, s);
        } else if (blockIdx.y == 0) {
            atomicAdd(gb + co, s);
        }
    }
}

// output layer (1x1, one channel): gw[c] = sum gy x[c], gb = sum gy, gx[c] = w[c] gy
__global__ void conv1x1_out_bwd_kernel(int B, int Ci, int HW, const float *__restrict__ x,
                                       const float *__restrict__ w, const float *__restrict__ gy,
                                       float *__restrict__ gw, float *__restrict__ gb,
                                       float *__restrict__ gx) {
    const int64_t n = (int64_t)B * HW;
    float acc[64];
    const int C = min(Ci, 64);
    for (int c = 0; c < C; ++c) acc[c] = 0.f;
    float accb = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / HW);
        const int64_t p = i % HW;
        const float g = gy[i];
        accb += g;
        for (int c = 0; c < C; ++c) {
            const int64_t xi = ((int64_t)b * Ci + c) * HW + p;
            acc[c] = fmaf(g, x[xi], acc[c]);
            gx[xi] = w[c] * g;
        }
    }
    for (int c = 0; c < C; ++c) {
        float v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(gw + c, v);
    }
    for (int o = 16; o > 0; o >>= 1) accb += __shfl_down_sync(0xffffffffu, accb, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(gb, accb);
}

__global__ void adam_kernel(int64_t n, float *__restrict__ th, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

adlbr_status conv3x3(const adlbr_unet *n, int Ci, int Co, int H, int W, const float *x, const float *w,
                     const float *bias, float *y, bool relu, cudaStream_t st) {
    dim3 grid((W + CTW - 1) / CTW, (H + CTH - 1) / CTH, n->B * ((Co + COB - 1) / COB));
    if (relu)
        conv3x3_kernel<true, true><<<grid, CTW * CTH, 0, st>>>(n->B, Ci, Co, H, W, x, w, bias, y);
    else if (bias)
        conv3x3_kernel<false, true><<<grid, CTW * CTH, 0, st>>>(n->B, Ci, Co, H, W, x, w, bias, y);
    else
        conv3x3_kernel<false, false><<<grid, CTW * CTH, 0, st>>>(n->B, Ci, Co, H, W, x, w, bias, y);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

// backward of y = relu(conv3x3(x)) given gy (modified in place by the ReLU
// mask): gw, gb accumulate; gx = conv3x3^T(gy) (written, not accumulated)
adlbr_status conv3x3_bwd(const adlbr_unet *n, const Layer &L, int H, int W, const float *x,
                         const float *y, float *gy, const float *params, float *gparams, float *gx,
                         float *wt, cudaStream_t st) {
    const int64_t ny = (int64_t)n->B * L.co * H * W;
    relu_bwd_kernel<<<nb(ny), 256, 0, st>>>(ny, y, gy);
    const int64_t P = (int64_t)n->B * H * W;
    const int64_t ppc = 4096;
    dim3 g((unsigned)L.co, (unsigned)((L.ci + WG_CI - 1) / WG_CI), (unsigned)((P + ppc - 1) / ppc));
    conv3x3_wgrad_kernel<<<g, WG_THREADS, 0, st>>>(n->B, L.ci, L.co, H, W, ppc, x, gy,
                                                   gparams + L.w_off, gparams + L.b_off);
    if (gx) {
        transpose_flip_kernel<<<nb((int64_t)L.co * L.ci * 9), 256, 0, st>>>(L.co, L.ci, params + L.w_off, wt);
        if (adlbr_status e = conv3x3(n, L.co, L.ci, H, W, gy, wt, nullptr, gx, false, st)) return e;
    }
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace

namespace {

// The tensor-core forward from the BF16 channels-last input n->hx.
// The BF16 operand copies of the ten 3x3 layers' weights (n->wpack).
adlbr_status tc_pack(adlbr_unet *n, const float *params, cudaStream_t st) {
    Layer L[11];
    layer_table(n, L);
    ConvPackTable T;
    T.n = 10;
    for (int l = 0; l < 10; ++l) {
        T.co[l] = L[l].co;
        T.ci[l] = L[l].ci;
        T.w_off[l] = L[l].w_off;
        T.out_off[l] = (int64_t)n->wpack_off[l];
    }
    return conv_tc_pack(T, params, n->wpack, st);
}

// The tensor-core forward from the BF16 channels-last input n->hx and the
// packed weights n->wpack (packed here when `pack`).
adlbr_status tc_forward(adlbr_unet *n, const float *params, float *yout, bool pack, cudaStream_t st) {
    Layer L[11];
    layer_table(n, L);
    const int H = n->H, W = n->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int B = n->B;
    {
        if (pack)
            if (adlbr_status e = tc_pack(n, params, st)) return e;
        n->fwd_tc = 1;
        const int c1 = n->c1, c2 = n->c2, c3 = n->c3, cp = (n->cin + 15) / 16 * 16;
        auto cv = [&](int l, int h, int w, const __nv_bfloat16 *x0, int C0, const __nv_bfloat16 *x1, int C1,
                      __nv_bfloat16 *y) {
            return conv_tc(B, h, w, x0, C0, x1, C1, L[l].co, n->wpack + n->wpack_off[l], params + L[l].b_off, y,
                           st);
        };
        if (adlbr_status e = cv(0, H, W, n->hx, cp, nullptr, 0, n->h1a)) return e;
        if (adlbr_status e = cv(1, H, W, n->h1a, c1, nullptr, 0, n->h1b)) return e;
        if (adlbr_status e = tc_pool(B, H2, W2, c1, n->h1b, n->hp1, st)) return e;
        if (adlbr_status e = cv(2, H2, W2, n->hp1, c1, nullptr, 0, n->h2a)) return e;
        if (adlbr_status e = cv(3, H2, W2, n->h2a, c2, nullptr, 0, n->h2b)) return e;
        if (adlbr_status e = tc_pool(B, H4, W4, c2, n->h2b, n->hp2, st)) return e;
        if (adlbr_status e = cv(4, H4, W4, n->hp2, c2, nullptr, 0, n->h3a)) return e;
        if (adlbr_status e = cv(5, H4, W4, n->h3a, c3, nullptr, 0, n->h3b)) return e;
        // [up(a3b), s2] and [up(d2b), s1]: the convolutions read both parts
        if (adlbr_status e = tc_up(B, H4, W4, c3, n->h3b, n->hu3, st)) return e;
        if (adlbr_status e = cv(6, H2, W2, n->hu3, c3, n->h2b, c2, n->hd2a)) return e;
        if (adlbr_status e = cv(7, H2, W2, n->hd2a, c2, nullptr, 0, n->hd2b)) return e;
        if (adlbr_status e = tc_up(B, H2, W2, c2, n->hd2b, n->hu2, st)) return e;
        if (adlbr_status e = cv(8, H, W, n->hu2, c2, n->h1b, c1, n->hd1a)) return e;
        if (adlbr_status e = cv(9, H, W, n->hd1a, c1, nullptr, 0, n->hd1b)) return e;
        if (adlbr_status e = tc_out1x1((int64_t)B * H * W, c1, n->hd1b, params + L[10].w_off, params + L[10].b_off,
                                       yout, st))
            return e;
        ADLBR_CUDA(cudaGetLastError());
        return ADLBR_OK;
    }
}

}  // namespace

__nv_bfloat16 *unet_tc_input(adlbr_unet *n, int *cp) {
    if (!n->tensor_cores) return nullptr;
    *cp = (n->cin + 15) / 16 * 16;
    return n->hx;
}

adlbr_status unet_tc_prepare(adlbr_unet *n, const float *params, cudaStream_t st) {
    if (!n->tensor_cores) return fail(ADLBR_E_ARG, "the packed weights need the tensor-core forward");
    return tc_pack(n, params, st);
}

adlbr_status unet_forward_from_input(adlbr_unet *n, const float *params, float *yout, cudaStream_t st) {
    if (!n->tensor_cores) return fail(ADLBR_E_ARG, "the network's input buffer needs the tensor-core forward");
    return tc_forward(n, params, yout, false, st);
}

adlbr_status unet_forward(adlbr_unet *n, const float *params, const float *xin, float *yout,
                          cudaStream_t st) {
    Layer L[11];
    layer_table(n, L);
    const int H = n->H, W = n->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int B = n->B;
    if (n->tensor_cores) {
        const int cp = (n->cin + 15) / 16 * 16;
        if (adlbr_status e = tc_to_nhwc(B, n->cin, cp, (int64_t)H * W, xin, n->hx, st)) return e;
        return tc_forward(n, params, yout, true, st);
    }
    n->fwd_tc = 0;
    auto cr = [&](int l, int h, int w, const float *x, float *y) {
        return conv3x3(n, L[l].ci, L[l].co, h, w, x, params + L[l].w_off, params + L[l].b_off, y, true, st);
    };
    if (adlbr_status e = cr(0, H, W, xin, n->a1a)) return e;
    if (adlbr_status e = cr(1, H, W, n->a1a, n->s1)) return e;
    int64_t m = (int64_t)B * n->c1 * H2 * W2;
    pool2_kernel<<<nb(m), 256, 0, st>>>(m, H2, W2, n->s1, n->p1);
    if (adlbr_status e = cr(2, H2, W2, n->p1, n->a2a)) return e;
    if (adlbr_status e = cr(3, H2, W2, n->a2a, n->s2)) return e;
    m = (int64_t)B * n->c2 * H4 * W4;
    pool2_kernel<<<nb(m), 256, 0, st>>>(m, H4, W4, n->s2, n->p2);
    if (adlbr_status e = cr(4, H4, W4, n->p2, n->a3a)) return e;
    if (adlbr_status e = cr(5, H4, W4, n->a3a, n->a3b)) return e;
    // cat2 = [up(a3b), s2]
    const int C2 = n->c3 + n->c2;
    up2_into_kernel<<<nb((int64_t)B * n->c3 * H2 * W2), 256, 0, st>>>(B, n->c3, H4, W4, C2, 0, n->a3b, n->cat2);
    slice_kernel<true, false><<<nb((int64_t)B * n->c2 * H2 * W2), 256, 0, st>>>(
        B, n->c2, (int64_t)H2 * W2, C2, n->c3, n->s2, n->cat2);
    if (adlbr_status e = cr(6, H2, W2, n->cat2, n->d2a)) return e;
    if (adlbr_status e = cr(7, H2, W2, n->d2a, n->d2b)) return e;
    const int C1 = n->c2 + n->c1;
    up2_into_kernel<<<nb((int64_t)B * n->c2 * H * W), 256, 0, st>>>(B, n->c2, H2, W2, C1, 0, n->d2b, n->cat1);
    slice_kernel<true, false><<<nb((int64_t)B * n->c1 * H * W), 256, 0, st>>>(
        B, n->c1, (int64_t)H * W, C1, n->c2, n->s1, n->cat1);
    if (adlbr_status e = cr(8, H, W, n->cat1, n->d1a)) return e;
    if (adlbr_status e = cr(9, H, W, n->d1a, n->d1b)) return e;
    conv1x1_out_kernel<<<nb((int64_t)B * H * W), 256, 0, st>>>(B, n->c1, H * W, n->d1b,
                                                               params + L[10].w_off, params + L[10].b_off,
                                                               yout);
    ADLBR_CUDA(cudaGetLastError());
    if (n->x != xin) n->x = const_cast<float *>(xin);
    return ADLBR_OK;
}

// gradient of <gy, forward(params, x)>: gparams (overwritten), gx (optional)
adlbr_status unet_backward(adlbr_unet *n, const float *params, const float *gy, float *gparams,
                           float *gx, cudaStream_t st) {
    Layer L[11];
    layer_table(n, L);
    const int H = n->H, W = n->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int B = n->B;
    ADLBR_CUDA(cudaMemsetAsync(gparams, 0, n->n_params * sizeof(float), st));
    float *g0 = n->g0, *g1 = n->g1, *gc = n->gcat;
    // output layer: g0 = d/d d1b
    {
        const int64_t HW = (int64_t)H * W;
        int blocks = (int)std::min<int64_t>(nb((int64_t)B * HW), vec_blocks());
        conv1x1_out_bwd_kernel<<<blocks, 256, 0, st>>>(B, n->c1, (int)HW, n->d1b, params + L[10].w_off, gy,
                                                      gparams + L[10].w_off, gparams + L[10].b_off, g0);
    }
    // dec1b: input d1a, output d1b ; grad into g1 (d/d d1a)
    if (adlbr_status e = conv3x3_bwd(n, L[9], H, W, n->d1a, n->d1b, g0, params, gparams, g1, n->wt, st)) return e;
    // dec1a: input cat1 -> gcat (d/d cat1)
    if (adlbr_status e = conv3x3_bwd(n, L[8], H, W, n->cat1, n->d1a, g1, params, gparams, gc, n->wt, st)) return e;
    const int C1 = n->c2 + n->c1;
    // s1 gradient part (channels c2..) -> g1 ; up part -> g0 (d/d d2b at H2)
    slice_kernel<false, false><<<nb((int64_t)B * n->c1 * H * W), 256, 0, st>>>(
        B, n->c1, (int64_t)H * W, C1, n->c2, g1, gc);
    float *g_s1 = g1;  // keep: gradient w.r.t. s1 from the skip
    up2_bwd_kernel<<<nb((int64_t)B * n->c2 * H2 * W2), 256, 0, st>>>(B, n->c2, H2, W2, C1, 0, gc, g0);
    // dec2b (input d2a, output d2b): g0 -> gc (d/d d2a)
    if (adlbr_status e = conv3x3_bwd(n, L[7], H2, W2, n->d2a, n->d2b, g0, params, gparams, gc, n->wt, st)) return e;
    // dec2a (input cat2): gc -> g0 (d/d cat2)
    if (adlbr_status e = conv3x3_bwd(n, L[6], H2, W2, n->cat2, n->d2a, gc, params, gparams, g0, n->wt, st)) return e;
    const int C2 = n->c3 + n->c2;
    // s2 skip gradient -> gc ; up part -> (d/d a3b) into a spare region after g_s1? use n->wt? no:
    // g_s2 is kept in gc, the up part goes into the tail of g0's buffer is unsafe, so reuse:
    slice_kernel<false, false><<<nb((int64_t)B * n->c2 * H2 * W2), 256, 0, st>>>(
        B, n->c2, (int64_t)H2 * W2, C2, n->c3, gc, g0);
    float *g_s2 = gc;
    // d/d a3b (H4): written to the buffer g_a3 (after g_s2 inside gcat)
    float *g_a3 = gc + (int64_t)B * n->c2 * H2 * W2;
    up2_bwd_kernel<<<nb((int64_t)B * n->c3 * H4 * W4), 256, 0, st>>>(B, n->c3, H4, W4, C2, 0, g0, g_a3);
    // mid_b (input a3a, output a3b): g_a3 -> g0 (d/d a3a)
    if (adlbr_status e = conv3x3_bwd(n, L[5], H4, W4, n->a3a, n->a3b, g_a3, params, gparams, g0, n->wt, st)) return e;
    // mid_a (input p2, output a3a): g0 -> g_a3 (d/d p2)
    if (adlbr_status e = conv3x3_bwd(n, L[4], H4, W4, n->p2, n->a3a, g0, params, gparams, g_a3, n->wt, st)) return e;
    // pool2 backward, add to the skip gradient of s2
    pool2_bwd_kernel<true><<<nb((int64_t)B * n->c2 * H2 * W2), 256, 0, st>>>((int64_t)B * n->c2 * H2 * W2,
                                                                           H4, W4, g_a3, g_s2);
    // enc2b (input a2a, output s2): g_s2 -> g0 (d/d a2a)
    if (adlbr_status e = conv3x3_bwd(n, L[3], H2, W2, n->a2a, n->s2, g_s2, params, gparams, g0, n->wt, st)) return e;
    // enc2a (input p1, output a2a): g0 -> gc (d/d p1)
    if (adlbr_status e = conv3x3_bwd(n, L[2], H2, W2, n->p1, n->a2a, g0, params, gparams, gc, n->wt, st)) return e;
    pool2_bwd_kernel<true><<<nb((int64_t)B * n->c1 * H * W), 256, 0, st>>>((int64_t)B * n->c1 * H * W, H2, W2,
                                                                        gc, g_s1);
    // enc1b (input a1a, output s1): g_s1 -> g0 (d/d a1a)
    if (adlbr_status e = conv3x3_bwd(n, L[1], H, W, n->a1a, n->s1, g_s1, params, gparams, g0, n->wt, st)) return e;
    // enc1a (input x, output a1a): g0 -> gx
    if (adlbr_status e = conv3x3_bwd(n, L[0], H, W, n->x, n->a1a, g0, params, gparams, gx, n->wt, st)) return e;
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status unet_adam(float *params, const float *grads, float *m, float *v, int64_t n, double lr,
                       double b1, double b2, double eps, int t, cudaStream_t st) {
    const float c1 = (float)(1.0 - std::pow(b1, t)), c2 = (float)(1.0 - std::pow(b2, t));
    adam_kernel<<<nb(n), 256, 0, st>>>(n, params, grads, m, v, (float)lr, (float)b1, (float)b2, (float)eps,
                                       c1, c2);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status unet_create(int cin, int c1, int c2, int c3, int B, int H, int W, adlbr_unet **out) {
    if (!out) return fail(ADLBR_E_ARG, "null output");
    if (cin < 1 || c1 < 1 || c2 < 1 || c3 < 1 || B < 1 || H < 4 || W < 4 || H % 4 || W % 4 || c1 > 64)
        return fail(ADLBR_E_SHAPE, "bad U-Net shape (H, W multiples of 4; c1 <= 64)");
    adlbr_unet *n = new (std::nothrow) adlbr_unet();
    if (!n) return fail(ADLBR_E_INTERNAL, "out of host memory");
    n->cin = cin;
    n->c1 = c1;
    n->c2 = c2;
    n->c3 = c3;
    n->B = B;
    n->H = H;
    n->W = W;
    cudaGetDevice(&n->device);
    Layer L[11];
    layer_table(n, L);
    n->n_params = L[10].b_off + 1;
    const int64_t F = (int64_t)H * W, F2 = F / 4, F4 = F / 16;
    std::vector<int64_t> sizes = {
        B * c1 * F,            B * c1 * F, B * c1 * F2, B * c2 * F2, B * c2 * F2, B * c2 * F4,
        B * c3 * F4,           B * c3 * F4, B * (c3 + c2) * F2, B * c2 * F2, B * c2 * F2,
        B * (c2 + c1) * F,     B * c1 * F, B * c1 * F};
    int64_t gmax = 0;
    for (int64_t s : sizes) gmax = std::max(gmax, s);
    gmax = std::max(gmax, (int64_t)B * cin * F);
    int64_t wmax = 0;
    for (auto &l : L) wmax = std::max<int64_t>(wmax, (int64_t)l.co * l.ci * 9);
    int64_t total = 0;
    for (int64_t s : sizes) total += s;
    total += 3 * gmax + gmax + wmax;  // g0, g1, gcat (+ room for the a3 gradient), wt
    n->mem_floats = (size_t)total;
    cudaError_t e = cudaMalloc(&n->mem, n->mem_floats * sizeof(float));
    if (e != cudaSuccess) {
        delete n;
        return cuda_fail(e, "allocating U-Net buffers");
    }
    float *p = n->mem;
    float **slots[] = {&n->a1a, &n->s1, &n->p1, &n->a2a, &n->s2, &n->p2, &n->a3a,
                       &n->a3b, &n->cat2, &n->d2a, &n->d2b, &n->cat1, &n->d1a, &n->d1b};
    for (size_t k = 0; k < sizes.size(); ++k) {
        *slots[k] = p;
        p += sizes[k];
    }
    n->g0 = p;
    p += gmax;
    n->g1 = p;
    p += gmax;
    n->gcat = p;
    p += 2 * gmax;
    n->wt = p;
    n->x = nullptr;
    *out = n;
    return ADLBR_OK;
}

// Forward convolutions on the tensor cores (BF16 operands, FP32 accumulation)
// or back on the FP32 SIMT kernels.  The backward pass always uses FP32.
adlbr_status unet_set_tensor_cores(adlbr_unet *n, int on) {
    if (!n) return fail(ADLBR_E_ARG, "null network");
    if (!on) {
        n->tensor_cores = 0;
        return ADLBR_OK;
    }
    Layer L[11];
    layer_table(n, L);
    size_t total = 0;
    for (int l = 0; l < 10; ++l) {
        if (!conv_tc_supported(L[l].co, L[l].ci))
            return fail(ADLBR_E_SHAPE, "layer %d (%d -> %d channels) has no tensor-core form", l, L[l].ci, L[l].co);
        n->wpack_off[l] = total;
        total += (conv_tc_pack_elems(L[l].co, L[l].ci) + 63) / 64 * 64;
    }
    if (!n->wpack) ADLBR_CUDA(cudaMalloc(&n->wpack, total * sizeof(__nv_bfloat16)));
    if (!n->hmem) {
        // BF16 channels-last activations of the tensor-core forward
        const int64_t B = n->B, P1 = (int64_t)n->H * n->W, P2 = P1 / 4, P4 = P1 / 16;
        const int64_t cp = (n->cin + 15) / 16 * 16;
        const int64_t sizes[15] = {B * P1 * cp,     B * P1 * n->c1, B * P1 * n->c1, B * P2 * n->c1, B * P2 * n->c2,
                                   B * P2 * n->c2,  B * P4 * n->c2, B * P4 * n->c3, B * P4 * n->c3, B * P2 * n->c3,
                                   B * P2 * n->c2,  B * P2 * n->c2, B * P1 * n->c2, B * P1 * n->c1, B * P1 * n->c1};
        int64_t tot = 0;
        for (int64_t v : sizes) tot += (v + 63) / 64 * 64;
        ADLBR_CUDA(cudaMalloc(&n->hmem, tot * sizeof(__nv_bfloat16)));
        __nv_bfloat16 **dst[15] = {&n->hx,  &n->h1a, &n->h1b,  &n->hp1,  &n->h2a, &n->h2b,  &n->hp2, &n->h3a,
                                   &n->h3b, &n->hu3, &n->hd2a, &n->hd2b, &n->hu2, &n->hd1a, &n->hd1b};
        __nv_bfloat16 *q = n->hmem;
        for (int k = 0; k < 15; ++k) {
            *dst[k] = q;
            q += (sizes[k] + 63) / 64 * 64;
        }
    }
    n->tensor_cores = 1;
    return ADLBR_OK;
}

adlbr_status unet_destroy(adlbr_unet *n) {
    if (!n) return ADLBR_OK;
    if (n->mem) cudaFree(n->mem);
    if (n->wpack) cudaFree(n->wpack);
    if (n->hmem) cudaFree(n->hmem);
    delete n;
    return ADLBR_OK;
}

int64_t unet_num_params(const adlbr_unet *n) { return n ? n->n_params : 0; }

void unet_shape(const adlbr_unet *n, int *cin, int *B, int *H, int *W) {
    *cin = n->cin;
    *B = n->B;
    *H = n->H;
    *W = n->W;
}

}  // namespace adlbr

using namespace adlbr;

extern "C" {

adlbr_status adlbr_unet_create(int cin, int c1, int c2, int c3, int batch, int H, int W,
                               adlbr_unet **out) {
    return unet_create(cin, c1, c2, c3, batch, H, W, out);
}

adlbr_status adlbr_unet_destroy(adlbr_unet *n) { return unet_destroy(n); }

adlbr_status adlbr_unet_set_tensor_cores(adlbr_unet *n, int on) { return unet_set_tensor_cores(n, on); }

int64_t adlbr_unet_num_params(const adlbr_unet *n) { return unet_num_params(n); }

adlbr_status adlbr_unet_forward(adlbr_unet *n, const float *params, const float *x, float *y,
                                cudaStream_t stream) {
    ADLBR_NVTX("adlbr_unet_forward");
    if (!n || !params || !x || !y) return fail(ADLBR_E_ARG, "null argument");
    return unet_forward(n, params, x, y, stream);
}

adlbr_status adlbr_unet_backward(adlbr_unet *n, const float *params, const float *gy,
                                 float *gparams, float *gx, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_unet_backward");
    if (!n || !params || !gy || !gparams) return fail(ADLBR_E_ARG, "null argument");
    if (!n->x) return fail(ADLBR_E_ARG, "backward before any forward");
    if (n->fwd_tc) return fail(ADLBR_E_ARG, "backward after a tensor-core (BF16) forward");
    return unet_backward(n, params, gy, gparams, gx, stream);
}

adlbr_status adlbr_adam_step(float *params, const float *grads, float *m, float *v, int64_t n,
                             double lr, double beta1, double beta2, double eps, int t,
                             cudaStream_t stream) {
    if (!params || !grads || !m || !v || n < 0 || t < 1) return fail(ADLBR_E_ARG, "bad argument");
    return unet_adam(params, grads, m, v, n, lr, beta1, beta2, eps, t, stream);
}

}  // extern "C"

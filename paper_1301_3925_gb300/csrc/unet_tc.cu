// 3x3 convolution + bias + ReLU on the 5th-generation tensor cores
// (tcgen05), for the U-Net's inference path (the learned preconditioner).
//
// Implicit GEMM without im2col.  A CTA (4 warps) owns 128 consecutive output
// pixels of a strip of image rows, for all CO output channels:
//   D[128 x CO] (TMEM, FP32) = sum over the 9 taps (dy, dx) and the channel
//   blocks of 16 of A_(dy,dx)[128 x 16] * W_(dy,dx)[CO x 16]^T.
// Input rows are staged once each, in BF16, as 130 pixels (x0 - 1 ..
// x0 + 128) x Kp channels (Ci zero-padded to a multiple of 16) in the
// no-swizzle K-major layout with the pixel as the row:
//   element (q, ci) at (ci / 8) * LBO + q * 16 + (ci % 8) * 2, LBO = 136 * 16,
// i.e. core matrices of 8 pixels x 8 channels, 8-row groups 128 B apart
// (SBO = 128).  A shift of the tap by dx pixels is then a shift of the
// descriptor's start address by 16 dx bytes: every tap of a staged row is
// the same buffer.  The weights of all 9 taps stay in shared memory for the
// whole strip, prepacked per tap in the K-major layout (co / 8) * 16 Kp +
// (ci / 8) * 128 + (co % 8) * 16 + (ci % 8) * 2.
//
// Pipeline over the strip (4 input-row slots, 2 TMEM accumulators): while the
// 9 Kp / 16 MMAs of output row y run (issued by one thread, committed to the
// accumulator's mbarrier), the threads stage input row y + 2 and write output
// row y - 1 from the other accumulator (tcgen05.ld, bias, ReLU, FP32 NCHW).
// Waits are bounded; a CTA whose wait gives up writes NaN (the flexible
// solver then falls back to plain CG) and stops issuing.
#include <algorithm>

#include <cuda_bf16.h>

#include "internal.cuh"

struct adlbr_unet;

namespace adlbr {

namespace {

constexpr int TCM = 128;          // output pixels per CTA (MMA M)
constexpr int QR = TCM + 8;       // staged pixels per row slot (130 used), multiple of 8
constexpr int NSLOT = 4;          // input-row ring
constexpr unsigned kTcPolls = 1u << 22;

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);   // version bits 46-48 = 0b001; no swizzle
}

// byte offset of (co, ci) in one tap's packed weights (SBO = kp * 16, LBO = 128)
__device__ __forceinline__ int cm_off(int row, int k, int kp) {
    return (row >> 3) * (kp * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ bool bar_wait(uint64_t *bar, unsigned parity) {
    for (unsigned k = 0; k < kTcPolls; ++k) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

inline int kpad(int Ci) { return (Ci + 15) / 16 * 16; }

// Weights W[co][ci][3][3] (FP32) of every 3x3 layer -> packed BF16
// [dy * 3 + dx][co][Kp] in the operand layout; blockIdx.y = layer, one
// launch per forward.
__global__ void pack_weights_kernel(ConvPackTable T, const float *__restrict__ params,
                                    __nv_bfloat16 *__restrict__ out) {
    const int l = blockIdx.y;
    const int Co = T.co[l], Ci = T.ci[l], kp = (Ci + 15) / 16 * 16;
    const int per = Co * kp;
    const float *w = params + T.w_off[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * per; i += gridDim.x * blockDim.x) {
        const int tap = i / per, rem = i - tap * per, co = rem / kp, ci = rem - co * kp;
        const int dy = tap / 3, dx = tap - dy * 3;
        const float v = ci < Ci ? w[((co * Ci + ci) * 3 + dy) * 3 + dx] : 0.f;
        char *base = reinterpret_cast<char *>(out + T.out_off[l]) + (size_t)tap * per * 2;
        *reinterpret_cast<__nv_bfloat16 *>(base + cm_off(co, ci, kp)) = __float2bfloat16_rn(v);
    }
}

// Input row yy of image b into a slot: pixels x0 - 1 .. x0 + QR - 2, zero
// outside the image and for the padding channels.  Each thread takes SU
// (pixel, 8-channel group) items at a time, with all their loads issued
// before the first conversion (the copy is bound by load latency).
constexpr int SU = 4;
__device__ __forceinline__ void stage_row(unsigned char *slot, const float *__restrict__ xb, int Ci, int kp,
                                          int H, int W, int x0, int yy) {
    const int G = kp / 8, items = QR * G;
    const bool rin = (unsigned)yy < (unsigned)H;
    const int64_t plane = (int64_t)H * W;
    const float *row = xb + (int64_t)yy * W;
    for (int i0 = threadIdx.x; i0 < items; i0 += 128 * SU) {
        float v[SU][8];
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            const int i = i0 + u * 128;
            const int q = i % QR, g = i / QR;
            const int gx = x0 - 1 + q;
            const bool in = i < items && rin && (unsigned)gx < (unsigned)W;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int ci = 8 * g + c;
                v[u][c] = (in && ci < Ci) ? row[ci * plane + gx] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            const int i = i0 + u * 128;
            if (i >= items) break;
            const int q = i % QR, g = i / QR;
            uint4 pk;
            __nv_bfloat162 h0 = __floats2bfloat162_rn(v[u][0], v[u][1]), h1 = __floats2bfloat162_rn(v[u][2], v[u][3]);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(v[u][4], v[u][5]), h3 = __floats2bfloat162_rn(v[u][6], v[u][7]);
            pk.x = *reinterpret_cast<unsigned *>(&h0);
            pk.y = *reinterpret_cast<unsigned *>(&h1);
            pk.z = *reinterpret_cast<unsigned *>(&h2);
            pk.w = *reinterpret_cast<unsigned *>(&h3);
            *reinterpret_cast<uint4 *>(slot + (size_t)g * (QR * 16) + q * 16) = pk;
        }
    }
}

template <int CO>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(int Ci, int kp, int H, int W, int rows_per_cta,
                                                         const float *__restrict__ x,
                                                         const __nv_bfloat16 *__restrict__ wpack,
                                                         const float *__restrict__ bias, float *__restrict__ y) {
    static_assert(CO % 16 == 0 && CO >= 16 && CO <= 128, "MMA N");
    constexpr int TMEM_COLS = 2 * CO < 32 ? 32 : 2 * CO;   // two accumulators
    extern __shared__ __align__(1024) unsigned char sm[];
    const size_t wbytes = (size_t)9 * CO * kp * 2, slot_bytes = (size_t)(kp / 8) * QR * 16;
    unsigned char *sW = sm, *sX = sm + wbytes;   // weights, then NSLOT input-row slots
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t bar[2];
    const int t = threadIdx.x, warp = t >> 5;
    const int x0 = blockIdx.x * TCM, b = blockIdx.z;
    const int ya = blockIdx.y * rows_per_cta, yb = min(H, ya + rows_per_cta);
    if (ya >= yb) return;
    const int64_t plane = (int64_t)H * W;
    const float *xb = x + (int64_t)b * Ci * plane;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights of the 9 taps (16-byte copies), input rows ya - 1 and ya
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(wpack);
        uint4 *dst = reinterpret_cast<uint4 *>(sW);
        for (int i = t; i < (int)(wbytes / 16); i += 128) dst[i] = src[i];
    }
    auto slot = [&](int yy) { return sX + (size_t)(((yy % NSLOT) + NSLOT) % NSLOT) * slot_bytes; };
    stage_row(slot(ya - 1), xb, Ci, kp, H, W, x0, ya - 1);
    stage_row(slot(ya), xb, Ci, kp, H, W, x0, ya);
    // instruction descriptor: D f32, A and B bf16, both K-major, N = CO, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CO >> 3) << 17) |
                           ((uint32_t)(TCM >> 4) << 24);
    const unsigned lbo_a = QR * 16, sbo_w = (unsigned)kp * 16;
    bool ok = true;
    const int n = yb - ya;
    const int px = x0 + t;
    for (int j = 0; j <= n; ++j) {
        const int yo = ya + j;   // output row whose MMAs this iteration issues (j < n)
        if (j < n) {
            // input row yo + 1 goes to the slot of row yo - 3, last read by the
            // MMAs of output row yo - 2 (waited for in the previous iteration)
            stage_row(slot(yo + 1), xb, Ci, kp, H, W, x0, yo + 1);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (j < n && t == 0 && ok) {
            const uint32_t acc = tmem_base + (uint32_t)((j & 1) * CO);
            bool first = true;
            for (int dy = 0; dy < 3; ++dy) {
                const unsigned abase = su32(slot(yo + dy - 1));
                for (int dx = 0; dx < 3; ++dx) {
                    const unsigned wbase = su32(sW) + (unsigned)((dy * 3 + dx) * CO * kp * 2);
                    for (int s = 0; s < kp / 16; ++s) {
                        const uint64_t da = smem_desc(abase + dx * 16 + s * 2 * lbo_a, lbo_a, 128);
                        const uint64_t db = smem_desc(wbase + s * 256, 128, sbo_w);
                        const unsigned accum = first ? 0u : 1u;
                        first = false;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                            ::"r"(acc), "l"(da), "l"(db), "r"(idesc), "r"(accum)
                            : "memory");
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&bar[j & 1]))
                         : "memory");
        }
        if (j >= 1) {   // epilogue of output row yo - 1
            const int jj = j - 1, yr = yo - 1;
            ok = __syncthreads_and(ok && bar_wait(&bar[jj & 1], (jj >> 1) & 1));
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)((jj & 1) * CO);
#pragma unroll
            for (int c = 0; c < CO; c += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr + c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (px < W) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int co = c + q;
                        float r = __uint_as_float(v[q]) + bias[co];
                        r = ok ? fmaxf(r, 0.f) : __int_as_float(0x7fc00000);
                        y[((int64_t)b * CO + co) * plane + (int64_t)yr * W + px] = r;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
}

// dynamic shared memory of one CTA
size_t tc_smem(int Co, int Ci) {
    const size_t kp = kpad(Ci);
    return (size_t)9 * Co * kp * 2 + (size_t)NSLOT * (kp / 8) * QR * 16;
}

template <int CO>
adlbr_status launch_tc(int B, int Ci, int H, int W, const float *x, const __nv_bfloat16 *wpack, const float *bias,
                       float *y, cudaStream_t st) {
    const int kp = kpad(Ci);
    // At most 512 / TMEM_COLS CTAs may hold TMEM on one SM at a time; a
    // floor on the shared memory keeps more from being resident (the SM has
    // 228 KB), so tcgen05.alloc never waits for another CTA.
    constexpr int TMEM_COLS = 2 * CO < 32 ? 32 : 2 * CO;
    constexpr int max_ctas = 512 / TMEM_COLS;
    size_t smem = tc_smem(CO, Ci);
    if (max_ctas < 16) smem = std::max(smem, (size_t)(228 * 1024 / (max_ctas + 1)));
    static size_t set = 0;
    if (smem > set) {
        ADLBR_CUDA(cudaFuncSetAttribute(conv3x3_tc_kernel<CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
        set = smem;
    }
    // strips of rows: about two CTAs per SM, at least 2 rows each
    const int cols = (W + TCM - 1) / TCM;
    const int64_t tiles = (int64_t)cols * H * B;
    int rows = (int)std::max<int64_t>(2, (tiles + 2 * 152 - 1) / (2 * 152));
    rows = std::min(rows, H);
    dim3 grid(cols, (H + rows - 1) / rows, B);
    conv3x3_tc_kernel<CO><<<grid, 128, smem, st>>>(Ci, kp, H, W, rows, x, wpack, bias, y);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace

size_t conv_tc_pack_elems(int Co, int Ci) { return (size_t)9 * Co * kpad(Ci); }

adlbr_status conv_tc_pack(const ConvPackTable &T, const float *params, __nv_bfloat16 *out, cudaStream_t st) {
    pack_weights_kernel<<<dim3(32, T.n), 256, 0, st>>>(T, params, out);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

bool conv_tc_supported(int Co, int Ci) {
    // 227 KB of dynamic and static shared memory per CTA (1 KB static here)
    return (Co == 16 || Co == 32 || Co == 64) && Ci >= 1 && tc_smem(Co, Ci) <= 225 * 1024;
}

adlbr_status conv_tc(int B, int Ci, int Co, int H, int W, const float *x, const __nv_bfloat16 *wpack,
                     const float *bias, float *y, cudaStream_t st) {
    switch (Co) {
    case 16: return launch_tc<16>(B, Ci, H, W, x, wpack, bias, y, st);
    case 32: return launch_tc<32>(B, Ci, H, W, x, wpack, bias, y, st);
    case 64: return launch_tc<64>(B, Ci, H, W, x, wpack, bias, y, st);
    }
    return fail(ADLBR_E_ARG, "tensor-core convolution: %d output channels", Co);
}

}  // namespace adlbr

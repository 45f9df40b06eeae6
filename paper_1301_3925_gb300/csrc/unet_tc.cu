// 3x3 convolution + bias + ReLU on the 5th-generation tensor cores
// (tcgen05), for the U-Net's inference path (the learned preconditioner).
//
// Implicit GEMM: one CTA (4 warps) computes 128 consecutive output pixels of
// one image row for all CO output channels:
//   D[128 x CO] (TMEM, FP32) = sum over kernel rows dy of A_dy[128 x Kp] * B_dy[CO x Kp]^T
// with A_dy the BF16 im2col rows (k = dx * Ci + ci, zero-padded to Kp, a
// multiple of 16) built by the threads in shared memory, and B_dy the BF16
// weights, prepacked in the same layout.  Both operands use the K-major,
// no-swizzle core-matrix layout: element (row, k) at byte
//   (row / 8) * SBO + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2,
// SBO = Kp * 16 (descriptor LBO = 128, the K-direction core-matrix stride).
// One thread issues Kp / 16 MMAs (M = 128, N = CO, K = 16) per kernel row and
// commits them to an mbarrier; the epilogue reads the accumulator with
// tcgen05.ld (each warp its 32 TMEM lanes = rows), adds the bias, applies
// the ReLU and writes FP32 NCHW.  Waits are bounded; a block whose wait
// gives up writes NaN to its outputs (the flexible solver then falls back to
// plain CG).
#include <cuda_bf16.h>

#include "internal.cuh"

struct adlbr_unet;

namespace adlbr {

namespace {

constexpr int TCM = 128;   // pixels per CTA (MMA M)
constexpr unsigned kTcPolls = 1u << 22;

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);   // version bits 46-48 = 0b001; no swizzle
}

// byte offset of (row, k) in the core-matrix layout with SBO = kp * 16
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

// Weights W[co][ci][3][3] (FP32) of every 3x3 layer -> packed BF16
// [dy][co][Kp] in the operand layout; blockIdx.y = layer, one launch per forward.
__global__ void pack_weights_kernel(ConvPackTable T, const float *__restrict__ params,
                                    __nv_bfloat16 *__restrict__ out) {
    const int l = blockIdx.y;
    const int Co = T.co[l], Ci = T.ci[l], kp = (3 * Ci + 15) / 16 * 16;
    const int per = Co * kp;
    const float *w = params + T.w_off[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * per; i += gridDim.x * blockDim.x) {
        const int dy = i / per, rem = i - dy * per, co = rem / kp, k = rem - co * kp;
        float v = 0.f;
        if (k < 3 * Ci) {
            const int dx = k / Ci, ci = k - dx * Ci;
            v = w[((co * Ci + ci) * 3 + dy) * 3 + dx];
        }
        char *base = reinterpret_cast<char *>(out + T.out_off[l]) + (size_t)dy * per * 2;
        *reinterpret_cast<__nv_bfloat16 *>(base + cm_off(co, k, kp)) = __float2bfloat16_rn(v);
    }
}

template <int CO>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(int Ci, int kp, int H, int W,
                                                         const float *__restrict__ x,
                                                         const __nv_bfloat16 *__restrict__ wpack,
                                                         const float *__restrict__ bias, float *__restrict__ y) {
    static_assert(CO % 16 == 0 && CO >= 16 && CO <= 256, "MMA N");
    constexpr int TMEM_COLS = CO < 32 ? 32 : CO;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm;                              // 128 x kp bf16
    unsigned char *sB = sm + (size_t)TCM * kp * 2;       // CO x kp bf16
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t bar;
    const int t = threadIdx.x, warp = t >> 5;
    const int x0 = blockIdx.x * TCM, yrow = blockIdx.y, b = blockIdx.z;
    const int64_t plane = (int64_t)H * W;
    const float *xb = x + (int64_t)b * Ci * plane;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    bool ok = true;
    const int px = x0 + t;   // this thread's pixel (im2col row)
    // instruction descriptor: D f32, A and B bf16, both K-major, N = CO, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CO >> 3) << 17) |
                           ((uint32_t)(TCM >> 4) << 24);
    const unsigned sbo = (unsigned)kp * 16;
    for (int dy = 0; dy < 3; ++dy) {
        if (dy > 0) {   // the MMAs of the previous row have read the operands
            ok = ok && bar_wait(&bar, (dy - 1) & 1);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        // A: im2col row of pixel px for kernel row dy (zero outside the image)
        const int yy = yrow + dy - 1;
        const bool rin = (unsigned)yy < (unsigned)H;
        for (int k = 0; k < kp; k += 2) {
            float v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int kk = k + e;
                v[e] = 0.f;
                if (kk < 3 * Ci && rin) {
                    const int dx = kk / Ci, ci = kk - dx * Ci;
                    const int xx = px + dx - 1;
                    if ((unsigned)xx < (unsigned)W && px < W) v[e] = xb[(int64_t)ci * plane + (int64_t)yy * W + xx];
                }
            }
            *reinterpret_cast<__nv_bfloat162 *>(sA + cm_off(t, k, kp)) = __floats2bfloat162_rn(v[0], v[1]);
        }
        // B: this kernel row's packed weights (same layout, contiguous)
        const uint4 *src = reinterpret_cast<const uint4 *>(wpack + (size_t)dy * CO * kp);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        for (int i = t; i < CO * kp / 8; i += 128) dst[i] = src[i];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t == 0) {
            const uint32_t tmem = tmem_base;
            for (int s = 0; s < kp / 16; ++s) {
                const uint64_t da = smem_desc(su32(sA) + s * 256, 128, sbo);
                const uint64_t db = smem_desc(su32(sB) + s * 256, 128, sbo);
                const unsigned acc = (dy > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&bar))
                         : "memory");
        }
    }
    ok = ok && bar_wait(&bar, 0);   // third commit: phase parity 0
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: rows of this warp's 32 TMEM lanes
    const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c = 0; c < CO; c += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr + c));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (px < W) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int co = c + j;
                float r = __uint_as_float(v[j]) + bias[co];
                r = ok ? fmaxf(r, 0.f) : __int_as_float(0x7fc00000);
                y[((int64_t)b * CO + co) * plane + (int64_t)yrow * W + px] = r;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
}

template <int CO>
adlbr_status launch_tc(int B, int Ci, int H, int W, const float *x, const __nv_bfloat16 *wpack, const float *bias,
                       float *y, cudaStream_t st) {
    const int kp = (3 * Ci + 15) / 16 * 16;
    // At most 512 / TMEM_COLS CTAs may hold TMEM on one SM at a time; a
    // floor on the shared memory keeps that many from being resident (CO = 64:
    // 9 CTAs of 25 KB and more do not fit the SM's 228 KB), so tcgen05.alloc
    // never waits for another CTA.
    size_t smem = (size_t)(TCM + CO) * kp * 2;
    if (CO == 64 && smem < 25 * 1024 + 512) smem = 25 * 1024 + 512;
    static size_t set = 0;
    if (smem > set) {
        ADLBR_CUDA(cudaFuncSetAttribute(conv3x3_tc_kernel<CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
        set = smem;
    }
    dim3 grid((W + TCM - 1) / TCM, H, B);
    conv3x3_tc_kernel<CO><<<grid, 128, smem, st>>>(Ci, kp, H, W, x, wpack, bias, y);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace

size_t conv_tc_pack_elems(int Co, int Ci) { return (size_t)3 * Co * ((3 * Ci + 15) / 16 * 16); }

adlbr_status conv_tc_pack(const ConvPackTable &T, const float *params, __nv_bfloat16 *out, cudaStream_t st) {
    pack_weights_kernel<<<dim3(32, T.n), 256, 0, st>>>(T, params, out);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

bool conv_tc_supported(int Co, int Ci) { return (Co == 16 || Co == 32 || Co == 64) && 3 * Ci <= 480; }

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

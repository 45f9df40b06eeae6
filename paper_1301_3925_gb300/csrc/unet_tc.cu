// The U-Net's inference path on the 5th-generation tensor cores (tcgen05),
// for the learned preconditioner.  Activations are BF16, channels last
// ([B][H][W][C], C a multiple of 8); every 3x3 convolution + bias + ReLU is
// an implicit GEMM with an FP32 accumulator in tensor memory.
//
// Convolution.  A CTA (5 warps) owns 128 consecutive output pixels of a
// strip of image rows, for all CO output channels:
//   D[128 x CO] (TMEM, FP32) = sum over the 9 taps (dy, dx) and the channel
//   blocks of 16 of A_(dy,dx)[128 x 16] * W_(dy,dx)[CO x 16]^T.
// An input row is staged once: for every group of 8 channels one TMA copy of
// a box of 130 pixels (x0 - 1 .. x0 + 128) x 8 channels lands as 130 rows of
// 16 bytes, the no-swizzle K-major core-matrix layout with the pixel as the
// matrix row (8-row groups 128 B apart: SBO = 128; channel groups LBO = 136 *
// 16 B apart).  A tap shifted by dx pixels is the same buffer with the
// descriptor's start address 16 dx bytes later, so there is no im2col.  TMA
// fills pixels and rows outside the image with zeros (the padding of the
// convolution).  The decoder's concatenated input [up, skip] is read from
// its two tensors (the first groups from one map, the rest from the other),
// so it is never materialised.  The weights of the 9 taps, prepacked per tap
// in the K-major layout (co / 8) * 16 Kp + (ci / 8) * 128 + (co % 8) * 16 +
// (ci % 8) * 2, stay in shared memory for the whole strip.
//
// Pipeline over the strip, warp-specialised: one lane of a producer warp
// issues the TMA copies into 5 input-row slots (4 where 5 do not fit) and the
// 9 Kp / 16 MMAs of each output row into one of 2 TMEM accumulators; four
// epilogue warps read a finished accumulator (tcgen05.ld), add the bias,
// apply the ReLU and write BF16 with 16-byte stores while the next row's MMAs
// run.  The roles meet only at mbarriers (slot full / empty, accumulator full
// / empty); every wait is bounded and gives up early once another role has
// given up, and a CTA that gave up writes NaN (the flexible solver then falls
// back to plain CG).
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "tma.cuh"

namespace adlbr {

namespace {

constexpr int TCM = 128;          // output pixels per CTA (MMA M)
constexpr int QB = TCM + 2;       // staged pixels per row (box width)
constexpr int QR = TCM + 8;       // pixel rows per channel group in a slot (136 x 16 B)
constexpr int NSLOT = 5;          // input-row ring: two rows of prefetch (4 slots, one row, where
                                  // five do not fit)

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);   // version bits 46-48 = 0b001; no swizzle
}

// byte offset of (co, ci) in one tap's packed weights (SBO = kp * 16, LBO = 128)
__device__ __forceinline__ int cm_off(int row, int k, int kp) {
    return (row >> 3) * (kp * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
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

struct ConvMaps {
    CUtensorMap m0, m1;   // [B][H][W][C0] and [B][H][W][C1] (m1 = m0 when there is one input)
};

__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// Bounded wait on a barrier phase that also gives up as soon as *abort is set.
__device__ __forceinline__ bool bar_wait_or_abort(uint64_t *bar, unsigned parity, const volatile int *abort) {
    for (unsigned k = 0; k < tma::kMaxPolls; ++k) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort) return false;
    }
    return false;
}

// Warp-specialised: warps 0-3 are the epilogue (TMEM lanes 0-127), lane 0 of
// warp 4 is the producer (TMA copies and MMAs).  Barriers: full[s] (copies
// of slot s landed), empty[s] (the MMAs of the last output row reading slot
// s are done; committed by the producer), afull[b] (accumulator b holds a
// finished row), aempty[b] (the 4 epilogue warps have read accumulator b).
constexpr int NT_TC = 160;

template <int CO>
__global__ void __launch_bounds__(NT_TC) conv3x3_tc_kernel(const __grid_constant__ ConvMaps maps, int g0, int kp,
                                                           int nslot, int H, int W, int rows_per_cta,
                                                           const __nv_bfloat16 *__restrict__ wpack,
                                                           const float *__restrict__ bias,
                                                           __nv_bfloat16 *__restrict__ y) {
    static_assert(CO % 16 == 0 && CO >= 16 && CO <= 128, "MMA N");
    constexpr int TMEM_COLS = 2 * CO < 32 ? 32 : 2 * CO;   // two accumulators
    extern __shared__ __align__(1024) unsigned char sm[];
    const int G = kp / 8;
    const size_t wbytes = (size_t)9 * CO * kp * 2, slot_bytes = (size_t)G * QR * 16;
    unsigned char *sW = sm, *sX = sm + wbytes;   // weights, then nslot input-row slots
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t full[NSLOT], empty[NSLOT], afull[2], aempty[2];
    __shared__ volatile int abort_flag;
    __shared__ float sbias[CO];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int x0 = blockIdx.x * TCM, b = blockIdx.z;
    const int ya = blockIdx.y * rows_per_cta, yb = min(H, ya + rows_per_cta);
    if (ya >= yb) return;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        for (int s = 0; s < nslot; ++s) {
            tma::bar_init(&full[s], 1);
            tma::bar_init(&empty[s], 1);
        }
        for (int k = 0; k < 2; ++k) {
            tma::bar_init(&afull[k], 1);
            tma::bar_init(&aempty[k], 4);
        }
        abort_flag = 0;
    }
    {   // weights of the 9 taps (16-byte copies) and the bias
        const uint4 *src = reinterpret_cast<const uint4 *>(wpack);
        uint4 *dst = reinterpret_cast<uint4 *>(sW);
        for (int i = t; i < (int)(wbytes / 16); i += NT_TC) dst[i] = src[i];
        if (t < CO) sbias[t] = bias[t];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int n = yb - ya;
    // input row yy (>= ya - 1) lives in slot (yy - ya + 1) % nslot; it is
    // that slot's fill number (yy - ya + 1) / nslot
    auto slot_of = [&](int yy) { return (yy - ya + 1) % nslot; };
    auto fill_of = [&](int yy) { return (yy - ya + 1) / nslot; };
    if (warp == 4) {
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CO >> 3) << 17) |
                                   ((uint32_t)(TCM >> 4) << 24);
            const unsigned lbo_a = QR * 16, sbo_w = (unsigned)kp * 16;
            bool ok = true;
            // the copies of input row r into its slot, once the slot's previous
            // row is no longer read (its freeing commit is done)
            auto load = [&](int r) -> bool {
                const int s = slot_of(r), k = fill_of(r);
                if (k >= 1 && !bar_wait_or_abort(&empty[s], (unsigned)((k - 1) & 1), &abort_flag)) return false;
                unsigned char *dst = sX + (size_t)s * slot_bytes;
                tma::bar_expect_tx(&full[s], (unsigned)(G * QB * 16));
                for (int g = 0; g < G; ++g) {
                    const bool first = g < g0;
                    const CUtensorMap *m = first ? &maps.m0 : &maps.m1;
                    const int c = 8 * (first ? g : g - g0);
                    asm volatile(
                        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
                        "{%2, %3, %4, %5}], [%6];" ::"r"(su32(dst + (size_t)g * QR * 16)),
                        "l"(reinterpret_cast<uint64_t>(m)), "r"(c), "r"(x0 - 1), "r"(r), "r"(b),
                        "r"(su32(&full[s]))
                        : "memory");
                }
                return true;
            };
            int next = ya - 1;   // next input row to copy
            for (; ok && next <= min(yb, ya - 1 + nslot - 1); ++next) ok = load(next);
            int issued = 0;
            for (int j = 0; ok && j < n; ++j) {
                const int yo = ya + j;
                for (int dy = 0; ok && dy < 3; ++dy)
                    ok = bar_wait_or_abort(&full[slot_of(yo + dy - 1)], (unsigned)(fill_of(yo + dy - 1) & 1),
                                           &abort_flag);
                if (ok && j >= 2) ok = bar_wait_or_abort(&aempty[j & 1], (unsigned)(((j >> 1) - 1) & 1), &abort_flag);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem_base + (uint32_t)((j & 1) * CO);
                bool first = true;
                for (int dy = 0; dy < 3; ++dy) {
                    const unsigned abase = su32(sX + (size_t)slot_of(yo + dy - 1) * slot_bytes);
                    for (int dx = 0; dx < 3; ++dx) {
                        const unsigned wb = su32(sW) + (unsigned)((dy * 3 + dx) * CO * kp * 2);
                        for (int s = 0; s < kp / 16; ++s) {
                            const uint64_t da = smem_desc(abase + dx * 16 + s * 2 * lbo_a, lbo_a, 128);
                            const uint64_t db = smem_desc(wb + s * 256, 128, sbo_w);
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
                                 su32(&afull[j & 1]))
                             : "memory");
                // input row yo - 1 is read by no later output row
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&empty[slot_of(yo - 1)]))
                             : "memory");
                issued = j + 1;
                // refill slots freed by output rows up to yo - 1
                for (; ok && next <= min(yb, yo + nslot - 2); ++next) ok = load(next);
            }
            if (!ok) abort_flag = 1;
            // nothing may be in flight when the CTA exits: the last MMAs, and
            // the copies of the last nslot rows (bounded waits)
            if (issued > 0) tma::bar_wait(&afull[(issued - 1) & 1], (unsigned)(((issued - 1) >> 1) & 1));
            for (int r = max(ya - 1, next - nslot); r < next; ++r)
                tma::bar_wait(&full[slot_of(r)], (unsigned)(fill_of(r) & 1));
        }
        __syncwarp();   // the warp meets again before the block barrier below
    } else {
        const int px = x0 + t;   // this thread's pixel = TMEM lane
        const int64_t row_stride = (int64_t)W * CO;
        for (int j = 0; j < n; ++j) {
            const bool ok = bar_wait_or_abort(&afull[j & 1], (unsigned)((j >> 1) & 1), &abort_flag);
            if (!ok) abort_flag = 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)((j & 1) * CO);
            uint32_t pk[CO / 2];
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
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float r0 = __uint_as_float(v[2 * q]) + sbias[c + 2 * q];
                    float r1 = __uint_as_float(v[2 * q + 1]) + sbias[c + 2 * q + 1];
                    r0 = ok ? fmaxf(r0, 0.f) : __int_as_float(0x7fc00000);
                    r1 = ok ? fmaxf(r1, 0.f) : __int_as_float(0x7fc00000);
                    __nv_bfloat162 h = __floats2bfloat162_rn(r0, r1);
                    pk[c / 2 + q] = *reinterpret_cast<uint32_t *>(&h);
                }
            }
            // the accumulator is read: hand it back to the producer
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&aempty[j & 1]);
            if (px < W) {
                uint4 *d4 = reinterpret_cast<uint4 *>(y + ((int64_t)b * H + ya + j) * row_stride + (int64_t)px * CO);
#pragma unroll
                for (int q = 0; q < CO / 8; ++q) d4[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
}

// dynamic shared memory of one CTA with nslot row slots
size_t tc_smem(int Co, int kp, int nslot) { return (size_t)9 * Co * kp * 2 + (size_t)nslot * (kp / 8) * QR * 16; }
constexpr size_t kSmemCap = 225 * 1024;   // of 227 KB per CTA (about 1 KB static)

// 4D map over a BF16 [B][H][W][C] tensor, box 8 channels x QB pixels x 1 x 1.
bool encode_act(CUtensorMap *map, const __nv_bfloat16 *base, int B, int H, int W, int C) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tma::encoder();
    if (!encode || ((uintptr_t)base & 15) || C % 8) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)QB, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(base), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int CO>
adlbr_status launch_tc(int B, int H, int W, const ConvMaps &maps, int g0, int kp, const __nv_bfloat16 *wpack,
                       const float *bias, __nv_bfloat16 *y, cudaStream_t st) {
    // At most 512 / TMEM_COLS CTAs may hold TMEM on one SM at a time; a
    // floor on the shared memory keeps more from being resident (the SM has
    // 228 KB), so tcgen05.alloc never waits for another CTA.
    constexpr int TMEM_COLS = 2 * CO < 32 ? 32 : 2 * CO;
    constexpr int max_ctas = 512 / TMEM_COLS;
    const int nslot = tc_smem(CO, kp, NSLOT) <= kSmemCap ? NSLOT : NSLOT - 1;
    size_t smem = tc_smem(CO, kp, nslot);
    if (max_ctas < 16) smem = std::max(smem, (size_t)(228 * 1024 / (max_ctas + 1)));
    static size_t set = 0;
    if (smem > set) {
        ADLBR_CUDA(cudaFuncSetAttribute(conv3x3_tc_kernel<CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
        set = smem;
    }
    // strips of rows: about eight strips per SM (one row each on small
    // levels).  Measured forwards (25 -> 16/32/64, batch 1): 0.245 / 0.612 /
    // 0.141 ms at 512^2 / 1024^2 / 256^2 against 0.265 / 0.693 / 0.164 with
    // two strips per SM of at least 2 rows; deeper row prefetch (all rows of
    // a strip in flight) changed nothing, so the strips are not waiting on
    // their copies.
    const int cols = (W + TCM - 1) / TCM;
    const int64_t tiles = (int64_t)cols * H * B;
    int rows = (int)std::max<int64_t>(1, (tiles + vec_blocks() - 1) / vec_blocks());
    rows = std::min(rows, H);
    dim3 grid(cols, (H + rows - 1) / rows, B);
    conv3x3_tc_kernel<CO><<<grid, NT_TC, smem, st>>>(maps, g0, kp, nslot, H, W, rows, wpack, bias, y);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

// ---- the layers around the convolutions (BF16, channels last) ------------

// FP32 [B][C][HW] -> BF16 [B][HW][Cp], channels C .. Cp - 1 zero
__device__ __forceinline__ void unpack8(const uint4 &r, float (&f)[8]) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 v = __bfloat1622float2(h[k]);
        f[2 * k] = v.x;
        f[2 * k + 1] = v.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 r;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    return r;
}

// One thread per pixel: the C plane reads of a warp are 32 consecutive floats
// each, and the pixel's Cp channels (a multiple of 8) go out as 16-byte
// stores.  (Two channels per thread, with lanes across channels, read 8 bytes
// of each 32-byte sector and took 21 us at 512^2, 25 -> 32 channels.)
__global__ void to_nhwc_kernel(int B, int C, int Cp, int64_t HW, const float *__restrict__ x,
                               __nv_bfloat16 *__restrict__ y) {
    const int64_t n = (int64_t)B * HW;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = p / HW, q = p - b * HW;
        const float *xs = x + b * C * HW + q;
        uint4 *d = reinterpret_cast<uint4 *>(y + p * Cp);
        for (int c0 = 0; c0 < Cp; c0 += 8) {
            float f[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = c0 + k < C ? xs[(int64_t)(c0 + k) * HW] : 0.f;
            d[c0 / 8] = pack8(f);
        }
    }
}

// 2 x 2 average pooling: [B][2H2][2W2][C] -> [B][H2][W2][C], 8 channels a thread
__global__ void pool_nhwc_kernel(int B, int H2, int W2, int C, const __nv_bfloat16 *__restrict__ x,
                                 __nv_bfloat16 *__restrict__ y) {
    const int G = C / 8;
    const int64_t n = (int64_t)B * H2 * W2 * G;
    const uint4 *x4 = reinterpret_cast<const uint4 *>(x);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(i % G);
        int64_t p = i / G;
        const int w = (int)(p % W2);
        p /= W2;
        const int h = (int)(p % H2);
        const int64_t b = p / H2;
        const int64_t r0 = ((b * 2 * H2 + 2 * h) * 2 * W2 + 2 * w) * G + g, r1 = r0 + (int64_t)2 * W2 * G;
        float a[8], c[8], d[8], e[8], o[8];
        unpack8(x4[r0], a);
        unpack8(x4[r0 + G], c);
        unpack8(x4[r1], d);
        unpack8(x4[r1 + G], e);
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = 0.25f * (a[k] + c[k] + d[k] + e[k]);
        reinterpret_cast<uint4 *>(y)[i] = pack8(o);
    }
}

// nearest 2x upsampling: [B][H][W][C] -> [B][2H][2W][C]
__global__ void up_nhwc_kernel(int B, int H, int W, int C, const __nv_bfloat16 *__restrict__ x,
                               __nv_bfloat16 *__restrict__ y) {
    const int G = C / 8;
    const int64_t n = (int64_t)B * 4 * H * W * G;
    const uint4 *x4 = reinterpret_cast<const uint4 *>(x);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(i % G);
        int64_t p = i / G;
        const int w2 = (int)(p % (2 * W));
        p /= 2 * W;
        const int h2 = (int)(p % (2 * H));
        const int64_t b = p / (2 * H);
        reinterpret_cast<uint4 *>(y)[i] = x4[((b * H + h2 / 2) * W + w2 / 2) * G + g];
    }
}

// output layer: y[b][p] = bias + sum_c w[c] x[b][p][c] (FP32 out)
__global__ void out1x1_nhwc_kernel(int64_t n, int C, const __nv_bfloat16 *__restrict__ x,
                                   const float *__restrict__ w, const float *__restrict__ bias,
                                   float *__restrict__ y) {
    const int G = C / 8;
    const uint4 *x4 = reinterpret_cast<const uint4 *>(x);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float acc = bias[0];
        for (int g = 0; g < G; ++g) {
            float f[8];
            unpack8(x4[i * G + g], f);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc = fmaf(w[8 * g + k], f[k], acc);
        }
        y[i] = acc;
    }
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2 * vec_blocks())); }

}  // namespace

size_t conv_tc_pack_elems(int Co, int Ci) { return (size_t)9 * Co * kpad(Ci); }

adlbr_status conv_tc_pack(const ConvPackTable &T, const float *params, __nv_bfloat16 *out, cudaStream_t st) {
    pack_weights_kernel<<<dim3(32, T.n), 256, 0, st>>>(T, params, out);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

bool conv_tc_supported(int Co, int Ci) {
    return (Co == 16 || Co == 32 || Co == 64) && Ci >= 1 && tc_smem(Co, kpad(Ci), NSLOT - 1) <= kSmemCap;
}

adlbr_status conv_tc(int B, int H, int W, const __nv_bfloat16 *x0, int C0, const __nv_bfloat16 *x1, int C1,
                     int Co, const __nv_bfloat16 *wpack, const float *bias, __nv_bfloat16 *y, cudaStream_t st) {
    const int kp = C0 + C1;
    if (kp % 16 || C0 % 8 || C1 % 8 || (C1 && !x1) || W < 1 || H < 1)
        return fail(ADLBR_E_ARG, "tensor-core convolution: %d + %d input channels", C0, C1);
    ConvMaps maps;
    if (!encode_act(&maps.m0, x0, B, H, W, C0) || (C1 && !encode_act(&maps.m1, x1, B, H, W, C1)))
        return fail(ADLBR_E_CUDA, "tensor-core convolution: tensor map encoding failed");
    if (!C1) maps.m1 = maps.m0;
    const int g0 = C0 / 8;
    switch (Co) {
    case 16: return launch_tc<16>(B, H, W, maps, g0, kp, wpack, bias, y, st);
    case 32: return launch_tc<32>(B, H, W, maps, g0, kp, wpack, bias, y, st);
    case 64: return launch_tc<64>(B, H, W, maps, g0, kp, wpack, bias, y, st);
    }
    return fail(ADLBR_E_ARG, "tensor-core convolution: %d output channels", Co);
}

adlbr_status tc_to_nhwc(int B, int C, int Cp, int64_t HW, const float *x, __nv_bfloat16 *y, cudaStream_t st) {
    to_nhwc_kernel<<<grid_for((int64_t)B * HW), 256, 0, st>>>(B, C, Cp, HW, x, y);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status tc_pool(int B, int H2, int W2, int C, const __nv_bfloat16 *x, __nv_bfloat16 *y, cudaStream_t st) {
    pool_nhwc_kernel<<<grid_for((int64_t)B * H2 * W2 * C / 8), 256, 0, st>>>(B, H2, W2, C, x, y);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status tc_up(int B, int H, int W, int C, const __nv_bfloat16 *x, __nv_bfloat16 *y, cudaStream_t st) {
    up_nhwc_kernel<<<grid_for((int64_t)B * 4 * H * W * C / 8), 256, 0, st>>>(B, H, W, C, x, y);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status tc_out1x1(int64_t n, int C, const __nv_bfloat16 *x, const float *w, const float *bias, float *y,
                       cudaStream_t st) {
    out1x1_nhwc_kernel<<<grid_for(n), 256, 0, st>>>(n, C, x, w, bias, y);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace adlbr

// Tensor-memory-accelerator (TMA) copies of 2D tiles into shared memory,
// completed through an mbarrier (Hopper/Blackwell bulk-tensor path), and the
// host-side tensor-map encoding through the driver entry point.
//
// Every wait on the barrier is bounded: after kMaxPolls unsuccessful polls a
// thread gives up and reports it, so a copy that never lands cannot hang the
// kernel.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"

namespace adlbr {
namespace tma {

constexpr unsigned kMaxPolls = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Poll the barrier's phase `parity`; false after kMaxPolls failed polls.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, unsigned parity) {
    for (unsigned k = 0; k < kMaxPolls; ++k) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Block-wide wait for the barrier's phase `parity`: one thread polls (bounded,
// as bar_wait) while the others sleep in the block barrier, so that a waiting
// block takes no issue slots from the blocks that compute beside it on the
// SM.  Every thread of the block must call it; all get the same result.
// The polling thread's acquire of the phase and the block barrier after it
// make the copied data visible to every thread.
__device__ __forceinline__ bool bar_wait_block(uint64_t *bar, unsigned parity, int *flag) {
    if (threadIdx.x == 0) *flag = bar_wait(bar, parity) ? 1 : 0;
    __syncthreads();
    return *flag != 0;
}

// Box of the tensor map at element coordinates (x, y) into dst (16-byte
// aligned); x * 4 bytes must be a multiple of 16 (FP32 maps: x % 4 == 0).
// Cells outside the tensor are zero-filled.
__device__ __forceinline__ void load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

inline PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return encode;
}

// Host: a 3D FP32 tensor map over an nx x ny x nz array (x fastest) with a
// box of bx x by x bz elements (zero fill out of bounds).
inline bool encode_3d_f32(CUtensorMap *map, const float *base, int nx, int ny, int nz, int bx, int by, int bz) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = encoder();
    if (!encode) return false;
    if (((uintptr_t)base & 15) || (nx % 4) || bx > 256 || by > 256 || bz > 256 || (bx * 4) % 16) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Host: a 3D map of 16-bit elements (F16 / BF16 bits, zero fill) over an
// nx x ny x nz array with a box of bx x by x bz elements; the row pitch and
// every copy's x must be 16-byte multiples: nx % 8 == 0, x % 8 == 0.
inline bool encode_3d_u16(CUtensorMap *map, const void *base, int nx, int ny, int nz, int bx, int by, int bz) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = encoder();
    if (!encode) return false;
    if (((uintptr_t)base & 15) || (nx % 8) || bx > 256 || by > 256 || bz > 256 || (bx * 2) % 16) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 2, (cuuint64_t)nx * ny * 2};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Host: a 2D FP32 tensor map over a row-major nx x ny array with a box of
// bx x by elements (zero fill out of bounds).  False when the driver entry
// point is unavailable or the layout is not encodable (the caller then uses
// plain loads).
inline bool encode_2d_f32(CUtensorMap *map, const float *base, int nx, int ny, int bx, int by) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = encoder();
    if (!encode) return false;
    if (((uintptr_t)base & 15) || (nx % 4) || bx > 256 || by > 256 || (bx * 4) % 16) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)nx * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tma
}  // namespace adlbr

// Deterministic block and grid reductions in FP64 (shared by the solvers).
//
// Every block reduces its values with warp shuffles and one shared-memory
// pass, writes one partial, and the last block to arrive (atomic ticket)
// sums the partials in block order, so the result does not depend on
// scheduling.
#pragma once

#include "internal.cuh"

namespace adlbr {

constexpr int RT = 256;  // threads per reduction block

static __device__ __forceinline__ double block_sum(double v) {
    __shared__ double warp_part[RT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_part[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < RT / 32 ? warp_part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;  // valid in thread 0
}

// Writes this block's partial; returns true in thread 0 of the last block,
// after which total = sum of all partials in block order.
static __device__ __forceinline__ bool finish_reduction(double part, double *partials, unsigned int *count,
                                                 double &total) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = part;
        __threadfence();
        unsigned int t = atomicAdd(count, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RT) s += ((volatile double *)partials)[b];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        total = s;
        *count = 0;
    }
    return threadIdx.x == 0;
}

}  // namespace adlbr

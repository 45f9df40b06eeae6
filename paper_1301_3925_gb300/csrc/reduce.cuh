// Deterministic block and grid reductions (shared by the solvers): FP64
// across warps and blocks, float-float within a thread and a warp.
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

// Per-thread and per-warp accumulation in float-float (hi + lo, about 48
// significant bits): products are split exactly with an fma and the running
// sum is kept with Knuth's TwoSum, all in explicitly rounded FP32 operations;
// only the per-warp results are converted to FP64 for the block and grid
// sums.  (Per-element FP64 arithmetic runs on GB300's narrow FP64 pipe and
// dominated the vector kernels.)
struct FFAcc {
    float hi = 0.f, lo = 0.f;
};

__device__ __forceinline__ void ff_add(FFAcc &a, float x) {
    const float s = __fadd_rn(a.hi, x);
    const float bv = __fsub_rn(s, a.hi);
    const float av = __fsub_rn(s, bv);
    const float e = __fadd_rn(__fsub_rn(a.hi, av), __fsub_rn(x, bv));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}

__device__ __forceinline__ void ff_add_prod(FFAcc &a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);
    ff_add(a, p);
    a.lo = __fadd_rn(a.lo, pe);
}

static __device__ __forceinline__ double block_sum_ff(FFAcc v) {
    __shared__ double warp_part_ff[RT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_down_sync(0xffffffffu, v.hi, o);
        const float l = __shfl_down_sync(0xffffffffu, v.lo, o);
        ff_add(v, h);
        v.lo = __fadd_rn(v.lo, l);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_part_ff[wid] = (double)v.hi + (double)v.lo;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < RT / 32 ? warp_part_ff[lane] : 0.0;
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

// The same for two sums at once; the last block reduces both arrays of
// partials in parallel.
static __device__ __forceinline__ bool finish_reduction2(double part, double part2, double *partials,
                                                  double *partials2, unsigned int *count, double &total,
                                                  double &total2) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = part;
        partials2[blockIdx.x] = part2;
        __threadfence();
        unsigned int t = atomicAdd(count, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RT) {
        s += ((volatile double *)partials)[b];
        s2 += ((volatile double *)partials2)[b];
    }
    s = block_sum(s);
    s2 = block_sum(s2);
    if (threadIdx.x == 0) {
        total = s;
        total2 = s2;
        *count = 0;
    }
    return threadIdx.x == 0;
}

}  // namespace adlbr

// Writing one point's weights in the handle's storage format.
#pragma once

#include "exact.cuh"
#include "internal.cuh"

namespace adlbr {

__device__ __forceinline__ float to_f(FF v) { return __fadd_rn(v.hi, v.lo); }
__device__ __forceinline__ double to_d(FF v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ float to_f(double v) { return (float)v; }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ FF neg_half(FF v) { return FF{-0.5f * v.hi, -0.5f * v.lo}; }
__device__ __forceinline__ double neg_half(double v) { return -0.5 * v; }
__device__ __forceinline__ FF wmax0(FF v) { return (v.hi > 0.f || (v.hi == 0.f && v.lo > 0.f)) ? v : FF{0.f, 0.f}; }
__device__ __forceinline__ double wmax0(double v) { return fmax(v, 0.0); }

// w[0..K) are the weights (>= 0, +0 where zmask has the bit set).  Returns
// the stored record for the F16 format (its first 8 bytes for K = 3, all 16
// for K = 6), zeros for the other formats.
template <int K, typename V>
__device__ __forceinline__ uint4 store_weights(void *wbase, adlbr_dtype wt, int64_t i,
                                               const V (&w)[K], unsigned zmask) {
    constexpr int L = (K == 3) ? 4 : 8;
    if (wt == ADLBR_F16) {
        float wf[K];
        float wmax = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            wf[k] = to_f(w[k]);
            wmax = fmaxf(wmax, wf[k]);
        }
        // per-point scale 2^s with wmax / 2^s in [1/2, 1): 11 significant
        // bits for the largest weight, no underflow for ratios above 2^-14
        int s = 0;
        if (wmax > 0.f) {
            const int ex = (__float_as_int(wmax) >> 23) & 0xff;  // biased exponent
            s = (ex == 0 ? -126 : ex - 127) + 1;
            s = max(-120, min(120, s));
        }
        const float inv = __int_as_float((127 - s) << 23);
        __half h[L];
#pragma unroll
        for (int k = 0; k < L; ++k) h[k] = __ushort_as_half((unsigned short)0);
        // wf[k] * inv lies in [0, 1): the rounding of f2h_bits without its
        // sign and overflow cases (round to nearest even, subnormals too)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t bb = __float_as_uint(__fmul_rn(__fmul_rn(wf[k], inv), 0x1p-112f));
            h[k] = __ushort_as_half((unsigned short)((bb + 0x0fffu + ((bb >> 13) & 1u)) >> 13));
        }
        uint16_t meta = (uint16_t)((zmask & 0xffu) | ((unsigned)(uint8_t)(int8_t)s << 8));
        *reinterpret_cast<uint16_t *>(&h[K]) = meta;
        if (L == 4) {
            const uint2 r = *reinterpret_cast<uint2 *>(h);
            reinterpret_cast<uint2 *>(wbase)[i] = r;
            return make_uint4(r.x, r.y, 0u, 0u);
        }
        const uint4 r = *reinterpret_cast<uint4 *>(h);
        reinterpret_cast<uint4 *>(wbase)[i] = r;
        return r;
    } else if (wt == ADLBR_F32) {
        float v[L];
#pragma unroll
        for (int k = 0; k < L; ++k) v[k] = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = to_f(w[k]);
        v[K] = (float)zmask;
        float *p = reinterpret_cast<float *>(wbase) + i * L;
#pragma unroll
        for (int k = 0; k < L; k += 4) *reinterpret_cast<float4 *>(p + k) = *reinterpret_cast<float4 *>(v + k);
    } else {
        double v[L];
#pragma unroll
        for (int k = 0; k < L; ++k) v[k] = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = to_d(w[k]);
        v[K] = (double)zmask;
        double *p = reinterpret_cast<double *>(wbase) + i * L;
#pragma unroll
        for (int k = 0; k < L; k += 2) *reinterpret_cast<double2 *>(p + k) = *reinterpret_cast<double2 *>(v + k);
    }
    return make_uint4(0u, 0u, 0u, 0u);
}

}  // namespace adlbr

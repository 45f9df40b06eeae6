// Writing one point's weights in the handle's storage format.
#pragma once

#include "internal.cuh"

namespace adlbr {

// w[0..K) are the weights (>= 0, +0 where zmask has the bit set).
template <int K>
__device__ __forceinline__ void store_weights(void *wbase, adlbr_dtype wt, int64_t i,
                                              const double (&w)[K], unsigned zmask) {
    constexpr int L = (K == 3) ? 4 : 8;
    if (wt == ADLBR_F16) {
        double wmax = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) wmax = fmax(wmax, w[k]);
        // per-point scale 2^s with wmax / 2^s in [1/2, 1): 11 significant
        // bits for the largest weight, no underflow for ratios above 2^-14
        int s = 0;
        if (wmax > 0.0) {
            s = ilogb(wmax) + 1;
            s = max(-120, min(120, s));
        }
        double inv = ldexp(1.0, -s);
        __half h[L];
#pragma unroll
        for (int k = 0; k < L; ++k) h[k] = __float2half_rn(0.f);
#pragma unroll
        for (int k = 0; k < K; ++k) h[k] = __float2half_rn((float)(w[k] * inv));
        uint16_t meta = (uint16_t)((zmask & 0xffu) | ((unsigned)(uint8_t)(int8_t)s << 8));
        *reinterpret_cast<uint16_t *>(&h[K]) = meta;
        if (L == 4)
            reinterpret_cast<uint2 *>(wbase)[i] = *reinterpret_cast<uint2 *>(h);
        else
            reinterpret_cast<uint4 *>(wbase)[i] = *reinterpret_cast<uint4 *>(h);
    } else if (wt == ADLBR_F32) {
        float v[L];
#pragma unroll
        for (int k = 0; k < L; ++k) v[k] = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (float)w[k];
        v[K] = (float)zmask;
        float *p = reinterpret_cast<float *>(wbase) + i * L;
#pragma unroll
        for (int k = 0; k < L; k += 4) *reinterpret_cast<float4 *>(p + k) = *reinterpret_cast<float4 *>(v + k);
    } else {
        double v[L];
#pragma unroll
        for (int k = 0; k < L; ++k) v[k] = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = w[k];
        v[K] = (double)zmask;
        double *p = reinterpret_cast<double *>(wbase) + i * L;
#pragma unroll
        for (int k = 0; k < L; k += 2) *reinterpret_cast<double2 *>(p + k) = *reinterpret_cast<double2 *>(v + k);
    }
}

}  // namespace adlbr

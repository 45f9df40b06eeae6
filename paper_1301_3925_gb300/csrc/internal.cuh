// Internal declarations shared by the translation units of libadlbr.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "../../include/adlbr.h"

namespace adlbr {

// ---------------------------------------------------------------- errors
adlbr_status fail(adlbr_status st, const char *fmt, ...);
adlbr_status cuda_fail(cudaError_t e, const char *what);

#define ADLBR_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Sticky per-handle error bits written by device code (atomicOr).
enum : int {
    ERRBIT_NONFINITE = 1 << 0,
    ERRBIT_NOT_SPD = 1 << 1,
    ERRBIT_RANGE = 1 << 2,
    ERRBIT_NOT_CONVERGED = 1 << 3,
};

}  // namespace adlbr

// ---------------------------------------------------------------- handle
// Storage layout in HBM (one record per grid point, SoA planes):
//   2D  offs : short4  (e0.x, e0.y, e1.x, e1.y) of the obtuse superbase
//              (e0, e1, e2 = -e0 - e1);
//       w    : 4 lanes (w0, w1, w2, meta), gamma(+-e_i) = w_i;
//   3D  offs : 3 x char4 (e1, e2, e3; e0 = -e1 - e2 - e3), 12 bytes;
//       w    : 8 lanes (w01, w02, w03, w12, w13, w23, meta, 0), w_ij the
//              weight of the Selling offset e_k x e_l, {k,l} = {0..3}\{i,j}.
// Lane types: F64 double, F32 float, F16 half (+ power-of-two scale).
// meta: bit i (i < K) set when weight i is exactly zero; for F16 the high
//       byte holds the signed exponent s of the per-point scale 2^s.
struct adlbr_stencils {
    int dim;
    int bc;
    int64_t n[3];
    int64_t N;
    adlbr_dtype w_t;
    int device;
    void *offs;        // device
    void *w;           // device
    int *err;          // device, sticky error bits
    int *err_host;     // pinned host mirror
    // lazily allocated solver workspace
    void *ws;
    size_t ws_bytes;
};

namespace adlbr {

inline int K_of(int dim) { return dim == 2 ? 3 : 6; }
inline size_t offs_bytes_per_point(int dim) { return dim == 2 ? 8 : 12; }
inline size_t w_lane_bytes(adlbr_dtype t) { return t == ADLBR_F64 ? 8 : (t == ADLBR_F32 ? 4 : 2); }
inline size_t w_bytes_per_point(int dim, adlbr_dtype t) { return (dim == 2 ? 4 : 8) * w_lane_bytes(t); }

// ---------------------------------------------------------------- value types
template <typename T> struct UTraits;
template <> struct UTraits<double> { using acc = double; };
template <> struct UTraits<float> { using acc = float; };
template <> struct UTraits<__half> { using acc = float; };
template <> struct UTraits<__nv_bfloat16> { using acc = float; };

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_acc(typename UTraits<T>::acc v);
template <> __device__ __forceinline__ double from_acc<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_acc<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------- weights
// Reads the K weights of point i (widened to Acc) and the zero mask.
template <typename Acc, int K>
__device__ __forceinline__ unsigned load_weights(const void *wbase, adlbr_dtype wt, int64_t i,
                                                 Acc (&w)[K]) {
    constexpr int L = (K == 3) ? 4 : 8;
    if (wt == ADLBR_F16) {
        const uint4 *p = reinterpret_cast<const uint4 *>(wbase);
        if (L == 4) {
            uint2 r = reinterpret_cast<const uint2 *>(wbase)[i];
            __half h[4];
            *reinterpret_cast<uint2 *>(h) = r;
            uint16_t meta = *reinterpret_cast<uint16_t *>(&h[3]);
            int s = (int)(int8_t)(meta >> 8);
            float sc = __int_as_float((127 + s) << 23);
#pragma unroll
            for (int k = 0; k < K; ++k) w[k] = (Acc)(__half2float(h[k]) * sc);
            return meta & 0xffu;
        } else {
            uint4 r = p[i];
            __half h[8];
            *reinterpret_cast<uint4 *>(h) = r;
            uint16_t meta = *reinterpret_cast<uint16_t *>(&h[6]);
            int s = (int)(int8_t)(meta >> 8);
            float sc = __int_as_float((127 + s) << 23);
#pragma unroll
            for (int k = 0; k < K; ++k) w[k] = (Acc)(__half2float(h[k]) * sc);
            return meta & 0xffu;
        }
    } else if (wt == ADLBR_F32) {
        const float *p = reinterpret_cast<const float *>(wbase) + i * L;
        float v[L];
        if (L == 4) {
            *reinterpret_cast<float4 *>(v) = *reinterpret_cast<const float4 *>(p);
        } else {
            *reinterpret_cast<float4 *>(v) = *reinterpret_cast<const float4 *>(p);
            *reinterpret_cast<float4 *>(v + 4) = *reinterpret_cast<const float4 *>(p + 4);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = (Acc)v[k];
        return (unsigned)v[K];
    } else {
        const double *p = reinterpret_cast<const double *>(wbase) + i * L;
        double v[L];
#pragma unroll
        for (int k = 0; k < L; k += 2)
            *reinterpret_cast<double2 *>(v + k) = *reinterpret_cast<const double2 *>(p + k);
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = (Acc)v[k];
        return (unsigned)v[K];
    }
}

// ---------------------------------------------------------------- launch helpers
inline unsigned blocks_for(int64_t n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

// API-level validation helpers (api.cu)
adlbr_status check_handle(const adlbr_stencils *s);

// kernels' host launchers
adlbr_status launch_build2d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st);
adlbr_status launch_build3d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st);
adlbr_status launch_export(const adlbr_stencils *s, int16_t *offs, void *w, cudaStream_t st);
adlbr_status launch_apply(const adlbr_stencils *s, const void *u, void *Au, adlbr_dtype u_t,
                          cudaStream_t st);
adlbr_status launch_axpy_zero(const adlbr_stencils *s, void *u, void *acc, adlbr_dtype u_t,
                              double dt, cudaStream_t st);

}  // namespace adlbr

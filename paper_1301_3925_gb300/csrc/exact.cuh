// Exact signs and accurate values of sum_k n_k x_k (small integers n_k,
// floating-point x_k) on the device.
//
// Every decision of the stencil construction is such a sign.  The common
// case is settled by a filter: the sum evaluated in FP32 (FP64 for FP64
// inputs) together with a forward error bound; only when the computed value
// lies within the bound (ties and near-ties) the sum is evaluated exactly as
// a floating-point expansion, accumulated with Shewchuk's Grow-Expansion
// (J. R. Shewchuk, "Adaptive precision floating-point arithmetic and fast
// robust geometric predicates", 1997) over error-free products.  For FP32
// inputs every product n_k * x_k is exact in FP64 (24-bit mantissa times an
// integer below 2^24); for FP64 inputs each product is split by an fma into
// two doubles.  All arithmetic uses explicitly rounded intrinsics so that no
// contraction can change it.
#pragma once

#include <stdint.h>

namespace adlbr {

// An unevaluated float-float sum hi + lo (weights computed from FP32 tensors;
// no FP64 instruction on that path: GB300's FP64 rate is a small fraction of
// its FP32 rate).
struct FF {
    float hi, lo;
};

// Value type of the accurately evaluated weights for input element type T.
template <typename T> struct WVal;
template <> struct WVal<float> { using type = FF; };
template <> struct WVal<double> { using type = double; };

__device__ __forceinline__ void two_sum_d(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// Adds b to the non-overlapping expansion h[0..m) (increasing magnitude).
__device__ __forceinline__ int grow_expansion(double *h, int m, double b) {
    double q = b;
    int mm = 0;
    for (int i = 0; i < m; ++i) {
        double s, e;
        two_sum_d(q, h[i], s, e);
        q = s;
        if (e != 0.0) h[mm++] = e;
    }
    if (q != 0.0) h[mm++] = q;
    return mm;
}

// ---- FP32 inputs, |n_k| < 2^24 -------------------------------------------
template <int K>
__device__ __noinline__ int exact_sign_slow_f32(const float (&x)[K], const int (&n)[K]) {
    double h[K + 1];
    int m = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) m = grow_expansion(h, m, __dmul_rn((double)n[k], (double)x[k]));
    return m == 0 ? 0 : (h[m - 1] > 0.0 ? 1 : -1);
}

template <int K>
__device__ __forceinline__ int exact_sign_f32(const float (&x)[K], const int (&n)[K]) {
    float v = 0.f, A = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float p = __fmul_rn((float)n[k], x[k]);
        v = __fadd_rn(v, p);
        A = __fadd_rn(A, fabsf(p));
    }
    if (A == 0.f) return 0;
    // |v - exact| <= (2K) u A (1 + small); take a factor-2 margin and an
    // absolute term for underflowing products.
    float bound = __fmaf_rn(A, (float)(4 * K + 4) * 0x1p-24f, 0x1p-120f);
    if (fabsf(v) > bound) return v > 0.f ? 1 : -1;
    return exact_sign_slow_f32<K>(x, n);
}

// Nearly correctly rounded value (float-float accumulation of exact products).
template <int K>
__device__ __forceinline__ float accurate_value_f32(const float (&x)[K], const int (&n)[K]) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float nk = (float)n[k];
        float p = __fmul_rn(nk, x[k]);
        float pe = __fmaf_rn(nk, x[k], -p);
        float t = __fadd_rn(s, p);
        float bv = __fsub_rn(t, s);
        float av = __fsub_rn(t, bv);
        float err = __fadd_rn(__fsub_rn(s, av), __fsub_rn(p, bv));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, pe));
    }
    return __fadd_rn(s, c);
}

// ---- FP64 inputs, |n_k| < 2^31 -------------------------------------------
template <int K>
__device__ __noinline__ int exact_sign_slow_f64(const double (&x)[K], const int (&n)[K]) {
    double h[2 * K + 1];
    int m = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double nk = (double)n[k];
        double p = __dmul_rn(nk, x[k]);
        double pe = __fma_rn(nk, x[k], -p);
        m = grow_expansion(h, m, pe);
        m = grow_expansion(h, m, p);
    }
    return m == 0 ? 0 : (h[m - 1] > 0.0 ? 1 : -1);
}

template <int K>
__device__ __forceinline__ int exact_sign_f64(const double (&x)[K], const int (&n)[K]) {
    double v = 0.0, A = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double p = __dmul_rn((double)n[k], x[k]);
        v = __dadd_rn(v, p);
        A = __dadd_rn(A, fabs(p));
    }
    if (A == 0.0) return 0;
    double bound = __fma_rn(A, (double)(4 * K + 4) * 0x1p-53, 0x1p-1000);
    if (fabs(v) > bound) return v > 0.0 ? 1 : -1;
    return exact_sign_slow_f64<K>(x, n);
}

template <int K>
__device__ __forceinline__ double accurate_value_f64(const double (&x)[K], const int (&n)[K]) {
    double s = 0.0, c = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double nk = (double)n[k];
        double p = __dmul_rn(nk, x[k]);
        double pe = __fma_rn(nk, x[k], -p);
        double t, err;
        two_sum_d(s, p, t, err);
        s = t;
        c = __dadd_rn(c, __dadd_rn(err, pe));
    }
    return __dadd_rn(s, c);
}

// Exact sign and accurate value together.  The float-float accumulation has
// forward error below 4 K^2 u^2 sum|n_k x_k| (u = 2^-24): every product is
// split exactly, the running sum is kept with TwoSum, and only the small
// correction term is rounded.  With a factor-2 margin this is a filter some
// 10^6 times tighter than plain FP32 evaluation, so the exact expansion runs
// only for true ties (or differences below ~1e-13 of the terms).
template <int K>
__device__ __forceinline__ int sign_value(const float (&x)[K], const int (&n)[K], FF &val) {
    float s = 0.f, c = 0.f, A = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float nk = (float)n[k];
        const float p = __fmul_rn(nk, x[k]);
        const float pe = __fmaf_rn(nk, x[k], -p);
        const float t = __fadd_rn(s, p);
        const float bv = __fsub_rn(t, s);
        const float av = __fsub_rn(t, bv);
        const float err = __fadd_rn(__fsub_rn(s, av), __fsub_rn(p, bv));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, pe));
        A = __fadd_rn(A, fabsf(p));
    }
    val = FF{s, c};
    if (A == 0.f) return 0;
    const float v = __fadd_rn(s, c);
    const float bound = __fmaf_rn(A, (float)(8 * K * K) * 0x1p-48f, 0x1p-126f);
    if (fabsf(v) > bound) return v > 0.f ? 1 : -1;
    return exact_sign_slow_f32<K>(x, n);
}

template <int K>
__device__ __forceinline__ int sign_value(const double (&x)[K], const int (&n)[K], double &val) {
    double s = 0.0, c = 0.0, A = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double nk = (double)n[k];
        const double p = __dmul_rn(nk, x[k]);
        const double pe = __fma_rn(nk, x[k], -p);
        double t, err;
        two_sum_d(s, p, t, err);
        s = t;
        c = __dadd_rn(c, __dadd_rn(err, pe));
        A = __dadd_rn(A, fabs(p));
    }
    val = __dadd_rn(s, c);
    if (A == 0.0) return 0;
    const double bound = __fma_rn(A, (double)(8 * K * K) * 0x1p-106, 0x1p-1000);
    if (fabs(val) > bound) return val > 0.0 ? 1 : -1;
    return exact_sign_slow_f64<K>(x, n);
}

// sign_value with the integer multipliers given as floats (integers below
// 2^24, so exactly representable): the fast path has no integer-to-float
// conversion, and the first product starts the float-float sum (s = p,
// c = its fma error) instead of being added to zero.  Same filter and the
// same exact fallback as sign_value.
template <int K>
__device__ __forceinline__ int sign_value_nf(const float (&x)[K], const float (&nf)[K], FF &val) {
    float s = __fmul_rn(nf[0], x[0]);
    float c = __fmaf_rn(nf[0], x[0], -s);
    float A = fabsf(s);
#pragma unroll
    for (int k = 1; k < K; ++k) {
        const float p = __fmul_rn(nf[k], x[k]);
        const float pe = __fmaf_rn(nf[k], x[k], -p);
        const float t = __fadd_rn(s, p);
        const float bv = __fsub_rn(t, s);
        const float av = __fsub_rn(t, bv);
        const float err = __fadd_rn(__fsub_rn(s, av), __fsub_rn(p, bv));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, pe));
        A = __fadd_rn(A, fabsf(p));
    }
    val = FF{s, c};
    if (A == 0.f) return 0;
    const float v = __fadd_rn(s, c);
    const float bound = __fmaf_rn(A, (float)(8 * K * K) * 0x1p-48f, 0x1p-126f);
    if (fabsf(v) > bound) return v > 0.f ? 1 : -1;
    int n[K];
#pragma unroll
    for (int k = 0; k < K; ++k) n[k] = (int)nf[k];
    return exact_sign_slow_f32<K>(x, n);
}
template <int K>
__device__ __forceinline__ int sign_value_nf(const double (&x)[K], const float (&nf)[K], double &val) {
    int n[K];
#pragma unroll
    for (int k = 0; k < K; ++k) n[k] = (int)nf[k];
    return sign_value<K>(x, n, val);
}

// Dispatch on the input type.
template <int K>
__device__ __forceinline__ int exact_sign(const float (&x)[K], const int (&n)[K]) {
    return exact_sign_f32<K>(x, n);
}
template <int K>
__device__ __forceinline__ int exact_sign(const double (&x)[K], const int (&n)[K]) {
    return exact_sign_f64<K>(x, n);
}
template <int K>
__device__ __forceinline__ FF accurate_value(const float (&x)[K], const int (&n)[K]) {
    // float-float accumulation of the exact products, returned unevaluated
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float nk = (float)n[k];
        float p = __fmul_rn(nk, x[k]);
        float pe = __fmaf_rn(nk, x[k], -p);
        float t = __fadd_rn(s, p);
        float bv = __fsub_rn(t, s);
        float av = __fsub_rn(t, bv);
        float err = __fadd_rn(__fsub_rn(s, av), __fsub_rn(p, bv));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, pe));
    }
    return FF{s, c};
}
template <int K>
__device__ __forceinline__ double accurate_value(const double (&x)[K], const int (&n)[K]) {
    return accurate_value_f64<K>(x, n);
}

}  // namespace adlbr

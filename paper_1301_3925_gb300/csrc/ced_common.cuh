// Pieces of the CED tensor stage shared by its kernels (Sec. 4.4).
#pragma once

#include <cmath>
#include <vector>

#include "internal.cuh"

namespace adlbr {
namespace ced {

constexpr int kMaxR = 32;

// Normalised Gaussian taps, t[k] for |offset| = k; passed by value.
struct Taps {
    float t[kMaxR + 1];
};

// Standard deviation s -> truncation radius int(3 s + 0.5).
inline int radius_of(double s) { return (int)(3.0 * s + 0.5); }

inline Taps make_taps(double s) {
    Taps tp = {};
    int r = radius_of(s);
    std::vector<double> t(r + 1);
    double sum = 0.0;
    for (int k = 0; k <= r; ++k) {
        t[k] = std::exp(-0.5 * (double)k * k / (s * s));
        sum += (k == 0 ? 1.0 : 2.0) * t[k];
    }
    for (int k = 0; k <= r; ++k) tp.t[k] = (float)(t[k] / sum);
    return tp;
}

// Half-sample symmetric reflection about the border: u(-1) = u(0).
__device__ __forceinline__ int reflect(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;
    const int p = 2 * n;
    i %= p;
    if (i < 0) i += p;
    return i < n ? i : p - 1 - i;
}

// D(J) for J = [[p, q], [q, s]]: eigenvectors of J, lambda1 = alpha on v1
// (eigenvalue mu1 >= mu2), lambda2 = alpha + (1 - alpha) exp(-C / (mu1 -
// mu2)^2) on v2; written with (mu1 - mu2)^2 = d2 = (p - s)^2 + 4 q^2 and
// v1 v1^T = (I + [[cos 2t, sin 2t], [sin 2t, -cos 2t]]) / 2, cos 2t and
// sin 2t taken with one reciprocal square root of d2.  Where C / d2 > 87,
// exp(-C / d2) is below 2^-125 and lambda2 rounds to alpha in FP32: D = alpha I
// there, as for d2 = 0.  The same instructions in every kernel, so all of
// them compute bit-identical values.
__device__ __forceinline__ void d_from_j(float p, float q, float s, float alpha, float C,
                                         float &Dxx, float &Dxy, float &Dyy) {
    const float dps = __fsub_rn(p, s);
    const float d2 = __fmaf_rn(dps, dps, __fmul_rn(4.f, __fmul_rn(q, q)));
    Dxx = alpha;
    Dxy = 0.f;
    Dyy = alpha;
    if (d2 > 0.f && C < __fmul_rn(87.f, d2)) {
        const float rd = rsqrtf(d2);
        const float lam2 = __fmaf_rn(__fsub_rn(1.f, alpha), __expf(__fmul_rn(-C, __fmul_rn(rd, rd))), alpha);
        const float c2 = __fmul_rn(dps, rd), s2 = __fmul_rn(__fmul_rn(2.f, q), rd);
        const float m = __fmul_rn(0.5f, __fadd_rn(alpha, lam2));
        const float h = __fmul_rn(0.5f, __fsub_rn(alpha, lam2));
        Dxx = __fmaf_rn(h, c2, m);
        Dxy = __fmul_rn(h, s2);
        Dyy = __fmaf_rn(-h, c2, m);
    }
}

}  // namespace ced
}  // namespace adlbr

// The 2D AD-LBR stencil of one grid point (device function shared by the
// stand-alone build kernel and the fused CED tensor + build kernel).
//
// Sec. 2 of the paper: (i) an M(z)-reduced basis (e, f) by Lagrange's
// algorithm (Eq. GaussAlgo), (ii) f negated if <e, M f> > 0, (iii) the
// M-obtuse superbase (e, f, -e-f) (Corollary
// ObtuseSuperBaseFromReducedBasis2), stencil Eq. def:Vz and weights
// Eq. def:GammaZ.  M is a positive multiple of S = adj(D) (Eqs. def:M,
// eq:DM), and <e^perp, D f^perp> = <e, S f>.
//
// GPU design: the reduction loop runs in FP32 on a rescaled S (cheap, a few
// iterations); its output is then CERTIFIED: the three products
// <e_i, S e_j> of the superbase are signed exactly (exact.cuh) against the
// input D, and while one of them is positive a Selling step
// (e_i, e_j, e_k) -> (-e_i, e_j, e_i - e_j) (which lowers sum |e|_S^2 by
// 4 <e_i, S e_j>) repairs it.  The result is an exactly S-obtuse superbase;
// by Lemma indepBasis its positive-weight stencil is unique, so the offsets
// agree bit for bit with any other exact construction.
#pragma once

#include "exact.cuh"
#include "internal.cuh"
#include "store.cuh"

namespace adlbr {
namespace s2d {

// Integer vector held in floats: coordinates up to kMaxCoord, so every
// coordinate and every product below is an exact integer in FP32.
struct V2 {
    float x, y;
};

// <u, adj(D) v> = c ux vx - b (ux vy + uy vx) + a uy vy, terms (x_k, n_k)
// with the integers n_k as exact floats (|n_k| <= 2 * 2047^2 < 2^24).
template <typename T>
__device__ __forceinline__ void terms2(T a, T b, T c, V2 u, V2 v, T (&x)[3], float (&n)[3]) {
    x[0] = c;
    n[0] = __fmul_rn(u.x, v.x);
    x[1] = b;
    n[1] = -__fmaf_rn(u.x, v.y, __fmul_rn(u.y, v.x));
    x[2] = a;
    n[2] = __fmul_rn(u.y, v.y);
}

static __device__ __noinline__ bool det_positive_slow(float a, float b, float c) {
    // a c and b^2 are exact in FP64; the rounded difference keeps the sign
    return __dsub_rn(__dmul_rn((double)a, (double)c), __dmul_rn((double)b, (double)b)) > 0.0;
}
__device__ __forceinline__ bool det_positive(float a, float b, float c) {
    // a c - b^2 = (p1 + e1) - (p2 + e2) exactly (fma splits); FP32 filter first
    const float p1 = __fmul_rn(a, c), e1 = __fmaf_rn(a, c, -p1);
    const float p2 = __fmul_rn(b, b), e2 = __fmaf_rn(b, b, -p2);
    const float v = __fadd_rn(__fsub_rn(p1, p2), __fsub_rn(e1, e2));
    const float bound = __fmul_rn(__fadd_rn(fabsf(p1), fabsf(p2)), 0x1p-20f);
    if (fabsf(v) > bound) return v > 0.f;
    return det_positive_slow(a, b, c);
}
__device__ __forceinline__ bool det_positive(double a, double b, double c) {
    double p = __dmul_rn(a, c), pe = __fma_rn(a, c, -p);
    double q = __dmul_rn(-b, b), qe = __fma_rn(-b, b, -q);
    double h[5];
    int m = 0;
    m = grow_expansion(h, m, pe);
    m = grow_expansion(h, m, p);
    m = grow_expansion(h, m, qe);
    m = grow_expansion(h, m, q);
    return m > 0 && h[m - 1] > 0.0;
}

__device__ __forceinline__ bool finite(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// S = adj(D) / max(a, c) in FP32 (approximately: one reciprocal), for the
// approximate reduction loop.
__device__ __forceinline__ void scaled_adj(float a, float b, float c, float &sxx, float &sxy,
                                           float &syy) {
    const float m = __frcp_rn(fmaxf(a, c));
    sxx = c * m;
    sxy = -b * m;
    syy = a * m;
}
__device__ __forceinline__ void scaled_adj(double a, double b, double c, float &sxx, float &sxy,
                                           float &syy) {
    const double m = fmax(a, c);
    sxx = (float)(c / m);
    sxy = (float)(-b / m);
    syy = (float)(a / m);
}

// <u, S v> for integer-valued float vectors (exact coordinates below 2^24).
__device__ __forceinline__ float gramf(float sxx, float sxy, float syy, float ux, float uy, float vx,
                                       float vy) {
    return sxx * ux * vx + sxy * (ux * vy + uy * vx) + syy * uy * vy;
}

constexpr int kMaxReduce = 64;
constexpr int kMaxFix = 256;
// repair budget of a warm start (below): past it, the point is built cold.
// None: a stencil that no longer fits D is rebuilt from scratch (build and
// step at 4096^2: 0.4105 ms; 0.4111 with one repair, 0.4129 with two, 0.415
// with four)
constexpr int kWarmFix = 0;
// |coordinates| <= 2047 keeps every integer of the predicates below 2^24
constexpr int kMaxCoord = 2047;

}  // namespace s2d

// What build_point2d stored for a point: its offsets and, for F16 weights,
// its weight record (zeros for the other weight formats).
struct Built2 {
    short4 o;
    uint2 rec;
};

// Builds and stores the stencil of point i from D = [[a, b], [b, c]].
//
// warm: offs[i] holds this point's stencil from an earlier build of the
// same handle (the previous step of a CED loop, where D moves little).  Its
// superbase (e, f, -e-f), if it is one (|det(e, f)| = 1, coordinates in
// range), is certified like the reduced basis below (with kWarmFix repairs
// at most); the reduction runs only where that fails.  A
// certified S-obtuse superbase gives the unique stencil of Lemma indepBasis,
// so the result is the cold build's (the three vectors may come in another
// order or sign, which the canonical export removes).
template <typename T>
__device__ __forceinline__ Built2 build_point2d(T a, T b, T c, int64_t i, short4 *__restrict__ offs,
                                                void *wbase, adlbr_dtype wt, int *err, bool warm = false) {
    using namespace s2d;
    using WV = typename WVal<T>::type;
    // the previous stencil is read first, so that its load overlaps the
    // tensor's and the tests below
    const short4 p = warm ? offs[i] : make_short4(0, 0, 0, 0);
    WV wz[3] = {};
    int code = 0;
    if (!finite(a) || !finite(b) || !finite(c)) {
        code = ERRBIT_NONFINITE;
    } else if (!(a > (T)0) || !(c > (T)0) || !det_positive(a, b, c)) {
        code = ERRBIT_NOT_SPD;
    }
    if (code) {
        offs[i] = make_short4(0, 0, 0, 0);
        const uint4 r = store_weights<3>(wbase, wt, i, wz, 7u);
        atomicOr(err, code);
        return Built2{make_short4(0, 0, 0, 0), make_uint2(r.x, r.y)};
    }

    V2 v[3];
    int sg[3];
    WV val[3];
    // (iii) below: certify the superbase v with exact signs and repair it by
    // Selling steps, at most `budget` of them
    auto certify = [&](int budget) {
        for (int fix = 0;; ++fix) {
            int bad = -1;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                T x[3];
                float n[3];
                terms2(a, b, c, v[(k + 1) % 3], v[(k + 2) % 3], x, n);
                sg[k] = sign_value_nf<3>(x, n, val[k]);
                if (sg[k] > 0 && bad < 0) bad = k;
            }
            if (bad < 0) return true;
            if (fix == budget) return false;
            // pair (j, l) = (bad+1, bad+2) is acute: (v_j, v_l, v_bad) -> (-v_j, v_l, v_j - v_l)
            const int j = (bad + 1) % 3, l = (bad + 2) % 3;
            V2 vj = v[j], vl = v[l];
            v[j] = V2{-vj.x, -vj.y};
            v[bad] = V2{vj.x - vl.x, vj.y - vl.y};
            if (fabsf(v[bad].x) > (float)kMaxCoord || fabsf(v[bad].y) > (float)kMaxCoord) return false;
        }
    };
    bool ok = false;
    if (warm) {
        const int det = (int)p.x * p.w - (int)p.y * p.z;
        const int tx = -(int)p.x - p.z, ty = -(int)p.y - p.w;
        if ((det == 1 || det == -1) && abs(tx) <= kMaxCoord && abs(ty) <= kMaxCoord) {
            v[0] = V2{(float)p.x, (float)p.y};
            v[1] = V2{(float)p.z, (float)p.w};
            v[2] = V2{(float)tx, (float)ty};
            ok = certify(kWarmFix);
        }
    }
    if (!ok) {
        // (i) approximate Lagrange reduction in FP32 on S / max(a, c): the basis
        // vectors are kept as integer-valued floats, |f|_S^2 is carried over to
        // the next |e|_S^2, and the quotient is approximate (the result is
        // certified exactly below, so these shortcuts can only cost repair steps)
        float sxx, sxy, syy;
        scaled_adj(a, b, c, sxx, sxy, syy);
        // The Gram values of the running basis are updated, not recomputed:
        // f' = e - q f gives |f'|^2 = |e|^2 - q (2 <e,f> - q |f|^2) and
        // <f, f'> = <e,f> - q |f|^2.
        float ex = 1.f, ey = 0.f, fx = 0.f, fy = 1.f;
        float gee = sxx, gef = sxy, gff = syy;   // Gram values of e = (1, 0), f = (0, 1)
        for (int it = 0; it < kMaxReduce; ++it) {
            if (!(gff > 0.f)) break;
            const float q = fminf(fmaxf(rintf(__fdividef(gef, gff)), -2048.f), 2048.f);
            const float nx = fmaf(-q, fx, ex), ny = fmaf(-q, fy, ey);   // exact: integers below 2^24
            if (fabsf(nx) > (float)kMaxCoord || fabsf(ny) > (float)kMaxCoord) {
                ex = fx, ey = fy, fx = nx, fy = ny;
                break;
            }
            const float gnn = fmaf(-q, fmaf(-q, gff, 2.f * gef), gee);
            const float gfn = fmaf(-q, gff, gef);
            const bool shorter = gff > gnn;
            ex = fx, ey = fy, fx = nx, fy = ny;
            gee = gff, gef = gfn, gff = gnn;
            if (!shorter) break;
        }
        // (ii) orientation of f
        if (gef > 0.f) fx = -fx, fy = -fy;

        // (iii) superbase, certified and repaired with exact signs
        v[0] = V2{ex, ey};
        v[1] = V2{fx, fy};
        v[2] = V2{-ex - fx, -ey - fy};
        ok = certify(kMaxFix - 1);
    }
    bool range = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) range |= fabsf(v[k].x) > (float)kMaxCoord || fabsf(v[k].y) > (float)kMaxCoord;
    if (!ok || range) {
        offs[i] = make_short4(0, 0, 0, 0);
        const uint4 r = store_weights<3>(wbase, wt, i, wz, 7u);
        atomicOr(err, range ? ERRBIT_RANGE : ERRBIT_NOT_CONVERGED);
        return Built2{make_short4(0, 0, 0, 0), make_uint2(r.x, r.y)};
    }

    // weights gamma(+-e_k) = -<e_{k+1}, S e_{k+2}> / 2
    unsigned zmask = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (sg[k] == 0) {
            zmask |= 1u << k;
            wz[k] = WV{};
        } else {
            wz[k] = wmax0(neg_half(val[k]));
        }
    }
    if constexpr (kBoundsCheck) {
        // Remark "Stencil radius": every offset of non-zero weight has
        // |e| <= max(kappa(D), sqrt 2), i.e. |e|^2 det(D) <= max(2 det(D),
        // lambda_max(D)^2) (FP64, with a relative margin for the rounding of
        // det and lambda_max).  Below kappa = sqrt 2 the third superbase
        // vector, of length sqrt 2, can carry a small positive weight.
        const double da = (double)a, db = (double)b, dc = (double)c;
        const double det = fma(da, dc, -db * db);
        const double lmax = 0.5 * (da + dc + sqrt((da - dc) * (da - dc) + 4.0 * db * db));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double r2 = (double)v[k].x * v[k].x + (double)v[k].y * v[k].y;
            if (!(zmask >> k & 1u) && r2 * det > fmax(2.0 * det, lmax * lmax) * (1.0 + 1e-6))
                atomicOr(err, ERRBIT_BOUNDS);
        }
    }
    const short4 o = make_short4((short)(int)v[0].x, (short)(int)v[0].y, (short)(int)v[1].x, (short)(int)v[1].y);
    offs[i] = o;
    const uint4 r = store_weights<3>(wbase, wt, i, wz, zmask);
    return Built2{o, make_uint2(r.x, r.y)};
}

}  // namespace adlbr

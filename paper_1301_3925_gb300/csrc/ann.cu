// The axes-directed non-negative six-point scheme A-NN of Sec. 4.1 (Remark
// rem:WG), the paper's comparison scheme: one thread per grid point.
//
// For D = [[a, b], [b, c]]: b = 0 gives the four-point stencil
// {(+-1, 0), (0, +-1)}, 2 gamma = a, c; otherwise the stencil is
// {(+-1, 0), (0, +-1), +-(p, q)} with p, q non-zero, b p q >= 0,
// |b| / c <= |p / q| <= a / |b| (Eq. ineqPQ) and max(|p|, |q|) minimal, and
//   2 gamma(+-1, 0) = a - (p/q) b = (|q| a - |p| |b|) / |q|,
//   2 gamma(0, +-1) = c - (q/p) b = (|p| c - |q| |b|) / |p|,
//   2 gamma(+-(p, q)) = b / (p q) = |b| / (|p| |q|).
// The interval [|b|/c, a/|b|] is non-empty (a c > b^2).  Among its fractions
// the one of smallest denominator also has the smallest numerator (Stern-
// Brocot tree), so it is the unique minimiser of max(|p|, |q|).  It is found
// by descending the Stern-Brocot tree from 0/1 and 1/0, one continued-fraction
// run per step: the run length is estimated in floating point and then
// corrected, and every comparison of a fraction with an endpoint is the exact
// sign of |p| c - |q| |b| or |q| a - |p| |b| (exact.cuh), so the result does
// not depend on rounding.
//
// Storage: the offsets (1, 0), (0, 1) in the handle's short4 plane and the
// third offset (p, q) (sign of q = sign of b; (0, 0) when b = 0) in offs3.
#include "stencil2d.cuh"

namespace adlbr {

namespace {

constexpr int kMaxPQ = 2047;   // the 2D storage range

// sign(p/q - |b|/c) = sign(p c - q |b|) and sign(a/|b| - p/q) = sign(q a - p |b|)
// for p, q >= 0 and sb = sign(b)
template <typename T>
__device__ __forceinline__ int cmp_lo(T b, T c, int sb, int p, int q) {
    const T x[2] = {c, b};
    const int n[2] = {p, -q * sb};
    return exact_sign<2>(x, n);
}
template <typename T>
__device__ __forceinline__ int cmp_hi(T a, T b, int sb, int p, int q) {
    const T x[2] = {a, b};
    const int n[2] = {q, -p * sb};
    return exact_sign<2>(x, n);
}

// The simplest fraction p/q (p, q >= 1) of [|b|/c, a/|b|]; false if it
// needs a coordinate above kMaxPQ.
template <typename T>
__device__ __forceinline__ bool simplest_fraction(T a, T b, T c, int sb, int &p, int &q) {
    const double ab = fabs((double)b);
    const double lo = ab / (double)c, hi = (double)a / ab;
    int pl = 0, ql = 1, pr = 1, qr = 0;   // left 0/1 below, right 1/0 above the interval
    for (int it = 0; it < 128; ++it) {
        const int pm = pl + pr, qm = ql + qr;
        if (pm > kMaxPQ || qm > kMaxPQ) return false;
        if (cmp_lo(b, c, sb, pm, qm) < 0) {
            // the mediant lies below: the left end moves k steps towards the
            // right one, k the largest with (pl + k pr) / (ql + k qr) < |b|/c
            const double den = pr - lo * qr;
            double t = den > 0.0 ? (lo * ql - pl) / den : (double)kMaxPQ;
            int k = (int)fmin(fmax(floor(t), 1.0), (double)kMaxPQ);
            while (k > 1 && !(cmp_lo(b, c, sb, pl + k * pr, ql + k * qr) < 0)) --k;
            while (pl + (k + 1) * pr <= kMaxPQ && ql + (k + 1) * qr <= kMaxPQ &&
                   cmp_lo(b, c, sb, pl + (k + 1) * pr, ql + (k + 1) * qr) < 0)
                ++k;
            pl += k * pr;
            ql += k * qr;
        } else if (cmp_hi(a, b, sb, pm, qm) < 0) {
            // above: the right end moves k steps towards the left one, k the
            // largest with (pr + k pl) / (qr + k ql) > a/|b|
            const double den = hi * ql - pl;
            double t = den > 0.0 ? (pr - hi * qr) / den : (double)kMaxPQ;
            int k = (int)fmin(fmax(floor(t), 1.0), (double)kMaxPQ);
            while (k > 1 && !(cmp_hi(a, b, sb, pr + k * pl, qr + k * ql) < 0)) --k;
            while (pr + (k + 1) * pl <= kMaxPQ && qr + (k + 1) * ql <= kMaxPQ &&
                   cmp_hi(a, b, sb, pr + (k + 1) * pl, qr + (k + 1) * ql) < 0)
                ++k;
            pr += k * pl;
            qr += k * ql;
        } else {
            p = pm;
            q = qm;
            return true;
        }
    }
    return false;
}

template <typename T>
__device__ __forceinline__ typename WVal<T>::type div_int(typename WVal<T>::type v, int d);
template <> __device__ __forceinline__ FF div_int<float>(FF v, int d) {
    return FF{__fdiv_rn(to_f(v), (float)d), 0.f};
}
template <> __device__ __forceinline__ double div_int<double>(double v, int d) { return v / (double)d; }

template <typename T>
__global__ void __launch_bounds__(256) build_ann2d_kernel(int64_t N, const T *__restrict__ D,
                                                          short4 *__restrict__ offs, short2 *__restrict__ offs3,
                                                          void *wbase, adlbr_dtype wt, int *err) {
    using namespace s2d;
    using WV = typename WVal<T>::type;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T a = D[i], b = D[N + i], c = D[2 * N + i];
    WV wz[3] = {};
    int code = 0;
    if (!finite(a) || !finite(b) || !finite(c)) {
        code = ERRBIT_NONFINITE;
    } else if (!(a > (T)0) || !(c > (T)0) || !det_positive(a, b, c)) {
        code = ERRBIT_NOT_SPD;
    }
    int p = 0, q = 0;
    const int sb = b > (T)0 ? 1 : (b < (T)0 ? -1 : 0);
    if (!code && sb != 0 && !simplest_fraction(a, b, c, sb, p, q)) code = ERRBIT_RANGE;
    if (code) {
        offs[i] = make_short4(0, 0, 0, 0);
        offs3[i] = make_short2(0, 0);
        store_weights<3>(wbase, wt, i, wz, 7u);
        atomicOr(err, code);
        return;
    }
    unsigned zmask = 0;
    if (sb == 0) {
        // the four-point stencil: 2 gamma(+-1, 0) = a, 2 gamma(0, +-1) = c
        const T ax[1] = {a}, cx[1] = {c};
        const int one[1] = {1};
        wz[0] = div_int<T>(accurate_value<1>(ax, one), 2);
        wz[1] = div_int<T>(accurate_value<1>(cx, one), 2);
        zmask = 4u;
        offs3[i] = make_short2(0, 0);
    } else {
        // 2 gamma(1, 0) = (q a - p |b|) / q and 2 gamma(0, 1) = (p c - q |b|) / p,
        // both >= 0 by the choice of p / q (zero exactly at an interval end)
        const T xh[2] = {a, b}, xl[2] = {c, b};
        const int nh[2] = {q, -p * sb}, nl[2] = {p, -q * sb};
        WV vh, vl;
        const int sh = sign_value<2>(xh, nh, vh), sl = sign_value<2>(xl, nl, vl);
        if (sh == 0) zmask |= 1u;
        else wz[0] = wmax0(div_int<T>(vh, 2 * q));
        if (sl == 0) zmask |= 2u;
        else wz[1] = wmax0(div_int<T>(vl, 2 * p));
        // 2 gamma(p, q) = |b| / (p q)
        const T bx[1] = {b};
        const int nb[1] = {sb};
        wz[2] = div_int<T>(accurate_value<1>(bx, nb), 2 * p * q);
        offs3[i] = make_short2((short)p, (short)(q * sb));
    }
    offs[i] = make_short4(1, 0, 0, 1);
    store_weights<3>(wbase, wt, i, wz, zmask);
}

}  // namespace

adlbr_status launch_build_ann2d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st) {
    ADLBR_NVTX("build");
    stencils_changed(s);
    if (s->dim != 2 || !s->offs3) return fail(ADLBR_E_INTERNAL, "A-NN build on a handle without a third-offset plane");
    const int threads = 256;
    const unsigned blocks = blocks_for(s->N, threads);
    if (D_t == ADLBR_F32)
        build_ann2d_kernel<float><<<blocks, threads, 0, st>>>(s->N, (const float *)D, (short4 *)s->offs,
                                                              (short2 *)s->offs3, s->w, s->w_t, s->err);
    else
        build_ann2d_kernel<double><<<blocks, threads, 0, st>>>(s->N, (const double *)D, (short4 *)s->offs,
                                                               (short2 *)s->offs3, s->w, s->w_t, s->err);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace adlbr

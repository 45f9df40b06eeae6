// 2D AD-LBR stencil construction, one thread per grid point.
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
#include "exact.cuh"
#include "internal.cuh"
#include "store.cuh"

namespace adlbr {

namespace {

struct V2 {
    int x, y;
};

__device__ __forceinline__ float gram2(float sxx, float sxy, float syy, V2 u, V2 v) {
    float ux = (float)u.x, uy = (float)u.y, vx = (float)v.x, vy = (float)v.y;
    return sxx * ux * vx + sxy * (ux * vy + uy * vx) + syy * uy * vy;
}

// <u, adj(D) v> = c ux vx - b (ux vy + uy vx) + a uy vy, terms (x_k, n_k).
template <typename T>
__device__ __forceinline__ void terms2(T a, T b, T c, V2 u, V2 v, T (&x)[3], int (&n)[3]) {
    x[0] = c;
    n[0] = u.x * v.x;
    x[1] = b;
    n[1] = -(u.x * v.y + u.y * v.x);
    x[2] = a;
    n[2] = u.y * v.y;
}

template <typename T>
__device__ __forceinline__ int sgnS(T a, T b, T c, V2 u, V2 v) {
    T x[3];
    int n[3];
    terms2(a, b, c, u, v, x, n);
    return exact_sign<3>(x, n);
}

__device__ __forceinline__ bool det_positive(float a, float b, float c) {
    // a c and b^2 are exact in FP64; the rounded difference keeps the sign
    return __dsub_rn(__dmul_rn((double)a, (double)c), __dmul_rn((double)b, (double)b)) > 0.0;
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

constexpr int kMaxReduce = 64;
constexpr int kMaxFix = 256;
// |coordinates| <= 2047 keeps every integer of the predicates below 2^24
constexpr int kMaxCoord = 2047;

template <typename T>
__global__ void __launch_bounds__(256) build2d_kernel(int64_t N, const T *__restrict__ D,
                                                      short4 *__restrict__ offs, void *wbase,
                                                      adlbr_dtype wt, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T a = D[i], b = D[N + i], c = D[2 * N + i];
    double wz[3] = {0.0, 0.0, 0.0};
    int code = 0;
    if (!finite(a) || !finite(b) || !finite(c)) {
        code = ERRBIT_NONFINITE;
    } else if (!(a > (T)0) || !(c > (T)0) || !det_positive(a, b, c)) {
        code = ERRBIT_NOT_SPD;
    }
    if (code) {
        offs[i] = make_short4(0, 0, 0, 0);
        store_weights<3>(wbase, wt, i, wz, 7u);
        atomicOr(err, code);
        return;
    }

    // (i) approximate Lagrange reduction in FP32 on S / max(a, c)
    const double scl = 1.0 / fmax((double)a, (double)c);
    const float sxx = (float)((double)c * scl), sxy = (float)(-(double)b * scl),
                syy = (float)((double)a * scl);
    V2 e{1, 0}, f{0, 1};
    for (int it = 0; it < kMaxReduce; ++it) {
        float den = gram2(sxx, sxy, syy, f, f);
        if (!(den > 0.f)) break;
        float r = rintf(gram2(sxx, sxy, syy, e, f) / den);
        r = fminf(fmaxf(r, -2048.f), 2048.f);
        int q = (int)r;
        V2 nf{e.x - q * f.x, e.y - q * f.y};
        e = f;
        f = nf;
        if (abs(f.x) > kMaxCoord || abs(f.y) > kMaxCoord) break;
        if (!(gram2(sxx, sxy, syy, e, e) > gram2(sxx, sxy, syy, f, f))) break;
    }
    // (ii) orientation of f
    if (gram2(sxx, sxy, syy, e, f) > 0.f) f = V2{-f.x, -f.y};

    // (iii) superbase, certified and repaired with exact signs
    V2 v[3] = {e, f, V2{-e.x - f.x, -e.y - f.y}};
    int sg[3];
    bool ok = false;
    for (int fix = 0; fix < kMaxFix; ++fix) {
        int bad = -1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sg[k] = sgnS(a, b, c, v[(k + 1) % 3], v[(k + 2) % 3]);
            if (sg[k] > 0 && bad < 0) bad = k;
        }
        if (bad < 0) {
            ok = true;
            break;
        }
        // pair (j, l) = (bad+1, bad+2) is acute: (v_j, v_l, v_bad) -> (-v_j, v_l, v_j - v_l)
        const int j = (bad + 1) % 3, l = (bad + 2) % 3;
        V2 vj = v[j], vl = v[l];
        v[j] = V2{-vj.x, -vj.y};
        v[bad] = V2{vj.x - vl.x, vj.y - vl.y};
        if (abs(v[bad].x) > kMaxCoord || abs(v[bad].y) > kMaxCoord) break;
    }
    bool range = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) range |= abs(v[k].x) > kMaxCoord || abs(v[k].y) > kMaxCoord;
    if (!ok || range) {
        offs[i] = make_short4(0, 0, 0, 0);
        store_weights<3>(wbase, wt, i, wz, 7u);
        atomicOr(err, range ? ERRBIT_RANGE : ERRBIT_NOT_CONVERGED);
        return;
    }

    // weights gamma(+-e_k) = -<e_{k+1}, S e_{k+2}> / 2
    unsigned zmask = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (sg[k] == 0) {
            zmask |= 1u << k;
            wz[k] = 0.0;
        } else {
            T x[3];
            int n[3];
            terms2(a, b, c, v[(k + 1) % 3], v[(k + 2) % 3], x, n);
            wz[k] = fmax(-0.5 * accurate_value<3>(x, n), 0.0);
        }
    }
    offs[i] = make_short4((short)v[0].x, (short)v[0].y, (short)v[1].x, (short)v[1].y);
    store_weights<3>(wbase, wt, i, wz, zmask);
}

}  // namespace

adlbr_status launch_build2d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st) {
    const int threads = 256;
    unsigned blocks = blocks_for(s->N, threads);
    if (D_t == ADLBR_F32)
        build2d_kernel<float><<<blocks, threads, 0, st>>>(s->N, (const float *)D, (short4 *)s->offs,
                                                          s->w, s->w_t, s->err);
    else
        build2d_kernel<double><<<blocks, threads, 0, st>>>(s->N, (const double *)D,
                                                           (short4 *)s->offs, s->w, s->w_t, s->err);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace adlbr

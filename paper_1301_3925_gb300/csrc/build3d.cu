// 3D AD-LBR stencil construction, one thread per grid point.
//
// Sec. 2 of the paper: a D-reduced basis (Def. ReducedBasis, obtained with
// the greedy extension of Lagrange's algorithm to d = 3 that the paper
// cites), Prop. MakeObtuse (Eqs. SignedOrderedIneq, 3DSuperBase) for a
// D-obtuse superbase (e0, e1, e2, e3), and Selling's stencil (Lemma Selling,
// Eq. DSum3D): offsets e_k x e_l with weights -<e_i, D e_j>/2.
//
// GPU design, as in 2D: the reduction and MakeObtuse run in FP32 on a
// rescaled D, in Gram-matrix form (integer vectors, FP32 Gram values updated
// with them); the resulting superbase is certified with exact signs of the
// six products <e_i, D e_j> (exact.cuh) and repaired, while a product is
// positive, by Selling steps (e_i, e_j, e_k, e_l) -> (-e_i, e_j, e_k + e_i,
// e_l + e_i), each lowering sum |e|_D^2 by 2 <e_i, D e_j>.  The certified
// superbase is exactly D-obtuse.
#include "exact.cuh"
#include "internal.cuh"
#include "store.cuh"

namespace adlbr {

namespace {

// Integer vector held in floats: every coordinate (at most 4 * 127 during
// the reduction) and every product below is an exact integer in FP32, so
// the vector arithmetic is exact and needs no integer-to-float conversions.
struct V3 {
    float x, y, z;
};

__device__ __forceinline__ V3 add(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 neg(V3 a) { return V3{-a.x, -a.y, -a.z}; }
// a - k b (exact: integers below 2^24)
__device__ __forceinline__ V3 sub_mul(V3 a, float k, V3 b) {
    return V3{__fmaf_rn(-k, b.x, a.x), __fmaf_rn(-k, b.y, a.y), __fmaf_rn(-k, b.z, a.z)};
}
__device__ __forceinline__ float amax(V3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }

// d = (xx, yy, zz, xy, xz, yz)
__device__ __forceinline__ float g3(const float (&d)[6], V3 u, V3 v) {
    const float ux = u.x, uy = u.y, uz = u.z, vx = v.x, vy = v.y, vz = v.z;
    return d[0] * ux * vx + d[1] * uy * vy + d[2] * uz * vz + d[3] * (ux * vy + uy * vx) +
           d[4] * (ux * vz + uz * vx) + d[5] * (uy * vz + uz * vy);
}

// <u, D v> = sum_k n_k D_k with the integers n_k as exact floats
// (|n_k| <= 2 * 127^2)
template <typename T>
__device__ __forceinline__ void terms3(const T (&D)[6], V3 u, V3 v, T (&x)[6], float (&n)[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) x[k] = D[k];
    n[0] = __fmul_rn(u.x, v.x);
    n[1] = __fmul_rn(u.y, v.y);
    n[2] = __fmul_rn(u.z, v.z);
    n[3] = __fmaf_rn(u.x, v.y, __fmul_rn(u.y, v.x));
    n[4] = __fmaf_rn(u.x, v.z, __fmul_rn(u.z, v.x));
    n[5] = __fmaf_rn(u.y, v.z, __fmul_rn(u.z, v.y));
}

__device__ __forceinline__ bool finite(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

constexpr int kMaxCoord = 127;

// D is accepted when its leading principal minors are positive with relative
// margins: a, b, c > 0, ab - xy^2 > 1e-14 ab, det D > 1e-13 abc (FP64).
__device__ __forceinline__ bool spd64(double a, double b, double c, double xy, double xz, double yz) {
    const double m2 = a * b - xy * xy;
    const double det = a * (b * c - yz * yz) - xy * (xy * c - yz * xz) + xz * (xy * yz - b * xz);
    return a > 0.0 && b > 0.0 && c > 0.0 && m2 > 1e-14 * a * b && det > 1e-13 * a * b * c;
}
__device__ __forceinline__ bool spd3(const double (&D)[6]) { return spd64(D[0], D[1], D[2], D[3], D[4], D[5]); }

// FP32 input: the minors are first evaluated in FP32 with bounds on their
// rounding errors, |m2 - exact| <= 2^-21 s2 and |det - exact| <= 2^-19 s3 (8
// and 32 unit roundoffs of the sums of absolute terms s2, s3; valid while no
// product is subnormal or infinite).  A clear pass, each minor above twice its
// margin by more than its bound, is also a pass of the FP64 test; every other
// case is decided by the FP64 test.  (Evaluated for every point, the FP64
// test kept the narrow FP64 pipe 40% busy in the 256^3 build.)
__device__ __forceinline__ bool spd3(const float (&D)[6]) {
    const float a = D[0], b = D[1], c = D[2], xy = D[3], xz = D[4], yz = D[5];
    if (a > 0.f && b > 0.f && c > 0.f) {
        const float ab = a * b, xx = xy * xy, m2 = ab - xx, s2 = ab + xx;
        const float bc = b * c, yy = yz * yz;
        const float det = a * (bc - yy) - xy * (xy * c - yz * xz) + xz * (xy * yz - b * xz);
        const float s3 = a * (bc + yy) + fabsf(xy) * (fabsf(xy * c) + fabsf(yz * xz)) +
                         fabsf(xz) * (fabsf(xy * yz) + fabsf(b * xz));
        const float abc = ab * c;
        if (s2 > 1e-30f && abc > 1e-30f && s3 < 1e37f && m2 - 0x1p-21f * s2 > 2e-14f * ab &&
            det - 0x1p-19f * s3 > 2e-13f * abc)
            return true;
    }
    return spd64(a, b, c, xy, xz, yz);
}

// The Gram matrix of the basis b for the FP32 form d: G[i][j] = <b_i, d b_j>.
__device__ __forceinline__ void gram3(const float (&d)[6], const V3 (&b)[3], float (&G)[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            G[i][j] = g3(d, b[i], b[j]);
            G[j][i] = G[i][j];
        }
}

template <typename T>
__global__ void __launch_bounds__(128) build3d_kernel(int64_t N, const T *__restrict__ Dp,
                                                      char4 *__restrict__ offs, void *wbase,
                                                      adlbr_dtype wt, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T D[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) D[k] = Dp[(int64_t)k * N + i];
    using WV = typename WVal<T>::type;
    WV wz[6] = {};

    int code = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (!finite(D[k])) code = ERRBIT_NONFINITE;
    if (!code && !spd3(D)) code = ERRBIT_NOT_SPD;
    char4 *o = offs + 3 * i;
    if (code) {
        o[0] = o[1] = o[2] = make_char4(0, 0, 0, 0);
        store_weights<6>(wbase, wt, i, wz, 63u);
        atomicOr(err, code);
        return;
    }

    // ---- approximate greedy reduction (FP32) ----
    const T dmax = D[0] > D[1] ? (D[0] > D[2] ? D[0] : D[2]) : (D[1] > D[2] ? D[1] : D[2]);
    float d[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) d[k] = (float)(D[k] / dmax);
    // The basis vectors are exact integers; their Gram values are carried in
    // FP32 and updated with the vectors (f' = e - q f changes |f|^2 and the
    // products with the third vector linearly), and recomputed from the
    // vectors once per round.  The result is certified exactly below, so the
    // rounding of these values can only cost repair steps.
    V3 b[3] = {V3{1.f, 0.f, 0.f}, V3{0.f, 1.f, 0.f}, V3{0.f, 0.f, 1.f}};
    for (int it = 0; it < 24; ++it) {
        float G[3][3];
        gram3(d, b, G);
        // sort by norm (G follows the permutation)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2 - p; ++q)
                if (G[q + 1][q + 1] < G[q][q]) {
                    const int r = 3 - q - (q + 1);   // the third index
                    V3 tv = b[q];
                    b[q] = b[q + 1];
                    b[q + 1] = tv;
                    float t = G[q][q];
                    G[q][q] = G[q + 1][q + 1];
                    G[q + 1][q + 1] = t;
                    t = G[q][r];
                    G[q][r] = G[r][q] = G[q + 1][r];
                    G[q + 1][r] = G[r][q + 1] = t;
                }
        // Lagrange reduction of (e, f) = (b1, b0); h_e, h_f their products with b2
        V3 e = b[1], f = b[0];
        float gee = G[1][1], gff = G[0][0], gef = G[0][1], he = G[1][2], hf = G[0][2];
        for (int l = 0; l < 48; ++l) {
            if (!(gff > 0.f)) break;
            float r = rintf(gef / gff);
            r = fminf(fmaxf(r, -256.f), 256.f);
            const V3 nf = sub_mul(e, r, f);
            const float gnn = fmaf(-r, fmaf(-r, gff, 2.f * gef), gee);
            const float gfn = fmaf(-r, gff, gef);
            const float hn = fmaf(-r, hf, he);
            const bool shorter = gff > gnn;
            e = f;
            f = nf;
            gee = gff, gef = gfn, gff = gnn, he = hf, hf = hn;
            if (amax(f) > (float)(4 * kMaxCoord)) break;
            if (!shorter) break;
        }
        b[0] = e;
        b[1] = f;
        // closest vector to b2 in b0 Z + b1 Z, scored by
        // |b2 - k0 b0 - k1 b1|^2 = G22 - 2 (k0 h0 + k1 h1) + k0^2 G00 + 2 k0 k1 G01 + k1^2 G11
        const float G00 = gee, G01 = gef, G11 = gff, r0 = he, r1 = hf, G22 = G[2][2];
        const float det = G00 * G11 - G01 * G01;
        if (!(det > 0.f)) break;
        float y0 = (G11 * r0 - G01 * r1) / det, y1 = (G00 * r1 - G01 * r0) / det;
        y0 = fminf(fmaxf(y0, -512.f), 512.f);
        y1 = fminf(fmaxf(y1, -512.f), 512.f);
        const float f0 = floorf(y0), f1 = floorf(y1);
        float bk0 = 0.f, bk1 = 0.f;
        float bestn = 3.4e38f;
#pragma unroll
        for (int k0 = -1; k0 <= 2; ++k0)
#pragma unroll
            for (int k1 = -1; k1 <= 2; ++k1) {
                const float a0 = f0 + (float)k0, a1 = f1 + (float)k1;
                const float nt = fmaf(a0, fmaf(a0, G00, fmaf(2.f * a1, G01, -2.f * r0)),
                                      fmaf(a1, fmaf(a1, G11, -2.f * r1), G22));
                if (nt < bestn) {
                    bestn = nt;
                    bk0 = a0;
                    bk1 = a1;
                }
            }
        b[2] = sub_mul(sub_mul(b[2], bk0, b[0]), bk1, b[1]);
        if (amax(b[2]) > (float)(4 * kMaxCoord)) break;
        if (bestn >= G11) break;
    }

    // ---- Prop. MakeObtuse (approximate decisions) ----
    float Gf[3][3];
    gram3(d, b, Gf);
    float p01 = fabsf(Gf[0][1]), p02 = fabsf(Gf[0][2]), p12 = fabsf(Gf[1][2]);
    // the pair with the smallest |<.,D.>| is {b'1, b'2}; b'3 is the other vector,
    // b'2 the one of the pair whose product with b'3 is larger
    int i1, i2, i3;
    if (p01 <= p02 && p01 <= p12) {
        i3 = 2;
        if (p02 <= p12) { i1 = 0; i2 = 1; } else { i1 = 1; i2 = 0; }
    } else if (p02 <= p12) {
        i3 = 1;
        if (p01 <= p12) { i1 = 0; i2 = 2; } else { i1 = 2; i2 = 0; }
    } else {
        i3 = 0;
        if (p01 <= p02) { i1 = 1; i2 = 2; } else { i1 = 2; i2 = 1; }
    }
    V3 b1 = b[i1], b2 = b[i2], b3 = b[i3];
    float s13 = Gf[i1][i3], s23 = Gf[i2][i3], s12 = Gf[i1][i2];
    if (s13 > 0.f) b1 = neg(b1), s12 = -s12;
    if (s23 > 0.f) b2 = neg(b2), s12 = -s12;
    V3 e[4];
    if (s12 <= 0.f) {
        e[1] = b1;
        e[2] = b2;
        e[3] = b3;
        e[0] = neg(add(add(b1, b2), b3));
    } else {
        e[1] = neg(b1);
        e[2] = b2;
        e[3] = add(b1, b3);
        e[0] = neg(add(b2, b3));
    }

    // ---- certification with exact signs, Selling repair ----
    // pair q = (i, j), complement (k, l)
    constexpr int PI[6] = {0, 0, 0, 1, 1, 2};
    constexpr int PJ[6] = {1, 2, 3, 2, 3, 3};
    constexpr int PK[6] = {2, 1, 1, 0, 0, 0};
    constexpr int PL[6] = {3, 3, 2, 3, 2, 1};
    int sg[6];
    WV val[6];
    bool ok = false, range = false;
    for (int fix = 0; fix < 256; ++fix) {
        range = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) range |= amax(e[k]) > (float)kMaxCoord;
        if (range) break;
        int bad = -1;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            T x[6];
            float n[6];
            terms3(D, e[PI[q]], e[PJ[q]], x, n);
            sg[q] = sign_value_nf<6>(x, n, val[q]);
            if (sg[q] > 0 && bad < 0) bad = q;
        }
        if (bad < 0) {
            ok = true;
            break;
        }
        const int ii = PI[bad], kk = PK[bad], ll = PL[bad];
        V3 ei = e[ii];
        e[ii] = neg(ei);
        e[kk] = add(e[kk], ei);
        e[ll] = add(e[ll], ei);
    }
    if (!ok) {
        o[0] = o[1] = o[2] = make_char4(0, 0, 0, 0);
        store_weights<6>(wbase, wt, i, wz, 63u);
        atomicOr(err, range ? ERRBIT_RANGE : ERRBIT_NOT_CONVERGED);
        return;
    }

    unsigned zmask = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (sg[q] == 0) {
            zmask |= 1u << q;
        } else {
            wz[q] = wmax0(neg_half(val[q]));
        }
    }
#pragma unroll
    for (int k = 1; k < 4; ++k)
        o[k - 1] = make_char4((signed char)(int)e[k].x, (signed char)(int)e[k].y, (signed char)(int)e[k].z, 0);
    store_weights<6>(wbase, wt, i, wz, zmask);
}

}  // namespace

adlbr_status launch_build3d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st) {
    ADLBR_NVTX("build");
    stencils_changed(s);
    const int threads = 128;
    unsigned blocks = blocks_for(s->N, threads);
    if (D_t == ADLBR_F32)
        build3d_kernel<float><<<blocks, threads, 0, st>>>(s->N, (const float *)D, (char4 *)s->offs,
                                                          s->w, s->w_t, s->err);
    else
        build3d_kernel<double><<<blocks, threads, 0, st>>>(s->N, (const double *)D,
                                                           (char4 *)s->offs, s->w, s->w_t, s->err);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace adlbr

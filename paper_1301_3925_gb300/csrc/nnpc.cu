// Learned preconditioner for the implicit step (not in the paper) and the
// flexible preconditioned CG that uses it.
//
// For (I + dt A) x = b the preconditioner is
//   M(r) = r / d + s * P(N(R(f(r)))),
// d = 1 + dt A_zz (the Jacobi part), s = rms(r), N the U-Net of unet.cu, R the
// mean over 4 x 4 blocks, P the repetition of a coarse value over its block,
// and f the per-point features: r / s, log(1 + dt w_k) for the three
// canonical half-stencil weights, and the three canonical offsets / 8.  M is
// nonlinear (positively homogeneous in r), so the solver is flexible CG with
// the Polak-Ribiere beta = <r_{k+1} - r_k, z_{k+1}> / <r_k, z_k>.
//
// Training pairs come from the solver itself: CG is run to convergence for x*,
// then run again and at every `every` iterations the pair (coarse features of
// r_k, R((x* - x_k - r_k / d) / s)) is recorded.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "internal.cuh"
#include "reduce.cuh"

namespace adlbr {

namespace {

constexpr int RF = 4;                 // restriction factor
constexpr int NR = RF * RF;           // residual channels (space to depth)
constexpr int NS = 9;                 // static channels (stencil block means)
constexpr int NF = NR + NS;           // network input channels

struct FcgState {
    double rr, bb, tol2, rz, pq, alpha, beta, s, gamma;
    int conv, iters, max_iters;
    unsigned int count;
};

// A_zz: every in-grid pair (z, z +- e_k) adds w_k at both ends
__global__ void diag2d_kernel(int nx, int ny, int bc, const short4 *__restrict__ offs,
                              const short2 *__restrict__ offs3, const void *__restrict__ wbase, adlbr_dtype wt,
                              float *__restrict__ d) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int64_t z = (int64_t)y * nx + x;
    float w[3];
    load_weights<float, 3>(wbase, wt, z, w);
    int ex[3], ey[3];
    offsets2d(offs[z], offs3, z, ex, ey);
    float own = 0.f;
    for (int k = 0; k < 3; ++k) {
        if (w[k] == 0.f) continue;
        for (int s = -1; s <= 1; s += 2) {
            int xn = x + s * ex[k], yn = y + s * ey[k];
            if (bc == ADLBR_PERIODIC) {
                xn = ((xn % nx) + nx) % nx;
                yn = ((yn % ny) + ny) % ny;
            } else if (xn < 0 || xn >= nx || yn < 0 || yn >= ny) {
                continue;
            }
            const int64_t zn = (int64_t)yn * nx + xn;
            if (zn == z) continue;
            own += w[k];
            atomicAdd(d + zn, w[k]);
        }
    }
    atomicAdd(d + z, own);
}

// 3D: every in-grid pair (z, z +- c_q) of the six Selling offsets adds w_q
// at both ends
__global__ void diag3d_kernel(int nx, int ny, int nz, int bc, const char4 *__restrict__ offs,
                              const void *__restrict__ wbase, adlbr_dtype wt, float *__restrict__ d) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, zc = blockIdx.z;
    if (x >= nx) return;
    const int64_t z = ((int64_t)zc * ny + y) * nx + x;
    const char4 b[3] = {offs[3 * z], offs[3 * z + 1], offs[3 * z + 2]};
    int c[6][3];
    selling_offsets(b, c);
    float w[6];
    load_weights<float, 6>(wbase, wt, z, w);
    float own = 0.f;
    for (int q = 0; q < 6; ++q) {
        if (w[q] == 0.f) continue;
        for (int s = -1; s <= 1; s += 2) {
            int xn = x + s * c[q][0], yn = y + s * c[q][1], zn = zc + s * c[q][2];
            if (bc == ADLBR_PERIODIC) {
                xn = ((xn % nx) + nx) % nx;
                yn = ((yn % ny) + ny) % ny;
                zn = ((zn % nz) + nz) % nz;
            } else if (xn < 0 || xn >= nx || yn < 0 || yn >= ny || zn < 0 || zn >= nz) {
                continue;
            }
            const int64_t zz = ((int64_t)zn * ny + yn) * nx + xn;
            if (zz == z) continue;
            own += w[q];
            atomicAdd(d + zz, w[q]);
        }
    }
    atomicAdd(d + z, own);
}

// d <- 1 + dt d ; max of d over the grid into *dmax (as ordered bits; d >= 0)
__global__ void diag_finish_kernel(int64_t N, float dt, float *__restrict__ d, unsigned *dmax_bits) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (i < N) {
        m = d[i];
        if (dt > 0.f) d[i] = 1.f + dt * m;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && dmax_bits) atomicMax(dmax_bits, __float_as_uint(m));
}

// canonical half-stencil of one point (same rule as adlbr_stencils_export)
__device__ __forceinline__ void canonical2(short4 o, const float (&w)[3], unsigned zmask, int (&v)[3][2],
                                           float (&wc)[3]) {
    int t[3][2] = {{o.x, o.y}, {o.z, o.w}, {-o.x - o.z, -o.y - o.w}};
    float tw[3] = {w[0], w[1], w[2]};
    for (int k = 0; k < 3; ++k) {
        if (zmask >> k & 1u) {
            t[k][0] = t[k][1] = 0;
            tw[k] = 0.f;
        } else if (t[k][0] < 0 || (t[k][0] == 0 && t[k][1] < 0)) {
            t[k][0] = -t[k][0];
            t[k][1] = -t[k][1];
        }
    }
    int idx[3] = {0, 1, 2};
    for (int a = 1; a < 3; ++a)
        for (int b = a; b > 0; --b) {
            const int *p = t[idx[b]], *q = t[idx[b - 1]];
            if (p[0] < q[0] || (p[0] == q[0] && p[1] < q[1])) {
                int tmp = idx[b];
                idx[b] = idx[b - 1];
                idx[b - 1] = tmp;
            }
        }
    for (int k = 0; k < 3; ++k) {
        v[k][0] = t[idx[k]][0];
        v[k][1] = t[idx[k]][1];
        wc[k] = tw[idx[k]];
    }
}

// channels NR .. NR+8 of the coarse features: block means of log(1 + dt w_k)
// and offset / 8 (canonical order)
__global__ void static_features_kernel(int nx, int ny, float dt, const short4 *__restrict__ offs,
                                       const void *__restrict__ wbase, adlbr_dtype wt,
                                       float *__restrict__ feat) {
    const int Wc = nx / RF, Hc = ny / RF;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x, cy = blockIdx.y;
    if (cx >= Wc) return;
    float acc[NS] = {};
    for (int dy = 0; dy < RF; ++dy)
        for (int dx = 0; dx < RF; ++dx) {
            const int64_t z = (int64_t)(cy * RF + dy) * nx + cx * RF + dx;
            float w[3];
            const unsigned zm = load_weights<float, 3>(wbase, wt, z, w);
            int v[3][2];
            float wc[3];
            canonical2(offs[z], w, zm, v, wc);
            for (int k = 0; k < 3; ++k) {
                acc[k] += log1pf(dt * wc[k]);
                acc[3 + 2 * k] += 0.125f * (float)v[k][0];
                acc[4 + 2 * k] += 0.125f * (float)v[k][1];
            }
        }
    const int64_t Nc = (int64_t)Hc * Wc;
    for (int c = 0; c < NS; ++c) feat[(NR + c) * Nc + (int64_t)cy * Wc + cx] = acc[c] * (1.f / (RF * RF));
}

// channels 0 .. NR-1: the RF x RF values of r / s in each block (space to
// depth, channel dy * RF + dx)
__global__ void coarse_r_kernel(int nx, int ny, const float *__restrict__ r, const FcgState *S, int64_t N,
                                float *__restrict__ feat) {
    if (S && S->conv) return;
    const int Wc = nx / RF, Hc = ny / RF;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x, cy = blockIdx.y;
    if (cx >= Wc) return;
    const double s = S ? sqrt(S->rr / (double)N) : 1.0;
    const float inv = s > 0.0 ? (float)(1.0 / s) : 0.f;
    const int64_t Nc = (int64_t)Hc * Wc;
    for (int dy = 0; dy < RF; ++dy)
        for (int dx = 0; dx < RF; ++dx)
            feat[(dy * RF + dx) * Nc + (int64_t)cy * Wc + cx] =
                r[(int64_t)(cy * RF + dy) * nx + cx * RF + dx] * inv;
}

// The same two feature sets written straight into the tensor-core network's
// BF16 channels-last input x ([Hc][Wc][cp]), with the rounding of its own
// conversion (FP32 feature, then round to nearest BF16):
// channels 0 .. NR-1 = r / s per block (every iteration; four 16-byte row
// reads, two 16-byte stores per coarse point) ...
__global__ void coarse_r_nhwc_kernel(int nx, int ny, const float *__restrict__ r, const FcgState *S, int64_t N,
                                     int cp, __nv_bfloat16 *__restrict__ xh) {
    static_assert(RF == 4 && NR == 16, "one float4 per block row, two 8-channel stores");
    if (S->conv) return;
    const int Wc = nx / RF, Hc = ny / RF;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x, cy = blockIdx.y;
    if (cx >= Wc || cy >= Hc) return;
    const double s = sqrt(S->rr / (double)N);
    const float inv = s > 0.0 ? (float)(1.0 / s) : 0.f;
    float f[NR];
#pragma unroll
    for (int dy = 0; dy < RF; ++dy) {
        const float4 v = *reinterpret_cast<const float4 *>(r + (int64_t)(cy * RF + dy) * nx + cx * RF);
        f[dy * RF + 0] = v.x * inv;
        f[dy * RF + 1] = v.y * inv;
        f[dy * RF + 2] = v.z * inv;
        f[dy * RF + 3] = v.w * inv;
    }
    uint4 o[2];
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(o);
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    uint4 *d = reinterpret_cast<uint4 *>(xh + ((int64_t)cy * Wc + cx) * cp);
    d[0] = o[0];
    d[1] = o[1];
}

// ... and channels NR .. cp-1 = the static features, then zeros (once per solve).
__global__ void static_nhwc_kernel(int64_t Nc, int cp, const float *__restrict__ feat,
                                   __nv_bfloat16 *__restrict__ xh) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Nc; q += (int64_t)gridDim.x * blockDim.x) {
        for (int c0 = NR; c0 < cp; c0 += 8) {
            uint4 o;
            __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = c0 + 2 * k;
                h[k] = __floats2bfloat162_rn(c < NF ? feat[c * Nc + q] : 0.f, c + 1 < NF ? feat[(c + 1) * Nc + q] : 0.f);
            }
            reinterpret_cast<uint4 *>(xh + q * cp)[c0 / 8] = o;
        }
    }
}

// (Re)start of a refinement round: r = b - (x + dt A x) with dt A x
// accumulated in FP64 (acc), rounded once to FP32; |r|^2 of the FP32 copy and
// |b|^2; conv = 1 when it already meets the tolerance.
__global__ void __launch_bounds__(RT) fcg_init64_kernel(int64_t N, const float *__restrict__ b,
                                                        const float *__restrict__ x, const double *__restrict__ acc,
                                                        float *__restrict__ r, double *partials,
                                                        double *partials2, FcgState *S) {
    FFAcc s_rr, s_bb;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        const float ri = (float)((double)b[i] - ((double)x[i] + acc[i]));
        r[i] = ri;
        ff_add_prod(s_rr, ri, ri);
        ff_add_prod(s_bb, b[i], b[i]);
    }
    const double pr = block_sum_ff(s_rr);
    const double pb = block_sum_ff(s_bb);
    double tot, bb;
    if (finish_reduction2(pr, pb, partials, partials2, &S->count, tot, bb)) {
        S->rr = tot;
        S->bb = bb;
        S->conv = (tot <= S->tol2 * bb) ? 1 : 0;
    }
}

// The preconditioner alone (adlbr_nn_precondition): z = r / d + s P(y),
// with rz = <r,z> and p = q = z (the solver uses the Galerkin-step kernels
// below instead).
template <bool FIRST>
__global__ void __launch_bounds__(RT) fcg_z_kernel(int nx, int64_t N, const float *__restrict__ r,
                                                   const float *__restrict__ r_old,
                                                   const float *__restrict__ d,
                                                   const float *__restrict__ y, float *__restrict__ z,
                                                   float *__restrict__ p, float *__restrict__ q,
                                                   double *partials, double *partials2, FcgState *S) {
    if (S->conv) return;
    const int Wc = nx / RF;
    const float s = (float)sqrt(S->rr / (double)N);
    FFAcc s_rz, s_oz;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        const int xx = (int)(i % nx), yy = (int)(i / nx);
        const float zi = r[i] / d[i] + s * y[(int64_t)(yy / RF) * Wc + xx / RF];
        z[i] = zi;
        if (FIRST) p[i] = zi, q[i] = zi;
        ff_add_prod(s_rz, r[i], zi);
        if (!FIRST) ff_add_prod(s_oz, r_old[i], zi);
    }
    const double prz = block_sum_ff(s_rz);
    const double poz = block_sum_ff(s_oz);
    double tot, oz;
    if (finish_reduction2(prz, poz, partials, partials2, &S->count, tot, oz)) {
        if (!FIRST) S->beta = (tot - oz) / S->rz;
        S->rz = tot;
    }
}

// Step length of the network correction (flexible CG with a Galerkin step):
// the preconditioned residual is z = r/d + gamma c with c = s P(y), and gamma
// minimises the (I + dt A)-energy of the error of z as an approximation of
// (I + dt A)^{-1} r:  gamma = <c, r - (I + dt A) r/d> / <c, (I + dt A) c>.
// With c = 0 (no correction) gamma = 0 and z is the Jacobi step.
//
// w = r/d into z, c = s P(y), and the starting values g1 = w, g2 = c of the
// two operator accumulations.
__global__ void __launch_bounds__(RT) fcg_w_kernel(int nx, int64_t N, const float *__restrict__ r,
                                                   const float *__restrict__ d, const float *__restrict__ y,
                                                   float *__restrict__ w, float *__restrict__ c,
                                                   float *__restrict__ g1, float *__restrict__ g2,
                                                   const FcgState *S) {
    if (S->conv) return;
    const int Wc = nx / RF;
    const float s = (float)sqrt(S->rr / (double)N);
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        const int xx = (int)(i % nx), yy = (int)(i / nx);
        const float wi = r[i] / d[i];
        const float ci = s * y[(int64_t)(yy / RF) * Wc + xx / RF];
        w[i] = wi;
        g1[i] = wi;
        c[i] = ci;
        g2[i] = ci;
    }
}

// gamma = <c, r - g1> / <c, g2>   (g1 = (I + dt A) r/d, g2 = (I + dt A) c)
__global__ void __launch_bounds__(RT) fcg_gamma_kernel(int64_t N, const float *__restrict__ r,
                                                       const float *__restrict__ c, const float *__restrict__ g1,
                                                       const float *__restrict__ g2, double *partials,
                                                       double *partials2, FcgState *S) {
    if (S->conv) return;
    FFAcc sn, sm;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        ff_add_prod(sn, c[i], r[i] - g1[i]);
        ff_add_prod(sm, c[i], g2[i]);
    }
    const double pn = block_sum_ff(sn);
    const double pm = block_sum_ff(sm);
    double tot, m;
    if (finish_reduction2(pn, pm, partials, partials2, &S->count, tot, m)) {
        S->gamma = m > 0.0 ? tot / m : 0.0;
    }
}

// z = w + gamma c (in place over w), Az = g1 + gamma g2 (in place over g1);
// first: rz = <r,z>.  Otherwise: beta = (<r,z> - <r_old,z>) / rz, rz = <r,z>.
template <bool FIRST>
__global__ void __launch_bounds__(RT) fcg_z2_kernel(int64_t N, const float *__restrict__ r,
                                                    const float *__restrict__ r_old, float *__restrict__ z,
                                                    const float *__restrict__ c, float *__restrict__ g1,
                                                    const float *__restrict__ g2, double *partials,
                                                    double *partials2, FcgState *S) {
    if (S->conv) return;
    const float gamma = (float)S->gamma;
    FFAcc s_rz, s_oz;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        const float zi = fmaf(gamma, c[i], z[i]);
        z[i] = zi;
        g1[i] = fmaf(gamma, g2[i], g1[i]);
        ff_add_prod(s_rz, r[i], zi);
        if (!FIRST) ff_add_prod(s_oz, r_old[i], zi);
    }
    const double prz = block_sum_ff(s_rz);
    const double poz = block_sum_ff(s_oz);
    double tot, oz;
    if (finish_reduction2(prz, poz, partials, partials2, &S->count, tot, oz)) {
        if (!FIRST) S->beta = (tot - oz) / S->rz;
        S->rz = tot;
    }
}

// p = z + beta p ; q = Az + beta q   (first: p = z, q = Az), then
// alpha = rz / <p, q> from the values just written (q = p + dt A p)
template <bool FIRST>
__global__ void __launch_bounds__(RT) fcg_p2_kernel(int64_t N, const float *__restrict__ z,
                                                    const float *__restrict__ Az, float *__restrict__ p,
                                                    float *__restrict__ q, double *partials, FcgState *S) {
    if (S->conv) return;
    const float beta = FIRST ? 0.f : (float)S->beta;
    FFAcc s;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        const float pi = FIRST ? z[i] : fmaf(beta, p[i], z[i]);
        const float qi = FIRST ? Az[i] : fmaf(beta, q[i], Az[i]);
        p[i] = pi;
        q[i] = qi;
        ff_add_prod(s, pi, qi);
    }
    double part = block_sum_ff(s);
    double tot;
    if (finish_reduction(part, partials, &S->count, tot)) {
        S->pq = tot;
        S->alpha = S->rz / tot;
    }
}

// x += alpha p ; r_old = r ; r -= alpha q ; rr ; flag
__global__ void __launch_bounds__(RT) fcg_x_kernel(int64_t N, float *__restrict__ x,
                                                   const float *__restrict__ p, float *__restrict__ r,
                                                   float *__restrict__ r_old, const float *__restrict__ q,
                                                   double *partials, FcgState *S) {
    if (S->conv) return;
    const float alpha = (float)S->alpha;
    FFAcc s;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        x[i] += alpha * p[i];
        const float ro = r[i];
        r_old[i] = ro;
        const float ri = ro - alpha * q[i];
        r[i] = ri;
        ff_add_prod(s, ri, ri);
    }
    double part = block_sum_ff(s);
    double tot;
    if (finish_reduction(part, partials, &S->count, tot)) {
        S->rr = tot;
        S->iters += 1;
        if (!(tot == tot) || tot > 3.0e38)
            S->conv = 3;   // non-finite residual: stop, reported as a failure
        else if (tot <= S->tol2 * S->bb)
            S->conv = 1;
        else if (S->iters >= S->max_iters)
            S->conv = 2;
    }
}


// training target: R((xs - x - r / d) / s) with s = rms(r) (given)
__global__ void target_kernel(int nx, int ny, const float *__restrict__ xs, const float *__restrict__ x,
                              const float *__restrict__ r, const float *__restrict__ d, float inv_s,
                              float *__restrict__ t) {
    const int Wc = nx / RF;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x, cy = blockIdx.y;
    if (cx >= Wc) return;
    float a = 0.f;
    for (int dy = 0; dy < RF; ++dy)
        for (int dx = 0; dx < RF; ++dx) {
            const int64_t i = (int64_t)(cy * RF + dy) * nx + cx * RF + dx;
            a += xs[i] - x[i] - r[i] / d[i];
        }
    t[(int64_t)cy * Wc + cx] = a * (inv_s / (RF * RF));
}

// |b - (x + acc)|^2 (acc = dt A x accumulated in FP64) into S->rr, |b|^2 into S->bb
__global__ void __launch_bounds__(RT) resid64_kernel(int64_t N, const float *__restrict__ b,
                                                     const float *__restrict__ x,
                                                     const double *__restrict__ acc, double *partials,
                                                     double *partials2, FcgState *S) {
    double s_rr = 0.0, s_bb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        const double ri = (double)b[i] - ((double)x[i] + acc[i]);
        s_rr += ri * ri;
        s_bb += (double)b[i] * b[i];
    }
    const double pr = block_sum(s_rr);
    const double pb = block_sum(s_bb);
    double tot, bb;
    if (finish_reduction2(pr, pb, partials, partials2, &S->count, tot, bb)) {
        S->rr = tot;
        S->bb = bb;
    }
}

__global__ void __launch_bounds__(RT) sumsq_kernel(int64_t N, const float *__restrict__ v, double *partials,
                                                   unsigned *count, double *out) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT)
        s += (double)v[i] * v[i];
    double part = block_sum(s);
    double tot;
    if (finish_reduction(part, partials, count, tot)) *out = tot;
}

}  // namespace

struct NnWorkspace {
    float *r, *p, *q, *z, *r_old, *d, *feat, *y, *xs;
    float *c, *g1, *g2;   // network correction, (I + dt A) r/d, (I + dt A) c
    double *partials, *partials2, *scal;
    FcgState *S;
    unsigned *dmax, *cnt;
    // for the training-pair hook, which runs inside a solve
    double *partials_h, *scal_h;
    FcgState *Sh;
    unsigned *cnt_h;
};

static adlbr_status nn_workspace(adlbr_stencils *s, NnWorkspace &W) {
    const int64_t N = s->N, Nc = N / (RF * RF);
    size_t need = (10 * (size_t)N + (NF + 1) * (size_t)Nc) * sizeof(float) + 3 * vec_blocks() * sizeof(double) + 4096;
    if (!s->ws_nn || s->ws_nn_bytes < need) {
        if (s->ws_nn) cudaFree(s->ws_nn);
        s->ws_nn = nullptr;
        ADLBR_CUDA(cudaMalloc(&s->ws_nn, need));
        s->ws_nn_bytes = need;
    }
    float *f = (float *)s->ws_nn;
    W.r = f;
    W.p = W.r + N;
    W.q = W.p + N;
    W.z = W.q + N;
    W.r_old = W.z + N;
    W.d = W.r_old + N;
    W.xs = W.d + N;
    W.c = W.xs + N;
    W.g1 = W.c + N;
    W.g2 = W.g1 + N;
    W.feat = W.g2 + N;
    W.y = W.feat + NF * Nc;
    uintptr_t a = (uintptr_t)(W.y + Nc);
    a = (a + 255) & ~(uintptr_t)255;
    W.partials = (double *)a;
    W.partials2 = W.partials + vec_blocks();
    W.scal = W.partials2 + vec_blocks();
    a = (uintptr_t)(W.scal + 4);
    a = (a + 255) & ~(uintptr_t)255;
    W.S = (FcgState *)a;
    W.dmax = (unsigned *)(W.S + 1);
    W.cnt = W.dmax + 1;
    a = (uintptr_t)(W.cnt + 1);
    a = (a + 255) & ~(uintptr_t)255;
    W.Sh = (FcgState *)a;
    a = (uintptr_t)(W.Sh + 1);
    a = (a + 255) & ~(uintptr_t)255;
    W.partials_h = (double *)a;
    W.scal_h = W.partials_h + vec_blocks();
    W.cnt_h = (unsigned *)(W.scal_h + 2);
    return ADLBR_OK;
}

// d = 1 + dt A_zz into W.d (dt = 0 leaves A_zz); max A_zz into *dmax_host when
// non-NULL (synchronises)
static adlbr_status compute_diag(adlbr_stencils *s, NnWorkspace &W, double dt, double *dmax_host,
                                 cudaStream_t st) {
    ADLBR_CUDA(cudaMemsetAsync(W.d, 0, s->N * sizeof(float), st));
    ADLBR_CUDA(cudaMemsetAsync(W.dmax, 0, sizeof(unsigned), st));
    dim3 g(blocks_for(s->n[0], 256), (unsigned)s->n[1]);
    if (s->dim == 2)
        diag2d_kernel<<<g, 256, 0, st>>>((int)s->n[0], (int)s->n[1], s->bc, (const short4 *)s->offs, (const short2 *)s->offs3,
                                         s->w, s->w_t, W.d);
    else
        diag3d_kernel<<<dim3(blocks_for(s->n[0], 128), (unsigned)s->n[1], (unsigned)s->n[2]), 128, 0, st>>>(
            (int)s->n[0], (int)s->n[1], (int)s->n[2], s->bc, (const char4 *)s->offs, s->w, s->w_t, W.d);
    diag_finish_kernel<<<blocks_for(s->N, 256), 256, 0, st>>>(s->N, (float)dt, W.d, W.dmax);
    ADLBR_CUDA(cudaGetLastError());
    if (dmax_host) {
        unsigned bits = 0;
        ADLBR_CUDA(cudaMemcpyAsync(&bits, W.dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        ADLBR_CUDA(cudaStreamSynchronize(st));
        float f;
        memcpy(&f, &bits, sizeof f);
        *dmax_host = f;
    }
    return ADLBR_OK;
}

// 1 / (1 + dt A_zz) per point (the Jacobi preconditioner of the implicit step)
__global__ void invert_kernel(int64_t N, float *__restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) d[i] = 1.f / d[i];
}

adlbr_status launch_jacobi_inverse(const adlbr_stencils *s, double dt, float *inv_d, cudaStream_t st) {
    ADLBR_CUDA(cudaMemsetAsync(inv_d, 0, s->N * sizeof(float), st));
    if (s->dim == 2) {
        dim3 g(blocks_for(s->n[0], 256), (unsigned)s->n[1]);
        diag2d_kernel<<<g, 256, 0, st>>>((int)s->n[0], (int)s->n[1], s->bc, (const short4 *)s->offs, (const short2 *)s->offs3, s->w,
                                         s->w_t, inv_d);
    } else {
        diag3d_kernel<<<dim3(blocks_for(s->n[0], 128), (unsigned)s->n[1], (unsigned)s->n[2]), 128, 0, st>>>(
            (int)s->n[0], (int)s->n[1], (int)s->n[2], s->bc, (const char4 *)s->offs, s->w, s->w_t, inv_d);
    }
    diag_finish_kernel<<<blocks_for(s->N, 256), 256, 0, st>>>(s->N, (float)dt, inv_d, nullptr);
    invert_kernel<<<blocks_for(s->N, 256), 256, 0, st>>>(s->N, inv_d);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

static adlbr_status check_nn_grid(const adlbr_stencils *s, const adlbr_unet *net) {
    if (s->dim != 2) return fail(ADLBR_E_SHAPE, "the learned preconditioner is 2D only");
    if (s->scheme != ADLBR_SCHEME_ADLBR)
        return fail(ADLBR_E_ARG, "the learned preconditioner's features are defined for AD-LBR stencils");
    if (s->n[0] % (RF * 4) || s->n[1] % (RF * 4))
        return fail(ADLBR_E_SHAPE, "grid extents must be multiples of %d for the preconditioner", RF * 4);
    int cin, B, H, Wd;
    unet_shape(net, &cin, &B, &H, &Wd);
    if (cin != NF || B != 1 || H != s->n[1] / RF || Wd != s->n[0] / RF)
        return fail(ADLBR_E_SHAPE, "network shape must be cin=%d, batch 1, %lld x %lld", NF,
                    (long long)(s->n[1] / RF), (long long)(s->n[0] / RF));
    return ADLBR_OK;
}

static void static_features(adlbr_stencils *s, NnWorkspace &W, double dt, cudaStream_t st) {
    const int nx = (int)s->n[0], ny = (int)s->n[1];
    dim3 gc(blocks_for(nx / RF, 128), (unsigned)(ny / RF));
    static_features_kernel<<<gc, 128, 0, st>>>(nx, ny, (float)dt, (const short4 *)s->offs, s->w, s->w_t,
                                               W.feat);
}

// z = M(r) for the current r (uses S->rr for s); FIRST sets p = z and rz.
template <bool FIRST>
static adlbr_status precondition(adlbr_stencils *s, NnWorkspace &W, adlbr_unet *net, const float *params,
                                 cudaStream_t st) {
    const int nx = (int)s->n[0], ny = (int)s->n[1];
    dim3 gc(blocks_for(nx / RF, 128), (unsigned)(ny / RF));
    coarse_r_kernel<<<gc, 128, 0, st>>>(nx, ny, W.r, W.S, s->N, W.feat);
    if (adlbr_status e = unet_forward(net, params, W.feat, W.y, st)) return e;
    fcg_z_kernel<FIRST><<<vec_blocks(), RT, 0, st>>>(nx, s->N, W.r, W.r_old, W.d, W.y, W.z, W.p, W.q,
                                           W.partials, W.partials2, W.S);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

static adlbr_status run_fcg_hooked(adlbr_stencils *s, const float *b, float *x, double dt, double rtol,
                                   int maxit, const adlbr_nn_precond *nn, int *iters_out,
                                   double *relres_out, int every, CgHook hook, void *ctx,
                                   cudaStream_t st);

static thread_local int g_fallback = 0;

adlbr_status run_fcg(adlbr_stencils *s, const float *b, float *x, double dt, double rtol, int maxit,
                     const adlbr_nn_precond *nn, int *iters_out, double *relres_out, cudaStream_t st) {
    return run_fcg_hooked(s, b, x, dt, rtol, maxit, nn, iters_out, relres_out, 2, nullptr, nullptr, st);
}

// The next search direction of the flexible solve: network correction, its
// Galerkin step length, z and (I + dt A) z, then p and q = (I + dt A) p.
template <bool FIRST>
static adlbr_status galerkin_direction(adlbr_stencils *s, NnWorkspace &W, adlbr_unet *net, const float *params,
                                       double dt, const int *skip, cudaStream_t st) {
    const int nx = (int)s->n[0], ny = (int)s->n[1];
    const int64_t N = s->N;
    dim3 gc(blocks_for(nx / RF, 128), (unsigned)(ny / RF));
    int cp = 0;
    if (__nv_bfloat16 *xh = unet_tc_input(net, &cp)) {
        // the static channels and the packed weights were set up at the start
        // of the solve
        coarse_r_nhwc_kernel<<<gc, 128, 0, st>>>(nx, ny, W.r, W.S, N, cp, xh);
        if (adlbr_status e = unet_forward_from_input(net, params, W.y, st)) return e;
    } else {
        coarse_r_kernel<<<gc, 128, 0, st>>>(nx, ny, W.r, W.S, N, W.feat);
        if (adlbr_status e = unet_forward(net, params, W.feat, W.y, st)) return e;
    }
    fcg_w_kernel<<<vec_blocks(), RT, 0, st>>>(nx, N, W.r, W.d, W.y, W.z, W.c, W.g1, W.g2, W.S);
    if (adlbr_status e = launch_accumulate(s, W.z, W.g1, ADLBR_F32, dt, skip, st)) return e;
    if (adlbr_status e = launch_accumulate(s, W.c, W.g2, ADLBR_F32, dt, skip, st)) return e;
    fcg_gamma_kernel<<<vec_blocks(), RT, 0, st>>>(N, W.r, W.c, W.g1, W.g2, W.partials, W.partials2, W.S);
    fcg_z2_kernel<FIRST><<<vec_blocks(), RT, 0, st>>>(N, W.r, W.r_old, W.z, W.c, W.g1, W.g2, W.partials, W.partials2,
                                            W.S);
    fcg_p2_kernel<FIRST><<<vec_blocks(), RT, 0, st>>>(N, W.z, W.g1, W.p, W.q, W.partials, W.S);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

// Flexible PCG (Polak-Ribiere beta) with the Galerkin-step preconditioner:
// per iteration two operator applications (to r/d and to the correction c)
// and no other; q = (I + dt A) p follows from them by linearity.  When hook
// != NULL it is called with the current residual and iterate every `every`
// iterations while the solve runs.
static adlbr_status run_fcg_hooked(adlbr_stencils *s, const float *b, float *x, double dt, double rtol,
                                   int maxit, const adlbr_nn_precond *nn, int *iters_out,
                                   double *relres_out, int every, CgHook hook, void *ctx,
                                   cudaStream_t st) {
    if (!nn || !nn->net || !nn->params) return fail(ADLBR_E_ARG, "null preconditioner");
    if (adlbr_status e = check_nn_grid(s, nn->net)) return e;
    NnWorkspace W;
    if (adlbr_status e = nn_workspace(s, W)) return e;
    const int64_t N = s->N;
    if (adlbr_status e = compute_diag(s, W, dt, nullptr, st)) return e;
    static_features(s, W, dt, st);
    {   // tensor-core network: its input buffer keeps the static channels and
        // its packed weights stay for the whole solve
        int cp = 0;
        if (__nv_bfloat16 *xh = unet_tc_input(nn->net, &cp)) {
            const int64_t Nc = N / (RF * RF);
            static_nhwc_kernel<<<(unsigned)std::min<int64_t>((Nc + 255) / 256, vec_blocks()), 256, 0, st>>>(Nc, cp, W.feat,
                                                                                                     xh);
            if (adlbr_status e = unet_tc_prepare(nn->net, nn->params, st)) return e;
        }
    }
    FcgState init = {};
    init.tol2 = rtol * rtol;
    const int *skip = (const int *)((const char *)W.S + offsetof(FcgState, conv));
    // q and z hold 8N bytes: the FP64 accumulator of dt A x between rounds
    double *acc64 = (double *)W.q;
    FcgState host = {};
    const int chunk = every > 0 ? every : 2;
    // Plain CG is the fallback of a user solve: the initial guess is kept, and
    // when the recursive residual of the preconditioned solve grows tenfold
    // above its best value, or fails to halve within kStall iterations, the
    // solve restarts from it with plain CG.
    constexpr int kStall = 100;
    if (!hook) {
        g_fallback = 0;
        ADLBR_CUDA(cudaMemcpyAsync(W.xs, x, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    auto enqueue_chunk = [&](cudaStream_t cs) -> adlbr_status {
        for (int k = 0; k < chunk; ++k) {
            // q = (I + dt A) p is carried by the recurrences (no operator
            // here) and alpha was set with p and q
            fcg_x_kernel<<<vec_blocks(), RT, 0, cs>>>(N, x, W.p, W.r, W.r_old, W.q, W.partials, W.S);
            if (adlbr_status e = galerkin_direction<false>(s, W, nn->net, nn->params, dt, skip, cs)) return e;
        }
        ADLBR_CUDA(cudaGetLastError());
        return ADLBR_OK;
    };
    // the chunk (about 25 launches per iteration, most of them the network's)
    // is recorded once per solve, after the first direction ran uncaptured
    // (so the kernels' one-time attribute settings are done), and replayed
    ChunkGraph graph;
    // Refinement rounds, as in plain CG: every round starts from the true
    // residual b - (I + dt A) x evaluated in FP64 and runs the flexible
    // iteration until the recursive residual meets rtol; a new round follows
    // while the true residual is above rtol and still halves per round.
    const int kMaxRestarts = 3;
    int total_iters = 0;
    double relres = INFINITY, prev = INFINITY;
    bool converged = false, fall_back = false;
    for (int round = 0; round <= kMaxRestarts; ++round) {
        init.max_iters = maxit - total_iters;
        ADLBR_CUDA(cudaMemcpyAsync(W.S, &init, sizeof(FcgState), cudaMemcpyHostToDevice, st));
        ADLBR_CUDA(cudaMemsetAsync(acc64, 0, N * sizeof(double), st));
        if (adlbr_status e = launch_accumulate_f64(s, x, acc64, dt, st)) return e;
        fcg_init64_kernel<<<vec_blocks(), RT, 0, st>>>(N, b, x, acc64, W.r, W.partials, W.partials2, W.S);
        ADLBR_CUDA(cudaGetLastError());
        ADLBR_CUDA(cudaMemcpyAsync(&host, W.S, sizeof(FcgState), cudaMemcpyDeviceToHost, st));
        ADLBR_CUDA(cudaStreamSynchronize(st));
        if (!std::isfinite(host.bb) || !std::isfinite(host.rr))
            return fail(ADLBR_E_NONFINITE, "non-finite right-hand side or iterate in the preconditioned solve");
        // the FP32 residual's norm stands for the true one at the round start
        relres = host.bb > 0 ? std::sqrt(host.rr / host.bb) : 0.0;
        if (relres <= rtol || total_iters >= maxit || round == kMaxRestarts) break;
        if (round > 0 && (relres <= 10.0 * rtol || !(relres < 0.5 * prev))) break;
        prev = relres;
        if (adlbr_status e = galerkin_direction<true>(s, W, nn->net, nn->params, dt, skip, st)) return e;
        if (!hook && !graph.exec)
            if (adlbr_status e = graph.capture(enqueue_chunk)) return e;
        double best = INFINITY;
        int best_it = 0, it = 0;
        while (it < maxit - total_iters) {
            if (hook && round == 0)
                if (adlbr_status e = hook(ctx, W.r, x, it, st)) return e;
            if (graph.exec) {
                ADLBR_CUDA(cudaGraphLaunch(graph.exec, st));
            } else if (adlbr_status e = enqueue_chunk(st)) {
                return e;
            }
            it += chunk;
            ADLBR_CUDA(cudaMemcpyAsync(&host, W.S, sizeof(FcgState), cudaMemcpyDeviceToHost, st));
            ADLBR_CUDA(cudaStreamSynchronize(st));
            if (host.conv == 3 && !hook) {   // non-finite: the preconditioner failed
                fall_back = true;
                break;
            }
            if (host.conv) break;
            if (!hook) {
                const double rel = host.bb > 0 ? std::sqrt(host.rr / host.bb) : 0.0;
                if (rel < 0.5 * best) best = rel, best_it = it;
                if (!(rel <= 10.0 * best) || it - best_it >= kStall) {
                    fall_back = true;
                    break;
                }
            }
        }
        total_iters += host.iters;
        if (fall_back) break;
        converged = host.conv == 1;
        if (host.conv == 3)
            return fail(ADLBR_E_NONFINITE, "preconditioned CG residual became non-finite after %d iterations",
                        total_iters);
        if (!converged) break;   // iteration limit
    }
    if (fall_back) {
        g_fallback = 1;
        ADLBR_CUDA(cudaMemcpyAsync(x, W.xs, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        int cg_it = 0;
        const adlbr_status e = run_cg(s, b, x, dt, rtol, std::max(1, maxit - total_iters), &cg_it, relres_out, st);
        if (iters_out) *iters_out = total_iters + cg_it;
        return e;
    }
    // the final true residual, FP64 throughout
    ADLBR_CUDA(cudaMemsetAsync(acc64, 0, N * sizeof(double), st));
    if (adlbr_status e = launch_accumulate_f64(s, x, acc64, dt, st)) return e;
    ADLBR_CUDA(cudaMemcpyAsync(W.S, &init, sizeof(FcgState), cudaMemcpyHostToDevice, st));
    resid64_kernel<<<vec_blocks(), RT, 0, st>>>(N, b, x, acc64, W.partials, W.partials2, W.S);
    FcgState fin = {};
    ADLBR_CUDA(cudaMemcpyAsync(&fin, W.S, sizeof(FcgState), cudaMemcpyDeviceToHost, st));
    ADLBR_CUDA(cudaStreamSynchronize(st));
    if (!std::isfinite(fin.bb) || !std::isfinite(fin.rr))
        return fail(ADLBR_E_NONFINITE, "non-finite right-hand side or iterate in the preconditioned solve");
    relres = fin.bb > 0 ? std::sqrt(fin.rr / fin.bb) : 0.0;
    if (iters_out) *iters_out = total_iters;
    if (relres_out) *relres_out = relres;
    set_last_residual_met(relres <= rtol);
    if (!(relres <= rtol) && !converged)
        return fail(ADLBR_E_NOT_CONVERGED, "preconditioned CG stopped after %d iterations (residual %.3e)",
                    total_iters, relres);
    return ADLBR_OK;
}

extern "C" int adlbr_last_fallback(void) { return g_fallback; }

// ---------------------------------------------------------------- training pairs
namespace {
struct PairCtx {
    adlbr_stencils *s;
    NnWorkspace *W;
    int max_pairs, n;
    float *feats, *targets;
};

adlbr_status pair_hook(void *vctx, const float *r, const float *x, int iter, cudaStream_t st) {
    PairCtx *c = (PairCtx *)vctx;
    if (c->n >= c->max_pairs) return ADLBR_OK;
    adlbr_stencils *s = c->s;
    NnWorkspace &W = *c->W;
    const int nx = (int)s->n[0], ny = (int)s->n[1];
    const int64_t Nc = s->N / (RF * RF);
    // the hook runs inside a solve: it uses its own state and partials
    ADLBR_CUDA(cudaMemsetAsync(W.cnt_h, 0, sizeof(unsigned), st));
    sumsq_kernel<<<vec_blocks(), RT, 0, st>>>(s->N, r, W.partials_h, W.cnt_h, W.scal_h);
    double ss = 0.0;
    ADLBR_CUDA(cudaMemcpyAsync(&ss, W.scal_h, sizeof(double), cudaMemcpyDeviceToHost, st));
    ADLBR_CUDA(cudaStreamSynchronize(st));
    const double rms = std::sqrt(ss / (double)s->N);
    if (!(rms > 0.0)) return ADLBR_OK;
    float *f = c->feats + (int64_t)c->n * NF * Nc;
    float *t = c->targets + (int64_t)c->n * Nc;
    // static channels: copied from the feature buffer, whose residual channels
    // the solver may be using -- only the static ones are read
    ADLBR_CUDA(cudaMemcpyAsync(f + NR * Nc, W.feat + NR * Nc, NS * Nc * sizeof(float),
                               cudaMemcpyDeviceToDevice, st));
    FcgState tmp = {};
    tmp.rr = ss;
    ADLBR_CUDA(cudaMemcpyAsync(W.Sh, &tmp, sizeof(FcgState), cudaMemcpyHostToDevice, st));
    dim3 gc(blocks_for(nx / RF, 128), (unsigned)(ny / RF));
    coarse_r_kernel<<<gc, 128, 0, st>>>(nx, ny, r, W.Sh, s->N, f);
    target_kernel<<<gc, 128, 0, st>>>(nx, ny, W.xs, x, r, W.d, (float)(1.0 / rms), t);
    ADLBR_CUDA(cudaGetLastError());
    ADLBR_CUDA(cudaStreamSynchronize(st));  // tmp is a stack value copied asynchronously
    c->n += 1;
    (void)iter;
    return ADLBR_OK;
}
}  // namespace

adlbr_status nn_pairs(adlbr_stencils *s, const float *b, double dt, double rtol, int maxit, int every,
                      int max_pairs, const adlbr_nn_precond *nn, float *feats, float *targets,
                      float *xbuf, int *n_pairs, cudaStream_t st) {
    if (s->dim != 2 || s->n[0] % (RF * 4) || s->n[1] % (RF * 4))
        return fail(ADLBR_E_SHAPE, "2D grid with extents multiple of %d required", RF * 4);
    if (every < 1 || max_pairs < 1) return fail(ADLBR_E_ARG, "bad every / max_pairs");
    NnWorkspace W;
    if (adlbr_status e = nn_workspace(s, W)) return e;
    if (adlbr_status e = compute_diag(s, W, dt, nullptr, st)) return e;
    static_features(s, W, dt, st);
    // x* by CG to convergence (the CG workspace is separate from W)
    ADLBR_CUDA(cudaMemcpyAsync(xbuf, b, s->N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    int it = 0;
    double rel = 0.0;
    if (adlbr_status e = run_cg(s, b, xbuf, dt, rtol, maxit, &it, &rel, st)) return e;
    ADLBR_CUDA(cudaMemcpyAsync(W.xs, xbuf, s->N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    // the same solve again, recording pairs
    ADLBR_CUDA(cudaMemcpyAsync(xbuf, b, s->N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    PairCtx ctx = {s, &W, max_pairs, 0, feats, targets};
    adlbr_status e;
    if (nn)  // residuals of the preconditioned solver itself
        e = run_fcg_hooked(s, b, xbuf, dt, rtol, maxit, nn, &it, &rel, every, pair_hook, &ctx, st);
    else
        e = run_cg_hooked(s, b, xbuf, dt, rtol, maxit, &it, &rel, every, pair_hook, &ctx, st);
    if (n_pairs) *n_pairs = ctx.n;
    // a recording solve that stops at the iteration limit still yields pairs
    if (e == ADLBR_E_NOT_CONVERGED && ctx.n > 0) return ADLBR_OK;
    return e;
}

adlbr_status nn_apply(adlbr_stencils *s, const adlbr_nn_precond *nn, double dt, const float *r,
                      float *z, cudaStream_t st) {
    if (!nn || !nn->net || !nn->params) return fail(ADLBR_E_ARG, "null preconditioner");
    if (adlbr_status e = check_nn_grid(s, nn->net)) return e;
    NnWorkspace W;
    if (adlbr_status e = nn_workspace(s, W)) return e;
    if (adlbr_status e = compute_diag(s, W, dt, nullptr, st)) return e;
    static_features(s, W, dt, st);
    ADLBR_CUDA(cudaMemcpyAsync(W.r, r, s->N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ADLBR_CUDA(cudaMemsetAsync(W.cnt, 0, sizeof(unsigned), st));
    sumsq_kernel<<<vec_blocks(), RT, 0, st>>>(s->N, r, W.partials, W.cnt, W.scal);
    double ss = 0.0;
    ADLBR_CUDA(cudaMemcpyAsync(&ss, W.scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    ADLBR_CUDA(cudaStreamSynchronize(st));
    if (!(ss > 0.0)) {
        ADLBR_CUDA(cudaMemsetAsync(z, 0, s->N * sizeof(float), st));
        return ADLBR_OK;
    }
    FcgState tmp = {};
    tmp.rr = ss;
    ADLBR_CUDA(cudaMemcpyAsync(W.S, &tmp, sizeof(FcgState), cudaMemcpyHostToDevice, st));
    if (adlbr_status e = precondition<true>(s, W, nn->net, nn->params, st)) return e;
    ADLBR_CUDA(cudaMemcpyAsync(z, W.z, s->N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ADLBR_CUDA(cudaStreamSynchronize(st));
    return ADLBR_OK;
}

adlbr_status max_diag(adlbr_stencils *s, double *out, cudaStream_t st) {
    NnWorkspace W;
    if (adlbr_status e = nn_workspace(s, W)) return e;
    return compute_diag(s, W, 0.0, out, st);
}

namespace {
__global__ void __launch_bounds__(RT) mse_kernel(int64_t n, const float *__restrict__ y,
                                                 const float *__restrict__ t, float *__restrict__ gy,
                                                 double *partials, unsigned *count, double *out) {
    double s = 0.0;
    const float sc = 2.f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        const float d = y[i] - t[i];
        gy[i] = sc * d;
        s += (double)d * d;
    }
    double part = block_sum(s);
    double tot;
    if (finish_reduction(part, partials, count, tot)) *out = tot / (double)n;
}
}  // namespace

adlbr_status mse_grad(const float *y, const float *t, int64_t n, float *gy, double *loss, cudaStream_t st) {
    // small persistent buffer for the reduction (partials, counter, result)
    static thread_local double *buf = nullptr;
    static thread_local int dev_of_buf = -1;
    int dev = -1;
    ADLBR_CUDA(cudaGetDevice(&dev));
    if (!buf || dev != dev_of_buf) {
        ADLBR_CUDA(cudaMalloc(&buf, (vec_blocks() + 64) * sizeof(double)));
        ADLBR_CUDA(cudaMemset(buf, 0, (vec_blocks() + 64) * sizeof(double)));
        dev_of_buf = dev;
    }
    unsigned *count = (unsigned *)(buf + vec_blocks());
    double *out = buf + vec_blocks() + 8;
    mse_kernel<<<vec_blocks(), RT, 0, st>>>(n, y, t, gy, buf, count, out);
    ADLBR_CUDA(cudaGetLastError());
    if (loss) {
        ADLBR_CUDA(cudaMemcpyAsync(loss, out, sizeof(double), cudaMemcpyDeviceToHost, st));
        ADLBR_CUDA(cudaStreamSynchronize(st));
    }
    return ADLBR_OK;
}

}  // namespace adlbr

// Operator application A u = (1/2) grad E_h(u) (Eq. def:E*, h = 1), the
// explicit step, and the canonical export of the stencils.
//
// The operator is a sum over the directed edges (z, e), e in V(z), of
// gamma_z(e) (u(z) - u(z+e)) added at z and subtracted at z+e.  Pairs that
// leave the grid are dropped (Neumann rule of Sec. 1) or wrapped (periodic).
//
// Scatter formulation: one thread per point z accumulates its own edges into
// a register and pushes the opposite contributions to the far ends.  The 2D
// kernel for FP32/F16/BF16 vectors works on a shared-memory window (see the
// tiled kernel below; 95% of the edges of the kappa <= 100 CED stencils are
// at most 8 points long).  The FP64 path and the 3D path push every
// contribution to L2 directly.
#include <type_traits>

#include "internal.cuh"

namespace adlbr {

namespace {

__device__ __forceinline__ int wrap(int c, int n) {
    c %= n;
    return c < 0 ? c + n : c;
}

__device__ __forceinline__ void red_add(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

// ---- 2D, shared-memory window ------------------------------------------
// A CTA owns a TW x TH tile.  It stages u over the tile plus an 8-point halo
// in shared memory, and keeps a shared accumulator over the same window.  An
// edge whose offset has Chebyshev length <= HALO stays inside the window for
// every point of the tile, so its neighbour value and both of its pushes are
// shared-memory operations; in a tile whose window lies inside the grid (or
// on a periodic grid) such edges need no boundary test either.  Longer edges
// read u from global memory and push to L2.  The window is then flushed with
// 16-byte vector reductions.
constexpr int HALO = 8;

// A warp covers WX x (32 / WX) points of the tile per pass; the row pitch P
// of the shared window puts the rows of one warp on disjoint bank ranges, so
// lanes that share an offset hit 32 different banks.
constexpr int window_pitch(int ww, int wx) {
    for (int p = ww;; p += 4) {
        bool ok = true;
        for (int r = 1; r < 32 / wx; ++r) {
            const int b = (r * p) % 32;
            if (b < wx || b > 32 - wx) ok = false;
        }
        if (ok) return p;
    }
}

template <int TW, int TH, int NT, int WX>
struct Tile {
    static constexpr int WW = TW + 2 * HALO, WH = TH + 2 * HALO;
    static constexpr int WR = 32 / WX;                   // rows per warp pass
    static constexpr int WARPS_X = TW / WX, WARPS_Y = NT / 32 / WARPS_X;
    static constexpr int P = window_pitch(WW, WX);       // shared row pitch (floats)
    static constexpr int PASSES = TH / (WR * WARPS_Y);
    static_assert(TW % WX == 0 && (NT / 32) % WARPS_X == 0 && TH % (WR * WARPS_Y) == 0, "tile");
    static_assert(WW % 4 == 0 && P % 4 == 0, "window rows must hold whole float4s");
};

// Weights of point z times `scale`.  For the F16 format the half is widened
// by moving its bits to the FP32 position and multiplying by 2^112 (exact,
// subnormal halves included); the per-point power of two and `scale` are
// applied by one more product, as in load_weights.
__device__ __forceinline__ void weights_f16_scaled(const void *wbase, int64_t z, float scale,
                                                   float (&w)[3]) {
    const uint2 r = reinterpret_cast<const uint2 *>(wbase)[z];
    const int s = (int)(int8_t)(r.y >> 24);
    const float c = __int_as_float((127 + s) << 23) * scale;
    w[0] = __uint_as_float((r.x & 0xffffu) << 13) * 0x1p112f * c;
    w[1] = __uint_as_float((r.x >> 16) << 13) * 0x1p112f * c;
    w[2] = __uint_as_float((r.y & 0xffffu) << 13) * 0x1p112f * c;
}

template <typename UT, int TW, int TH, int NT, int WX, bool F16W>
__global__ void __launch_bounds__(NT) apply2d_tiled(int nx, int ny, int bc, float scale,
                                                    const short4 *__restrict__ offs,
                                                    const void *__restrict__ wbase, adlbr_dtype wt,
                                                    const UT *__restrict__ u, float *__restrict__ acc,
                                                    const int *__restrict__ skip) {
    using T = Tile<TW, TH, NT, WX>;
    constexpr int WW = T::WW, WH = T::WH, P = T::P;
    extern __shared__ __align__(16) float smem[];
    float *uw = smem, *aw = smem + WH * P;
    if (skip && *skip) return;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const bool periodic = bc == ADLBR_PERIODIC;
    // full: every point of the tile is in the grid; inside: every short edge
    // of the tile stays in the grid (or wraps, on a periodic grid)
    const bool full = x0 + TW <= nx && y0 + TH <= ny;
    const bool inside = periodic || (x0 >= HALO && y0 >= HALO && x0 + TW + HALO <= nx &&
                                     y0 + TH + HALO <= ny);
    // stage u over the window (4 cells per step), zero the accumulator
    const bool vec = std::is_same<UT, float>::value && (nx % 4) == 0 && !periodic &&
                     ((uintptr_t)u % 16) == 0;
    for (int c4 = threadIdx.x; c4 < WH * WW / 4; c4 += NT) {
        const int wy = c4 / (WW / 4), wx = (c4 % (WW / 4)) * 4;
        const int gy = y0 - HALO + wy, gx = x0 - HALO + wx;
        float v[4];
        if (vec && (unsigned)gy < (unsigned)ny && gx >= 0 && gx + 3 < nx) {
            const float4 q = *reinterpret_cast<const float4 *>(
                reinterpret_cast<const float *>(u) + (int64_t)gy * nx + gx);
            v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                int xx = gx + t, yy = gy;
                v[t] = 0.f;
                if (periodic) {
                    xx = wrap(xx, nx);
                    yy = wrap(yy, ny);
                } else if ((unsigned)xx >= (unsigned)nx || (unsigned)yy >= (unsigned)ny) {
                    continue;
                }
                v[t] = to_acc(u[(int64_t)yy * nx + xx]);
            }
        }
        *reinterpret_cast<float4 *>(&uw[wy * P + wx]) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(&aw[wy * P + wx]) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx = (warp % T::WARPS_X) * WX + lane % WX;
    const int ty = (warp / T::WARPS_X) * T::WR + lane / WX;
    const int x = x0 + tx;
#pragma unroll 2
    for (int k = 0; k < T::PASSES; ++k) {
        const int ly = ty + k * T::WR * T::WARPS_Y, y = y0 + ly;
        if (!full && (x >= nx || y >= ny)) continue;
        const int64_t z = (int64_t)y * nx + x;
        const short4 o = offs[z];
        float w[3];
        if (F16W) {
            weights_f16_scaled(wbase, z, scale, w);
        } else {
            load_weights<float, 3>(wbase, wt, z, w);
#pragma unroll
            for (int i = 0; i < 3; ++i) w[i] *= scale;
        }
        const int ex[3] = {o.x, o.z, -o.x - o.z}, ey[3] = {o.y, o.w, -o.y - o.w};
        const int zw = (ly + HALO) * P + tx + HALO;
        const float uz = uw[zw];
        float own = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float wi = w[i];
            if (abs(ex[i]) <= HALO && abs(ey[i]) <= HALO) {
                const int d = ey[i] * P + ex[i];
#pragma unroll
                for (int sg = -1; sg <= 1; sg += 2) {
                    if (!inside) {
                        const int xn = x + sg * ex[i], yn = y + sg * ey[i];
                        if ((unsigned)xn >= (unsigned)nx || (unsigned)yn >= (unsigned)ny) continue;
                    }
                    const int zn = zw + sg * d;
                    const float f = wi * (uz - uw[zn]);
                    own += f;
                    atomicAdd(&aw[zn], -f);
                }
            } else if (wi != 0.f) {
#pragma unroll
                for (int sg = -1; sg <= 1; sg += 2) {
                    int xn = x + sg * ex[i], yn = y + sg * ey[i];
                    if (periodic) {
                        xn = wrap(xn, nx);
                        yn = wrap(yn, ny);
                    } else if ((unsigned)xn >= (unsigned)nx || (unsigned)yn >= (unsigned)ny) {
                        continue;
                    }
                    const int64_t zn = (int64_t)yn * nx + xn;
                    const float f = wi * (uz - to_acc(u[zn]));
                    own += f;
                    red_add(acc + zn, -f);
                }
            }
        }
        atomicAdd(&aw[zw], own);
    }
    __syncthreads();
    // flush the window: 4 consecutive cells per thread and step
    const bool vec_ok = (nx % 4) == 0 && ((uintptr_t)acc % 16) == 0;
    for (int c4 = threadIdx.x; c4 < WH * WW / 4; c4 += NT) {
        const int wy = c4 / (WW / 4), wx = (c4 % (WW / 4)) * 4;
        const float4 v = *reinterpret_cast<const float4 *>(&aw[wy * P + wx]);
        if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
        int gy = y0 - HALO + wy;
        const int gx = x0 - HALO + wx;
        if (periodic) gy = wrap(gy, ny);
        else if (gy < 0 || gy >= ny) continue;
        if (vec_ok && gx >= 0 && gx + 3 < nx) {
            red_add_v4(acc + (int64_t)gy * nx + gx, v.x, v.y, v.z, v.w);
        } else {
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (vv[t] == 0.f) continue;
                int xx = gx + t;
                if (periodic) xx = wrap(xx, nx);
                else if (xx < 0 || xx >= nx) continue;
                red_add(acc + (int64_t)gy * nx + xx, vv[t]);
            }
        }
    }
}

// ---- direct scatter (FP64 in 2D) ----------------------------------------
template <typename UT, typename AT = typename UTraits<UT>::acc>
__global__ void __launch_bounds__(256) apply2d_scatter(int nx, int ny, int bc, AT scale,
                                                       const short4 *__restrict__ offs,
                                                       const void *__restrict__ wbase, adlbr_dtype wt,
                                                       const UT *__restrict__ u, AT *__restrict__ Au) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const int64_t z = (int64_t)y * nx + x;
    const short4 o = offs[z];
    AT w[3];
    load_weights<AT, 3>(wbase, wt, z, w);
    const int ex[3] = {o.x, o.z, -o.x - o.z};
    const int ey[3] = {o.y, o.w, -o.y - o.w};
    const AT uz = to_acc(u[z]);
    AT acc = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const AT wk = scale * w[k];
        if (wk == (AT)0) continue;
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            int xn = x + s * ex[k], yn = y + s * ey[k];
            if (bc == ADLBR_PERIODIC) {
                xn = wrap(xn, nx);
                yn = wrap(yn, ny);
            } else if (xn < 0 || xn >= nx || yn < 0 || yn >= ny) {
                continue;
            }
            const int64_t zn = (int64_t)yn * nx + xn;
            const AT flux = wk * (uz - to_acc(u[zn]));
            acc += flux;
            red_add(Au + zn, -flux);
        }
    }
    red_add(Au + z, acc);
}

template <typename UT, typename AT = typename UTraits<UT>::acc>
__global__ void __launch_bounds__(128) apply3d_scatter(int nx, int ny, int nz, int bc, AT scale,
                                                       const char4 *__restrict__ offs,
                                                       const void *__restrict__ wbase, adlbr_dtype wt,
                                                       const UT *__restrict__ u, AT *__restrict__ Au) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zc = blockIdx.z;
    if (x >= nx) return;
    const int64_t z = ((int64_t)zc * ny + y) * nx + x;
    const char4 b[3] = {offs[3 * z], offs[3 * z + 1], offs[3 * z + 2]};
    int c[6][3];
    selling_offsets(b, c);
    AT w[6];
    load_weights<AT, 6>(wbase, wt, z, w);
    const AT uz = to_acc(u[z]);
    AT acc = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const AT wq = scale * w[q];
        if (wq == (AT)0) continue;
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            int xn = x + s * c[q][0], yn = y + s * c[q][1], zn = zc + s * c[q][2];
            if (bc == ADLBR_PERIODIC) {
                xn = wrap(xn, nx);
                yn = wrap(yn, ny);
                zn = wrap(zn, nz);
            } else if (xn < 0 || xn >= nx || yn < 0 || yn >= ny || zn < 0 || zn >= nz) {
                continue;
            }
            const int64_t zz = ((int64_t)zn * ny + yn) * nx + xn;
            const AT flux = wq * (uz - to_acc(u[zz]));
            acc += flux;
            red_add(Au + zz, -flux);
        }
    }
    red_add(Au + z, acc);
}

// u <- u - acc   (acc holds dt A u).  The accumulator is cleared by a
// separate memset before the next accumulation: a pass that rewrites both
// arrays in place runs at about a quarter of the HBM rate on this GPU, the
// two passes apart at nearly the full rate.
template <typename UT>
__global__ void finalize_kernel(int64_t N, UT *__restrict__ u,
                                const typename UTraits<UT>::acc *__restrict__ acc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    u[i] = from_acc<UT>(to_acc(u[i]) - acc[i]);
}

__global__ void finalize_f32x4_kernel(int64_t N4, float4 *__restrict__ u, const float4 *__restrict__ acc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N4) return;
    const float4 a = acc[i], v = u[i];
    u[i] = make_float4(v.x - a.x, v.y - a.y, v.z - a.z, v.w - a.w);
}

// ---- canonical export --------------------------------------------------
template <int DIM>
__device__ __forceinline__ bool canon_less(const int (&a)[DIM], const int (&b)[DIM]) {
#pragma unroll
    for (int t = 0; t < DIM; ++t)
        if (a[t] != b[t]) return a[t] < b[t];
    return false;
}

template <int DIM, int K, typename WO>
__device__ __forceinline__ void write_canonical(int (&v)[K][DIM], double (&w)[K], unsigned zmask,
                                                int16_t *offs, WO *wo, int64_t i) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (zmask >> k & 1u) {
#pragma unroll
            for (int t = 0; t < DIM; ++t) v[k][t] = 0;
            w[k] = 0.0;
            continue;
        }
        int sgn = 0;
#pragma unroll
        for (int t = DIM - 1; t >= 0; --t)
            if (v[k][t] != 0) sgn = v[k][t] < 0 ? -1 : 1;
        if (sgn < 0) {
#pragma unroll
            for (int t = 0; t < DIM; ++t) v[k][t] = -v[k][t];
        }
    }
    int idx[K];
#pragma unroll
    for (int k = 0; k < K; ++k) idx[k] = k;
    for (int a = 1; a < K; ++a)
        for (int bb = a; bb > 0 && canon_less<DIM>(v[idx[bb]], v[idx[bb - 1]]); --bb) {
            int t = idx[bb];
            idx[bb] = idx[bb - 1];
            idx[bb - 1] = t;
        }
    for (int k = 0; k < K; ++k) {
        for (int t = 0; t < DIM; ++t) offs[(i * K + k) * DIM + t] = (int16_t)v[idx[k]][t];
        wo[i * K + k] = (WO)w[idx[k]];
    }
}

template <typename WO>
__global__ void export2d_kernel(int64_t N, const short4 *__restrict__ offs, const void *wbase,
                                adlbr_dtype wt, int16_t *out_offs, WO *out_w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    short4 o = offs[i];
    int v[3][2] = {{o.x, o.y}, {o.z, o.w}, {-o.x - o.z, -o.y - o.w}};
    double w[3];
    unsigned zm = load_weights<double, 3>(wbase, wt, i, w);
    write_canonical<2, 3, WO>(v, w, zm, out_offs, out_w, i);
}

template <typename WO>
__global__ void export3d_kernel(int64_t N, const char4 *__restrict__ offs, const void *wbase,
                                adlbr_dtype wt, int16_t *out_offs, WO *out_w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const char4 b[3] = {offs[3 * i], offs[3 * i + 1], offs[3 * i + 2]};
    int c[6][3];
    selling_offsets(b, c);
    double w[6];
    unsigned zm = load_weights<double, 6>(wbase, wt, i, w);
    write_canonical<3, 6, WO>(c, w, zm, out_offs, out_w, i);
}

}  // namespace

adlbr_status launch_export(const adlbr_stencils *s, int16_t *offs, void *w, cudaStream_t st) {
    const int threads = 256;
    unsigned blocks = blocks_for(s->N, threads);
    if (s->dim == 2) {
        if (s->w_t == ADLBR_F64)
            export2d_kernel<double><<<blocks, threads, 0, st>>>(s->N, (const short4 *)s->offs, s->w,
                                                                s->w_t, offs, (double *)w);
        else
            export2d_kernel<float><<<blocks, threads, 0, st>>>(s->N, (const short4 *)s->offs, s->w,
                                                               s->w_t, offs, (float *)w);
    } else {
        if (s->w_t == ADLBR_F64)
            export3d_kernel<double><<<blocks, threads, 0, st>>>(s->N, (const char4 *)s->offs, s->w,
                                                                s->w_t, offs, (double *)w);
        else
            export3d_kernel<float><<<blocks, threads, 0, st>>>(s->N, (const char4 *)s->offs, s->w,
                                                               s->w_t, offs, (float *)w);
    }
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

// acc += scale * A u   (acc must hold zero or a partial sum on entry)
template <typename UT>
static adlbr_status accumulate_t(const adlbr_stencils *s, const UT *u, typename UTraits<UT>::acc *acc,
                                 double scale, const int *skip, cudaStream_t st) {
    using AT = typename UTraits<UT>::acc;
    if (s->dim == 2) {
        if constexpr (sizeof(AT) == 4) {
            constexpr int TW = 64, TH = 32, NT = 256, WX = 16;
            using T = Tile<TW, TH, NT, WX>;
            dim3 grid(blocks_for(s->n[0], TW), blocks_for(s->n[1], TH));
            constexpr size_t smem = 2 * T::P * T::WH * sizeof(float);
            if (s->w_t == ADLBR_F16)
                apply2d_tiled<UT, TW, TH, NT, WX, true><<<grid, NT, smem, st>>>(
                    (int)s->n[0], (int)s->n[1], s->bc, (float)scale, (const short4 *)s->offs, s->w,
                    s->w_t, u, acc, skip);
            else
                apply2d_tiled<UT, TW, TH, NT, WX, false><<<grid, NT, smem, st>>>(
                    (int)s->n[0], (int)s->n[1], s->bc, (float)scale, (const short4 *)s->offs, s->w,
                    s->w_t, u, acc, skip);
        } else {
            const int threads = 256;
            dim3 grid(blocks_for(s->n[0], threads), (unsigned)s->n[1]);
            apply2d_scatter<UT><<<grid, threads, 0, st>>>((int)s->n[0], (int)s->n[1], s->bc, (AT)scale,
                                                          (const short4 *)s->offs, s->w, s->w_t, u,
                                                          acc);
        }
    } else {
        const int threads = 128;
        dim3 grid(blocks_for(s->n[0], threads), (unsigned)s->n[1], (unsigned)s->n[2]);
        apply3d_scatter<UT><<<grid, threads, 0, st>>>((int)s->n[0], (int)s->n[1], (int)s->n[2],
                                                      s->bc, (AT)scale, (const char4 *)s->offs, s->w,
                                                      s->w_t, u, acc);
    }
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status launch_accumulate(const adlbr_stencils *s, const void *u, void *acc, adlbr_dtype u_t,
                               double scale, const int *skip, cudaStream_t st) {
    switch (u_t) {
    case ADLBR_F64: return accumulate_t<double>(s, (const double *)u, (double *)acc, scale, skip, st);
    case ADLBR_F32: return accumulate_t<float>(s, (const float *)u, (float *)acc, scale, skip, st);
    case ADLBR_F16: return accumulate_t<__half>(s, (const __half *)u, (float *)acc, scale, skip, st);
    case ADLBR_BF16:
        return accumulate_t<__nv_bfloat16>(s, (const __nv_bfloat16 *)u, (float *)acc, scale, skip, st);
    }
    return fail(ADLBR_E_ARG, "bad u dtype %d", (int)u_t);
}

adlbr_status launch_accumulate_f64(const adlbr_stencils *s, const float *u, double *acc, double scale,
                                   cudaStream_t st) {
    if (s->dim == 2) {
        const int threads = 256;
        dim3 grid(blocks_for(s->n[0], threads), (unsigned)s->n[1]);
        apply2d_scatter<float, double><<<grid, threads, 0, st>>>(
            (int)s->n[0], (int)s->n[1], s->bc, scale, (const short4 *)s->offs, s->w, s->w_t, u, acc);
    } else {
        const int threads = 128;
        dim3 grid(blocks_for(s->n[0], threads), (unsigned)s->n[1], (unsigned)s->n[2]);
        apply3d_scatter<float, double><<<grid, threads, 0, st>>>(
            (int)s->n[0], (int)s->n[1], (int)s->n[2], s->bc, scale, (const char4 *)s->offs, s->w,
            s->w_t, u, acc);
    }
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status launch_apply(const adlbr_stencils *s, const void *u, void *Au, adlbr_dtype u_t,
                          cudaStream_t st) {
    const size_t es = u_t == ADLBR_F64 ? sizeof(double) : sizeof(float);
    ADLBR_CUDA(cudaMemsetAsync(Au, 0, (size_t)s->N * es, st));
    return launch_accumulate(s, u, Au, u_t, 1.0, nullptr, st);
}

adlbr_status launch_finalize(const adlbr_stencils *s, void *u, void *acc, adlbr_dtype u_t,
                             cudaStream_t st) {
    const int threads = 256;
    unsigned blocks = blocks_for(s->N, threads);
    switch (u_t) {
    case ADLBR_F64:
        finalize_kernel<double><<<blocks, threads, 0, st>>>(s->N, (double *)u, (double *)acc);
        break;
    case ADLBR_F32:
        if (s->N % 4 == 0 && ((uintptr_t)u % 16) == 0 && ((uintptr_t)acc % 16) == 0)
            finalize_f32x4_kernel<<<blocks_for(s->N / 4, threads), threads, 0, st>>>(
                s->N / 4, (float4 *)u, (float4 *)acc);
        else
            finalize_kernel<float><<<blocks, threads, 0, st>>>(s->N, (float *)u, (float *)acc);
        break;
    case ADLBR_F16:
        finalize_kernel<__half><<<blocks, threads, 0, st>>>(s->N, (__half *)u, (float *)acc);
        break;
    case ADLBR_BF16:
        finalize_kernel<__nv_bfloat16><<<blocks, threads, 0, st>>>(s->N, (__nv_bfloat16 *)u,
                                                                   (float *)acc);
        break;
    default: return fail(ADLBR_E_ARG, "bad u dtype %d", (int)u_t);
    }
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace adlbr

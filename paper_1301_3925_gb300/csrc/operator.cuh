// The operator's per-tile and per-point device code (Eq. def:E*, h = 1),
// shared by the single-grid kernels (apply.cu) and the batched step
// (batch.cu).
//
// The operator is a sum over the directed edges (z, e), e in V(z), of
// gamma_z(e) (u(z) - u(z+e)) added at z and subtracted at z+e.  Pairs that
// leave the grid are dropped (Neumann rule of Sec. 1) or wrapped (periodic).
#pragma once

#include <type_traits>

#include "internal.cuh"
#include "stencil2d.cuh"
#include "tma.cuh"

namespace adlbr {
namespace op {

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
__device__ __forceinline__ void weights_f16_rec(uint2 r, float scale, float (&w)[3]) {
    const int s = (int)(int8_t)(r.y >> 24);
    const float c = __int_as_float((127 + s) << 23) * scale;
    w[0] = __uint_as_float((r.x & 0xffffu) << 13) * 0x1p112f * c;
    w[1] = __uint_as_float((r.x >> 16) << 13) * 0x1p112f * c;
    w[2] = __uint_as_float((r.y & 0xffffu) << 13) * 0x1p112f * c;
}
__device__ __forceinline__ void weights_f16_scaled(const void *wbase, int64_t z, float scale,
                                                   float (&w)[3]) {
    weights_f16_rec(reinterpret_cast<const uint2 *>(wbase)[z], scale, w);
}

// Where tile2d takes each point's stencil from: the handle's arrays (the
// operator), or the point's tensor, built on the spot and stored (the fused
// build and step; FP32 tensors, F16 weights).
struct LoadStencil {};
struct BuildStencil {
    const float *D;    // planes Dxx, Dxy, Dyy of N points
    int64_t N;
    short4 *offs;      // the handle's stencil storage
    void *w;
    bool warm;         // offs holds a previous build's stencils (a start for each point)
};

// acc += scale A u over the tile at (x0, y0); every thread of the block
// calls it (block-wide barriers inside).  offs3: the third offsets of a
// general (A-NN) stencil, nullptr for AD-LBR.  smem: 2 * WH * P floats, 16-byte
// aligned (128-byte for TMA).  TMA: the u window (FP32, non-periodic grid,
// nx % 4 == 0) arrives as one bulk tensor copy of the map's WW x WH box;
// cells outside the grid are zero-filled, as the plain staging leaves them.
// One thread waits for the copy (bounded) while the others sleep in the block
// barrier.  If the wait gives up, the block records ERRBIT_TIMEOUT in *err,
// waits up to four more bounds for the copy to land, and returns.
template <typename UT, int TW, int TH, int NT, int WX, bool F16W, bool TMA = false, typename Src = LoadStencil>
__device__ __forceinline__ void tile2d(int nx, int ny, int bc, float scale, const short4 *__restrict__ offs,
                                       const short2 *__restrict__ offs3, const void *__restrict__ wbase,
                                       adlbr_dtype wt,
                                       const UT *__restrict__ u, float *__restrict__ acc, int x0, int y0,
                                       float *smem, const CUtensorMap *map = nullptr, int *err = nullptr,
                                       const Src &src = Src()) {
    using T = Tile<TW, TH, NT, WX>;
    constexpr int WW = T::WW, WH = T::WH, P = T::P;
    constexpr bool BUILD = std::is_same<Src, BuildStencil>::value;
    float *uw = smem, *aw = smem + WH * P;
    __syncthreads();   // the window of a previous tile may still be read
    const bool periodic = bc == ADLBR_PERIODIC;
    // full: every point of the tile is in the grid; inside: every short edge
    // of the tile stays in the grid (or wraps, on a periodic grid)
    const bool full = x0 + TW <= nx && y0 + TH <= ny;
    const bool inside = periodic || (x0 >= HALO && y0 >= HALO && x0 + TW + HALO <= nx &&
                                     y0 + TH + HALO <= ny);
    if constexpr (TMA) {
        static_assert(T::P == WW && std::is_same<UT, float>::value, "TMA box = window rows");
        __shared__ uint64_t bar;
        if (threadIdx.x == 0) tma::bar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            tma::bar_expect_tx(&bar, WW * WH * sizeof(float));
            tma::load_2d(uw, map, x0 - HALO, y0 - HALO, &bar);
        }
        for (int c4 = threadIdx.x; c4 < WH * WW / 4; c4 += NT)
            *reinterpret_cast<float4 *>(&aw[c4 * 4]) = make_float4(0.f, 0.f, 0.f, 0.f);
        __shared__ int landed;
        if (!tma::bar_wait_block(&bar, 0, &landed)) {
            // the copy has not landed: record it, and wait longer before the
            // block leaves, so that it does not exit while its window is
            // still being written
            if (threadIdx.x == 0) {
                if (err) atomicOr(err, ERRBIT_TIMEOUT);
                for (int t = 0; t < 4; ++t)
                    if (tma::bar_wait(&bar, 0)) break;
            }
            __syncthreads();
            return;
        }
    } else {
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
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx = (warp % T::WARPS_X) * WX + lane % WX;
    const int ty = (warp / T::WARPS_X) * T::WR + lane / WX;
    const int x = x0 + tx;
    // two passes per loop trip for the operator; one with the build inside
    // (its body is long: 0.673 against 0.682 ms per CED step unrolled twice)
#pragma unroll (BUILD ? 1 : 2)
    for (int k = 0; k < T::PASSES; ++k) {
        const int ly = ty + k * T::WR * T::WARPS_Y, y = y0 + ly;
        if (!full && (x >= nx || y >= ny)) continue;
        const int64_t z = (int64_t)y * nx + x;
        short4 o;
        float w[3];
        if constexpr (BUILD) {
            // (loading the next pass's tensor one pass ahead measured no faster)
            static_assert(F16W, "the fused build stores F16 weights");
            const Built2 bt = build_point2d<float>(src.D[z], src.D[src.N + z], src.D[2 * src.N + z], z, src.offs,
                                                   src.w, ADLBR_F16, err, src.warm);
            o = bt.o;
            weights_f16_rec(bt.rec, scale, w);
        } else if (F16W) {
            o = offs[z];
            weights_f16_scaled(wbase, z, scale, w);
        } else {
            o = offs[z];
            load_weights<float, 3>(wbase, wt, z, w);
#pragma unroll
            for (int i = 0; i < 3; ++i) w[i] *= scale;
        }
        int ex[3], ey[3];
        offsets2d(o, offs3, z, ex, ey);
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
                    if (!in_bounds(zn, WH * P, err)) continue;
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
                    if (!in_bounds(zn, (int64_t)nx * ny, err)) continue;
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


// ---- 3D, shared-memory window --------------------------------------------
// A CTA of TX * TY threads owns a TX x TY x TZ block (one thread per (x, y),
// looping over z).  u is staged over the block plus a halo of H3 points (XL
// along x, so that window rows start on a 16-byte boundary) and pushes stay
// in a shared accumulator over the same window; 98% of the edges of the
// kappa = 20 needle stencils are at most 2 points long (Chebyshev).
constexpr int H3 = 2, XL = 4;

template <int TX, int TY, int TZ>
struct Block3 {
    static_assert(TX % 4 == 0, "whole float4 rows");
    static constexpr int WX = TX + 2 * XL, WY = TY + 2 * H3, WZ = TZ + 2 * H3;
    static constexpr int PX = WX;                     // row pitch
    static constexpr int PY = WY * PX;                // plane pitch
    static constexpr int CELLS = WZ * PY;
    static constexpr int H16 = TX + 16;                // staged 16-bit box width (x0 - 8 .. x0 + TX + 8)
    static constexpr int STAGE16 = H16 * WY * WZ;      // its cells (2 bytes each)
};

// Weights of 3D point z (8 lanes: six F16 weights and the meta lane) times
// `scale`, widened as in weights_f16_scaled.
__device__ __forceinline__ void weights6_f16_scaled(const void *wbase, int64_t z, float scale,
                                                    float (&w)[6]) {
    const uint4 r = reinterpret_cast<const uint4 *>(wbase)[z];
    const int s = (int)(int8_t)(r.w >> 8);
    const float c = __int_as_float((127 + s) << 23) * scale;
    const unsigned h[6] = {r.x & 0xffffu, r.x >> 16, r.y & 0xffffu, r.y >> 16, r.z & 0xffffu, r.z >> 16};
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = __uint_as_float(h[k] << 13) * 0x1p112f * c;
}

// acc += scale A u over the block at (x0, y0, z0); all TX * TY threads of
// the CTA call it.  smem: 2 * Block3::CELLS floats, 16-byte aligned (128 for
// TMA), plus Block3::STAGE16 halves for 16-bit u with TMA.  TMA: as in
// tile2d, the window (a WX x WY x WZ box) arrives by one bulk tensor copy on
// non-periodic grids: FP32 u straight into the window; 16-bit u (x from
// x0 - 8, a 16-byte boundary) into a staging box that is then widened.
template <typename UT, int TX, int TY, int TZ, bool F16W, bool TMA = false>
__device__ __forceinline__ void tile3d(int nx, int ny, int nz, int bc, float scale,
                                       const char4 *__restrict__ offs, const void *__restrict__ wbase,
                                       adlbr_dtype wt, const UT *__restrict__ u, float *__restrict__ acc,
                                       int x0, int y0, int z0, float *smem, const CUtensorMap *map = nullptr,
                                       int *err = nullptr) {
    using B = Block3<TX, TY, TZ>;
    constexpr int WY = B::WY, WZ = B::WZ, PX = B::PX, PY = B::PY;
    constexpr int NT = TX * TY;
    float *uw = smem, *aw = smem + B::CELLS;
    __syncthreads();   // the window of a previous block may still be read
    const bool periodic = bc == ADLBR_PERIODIC;
    const bool inside = periodic || (x0 >= H3 && y0 >= H3 && z0 >= H3 && x0 + TX + H3 <= nx &&
                                     y0 + TY + H3 <= ny && z0 + TZ + H3 <= nz);
    const int wx0 = x0 - XL;   // grid x of window column 0 (a multiple of 4)
    const int64_t nxy = (int64_t)nx * ny;
    constexpr int Q = PX / 4;   // float4s per window row
    if constexpr (TMA) {
        // FP32 u lands in the window itself; 16-bit u lands in a staging box
        // after the two windows (x from x0 - 8, a 16-byte boundary, H16 wide)
        // and is widened below
        constexpr bool F32U = std::is_same<UT, float>::value;
        static_assert(F32U || sizeof(UT) == 2, "TMA windows: FP32 or 16-bit u");
        uint16_t *st16 = reinterpret_cast<uint16_t *>(smem + 2 * B::CELLS);
        __shared__ uint64_t bar;
        if (threadIdx.x == 0) tma::bar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            if constexpr (F32U) {
                tma::bar_expect_tx(&bar, B::CELLS * sizeof(float));
                tma::load_3d(uw, map, wx0, y0 - H3, z0 - H3, &bar);
            } else {
                tma::bar_expect_tx(&bar, B::H16 * WY * WZ * 2);
                tma::load_3d(st16, map, x0 - 8, y0 - H3, z0 - H3, &bar);
            }
        }
        for (int c4 = threadIdx.x; c4 < B::CELLS / 4; c4 += NT)
            *reinterpret_cast<float4 *>(&aw[c4 * 4]) = make_float4(0.f, 0.f, 0.f, 0.f);
        __shared__ int landed;
        if (!tma::bar_wait_block(&bar, 0, &landed)) {
            // the copy has not landed: record it, and wait longer before the
            // block leaves, so that it does not exit while its window is
            // still being written
            if (threadIdx.x == 0) {
                if (err) atomicOr(err, ERRBIT_TIMEOUT);
                for (int t = 0; t < 4; ++t)
                    if (tma::bar_wait(&bar, 0)) break;
            }
            __syncthreads();
            return;
        }
        if constexpr (!F32U) {
            // widen: window column wx is staged column wx + 8 - XL
            for (int c = threadIdx.x; c < B::CELLS; c += NT) {
                const int row = c / PX, wx = c - row * PX;
                const uint16_t h = st16[row * B::H16 + wx + 8 - XL];
                uw[c] = to_acc(*reinterpret_cast<const UT *>(&h));
            }
            __syncthreads();
        }
    } else {
    // stage u (4 cells per step), zero the accumulator
    const bool vec = std::is_same<UT, float>::value && (nx % 4) == 0 && !periodic &&
                     ((uintptr_t)u % 16) == 0;
    for (int c4 = threadIdx.x; c4 < WZ * WY * Q; c4 += NT) {
        const int wz = c4 / (WY * Q), rem = c4 - wz * (WY * Q);
        const int wy = rem / Q, wx = (rem - wy * Q) * 4;
        const int gz = z0 - H3 + wz, gy = y0 - H3 + wy, gx = wx0 + wx;
        float v[4];
        if (vec && (unsigned)gz < (unsigned)nz && (unsigned)gy < (unsigned)ny && gx >= 0 && gx + 3 < nx) {
            const float4 q = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(u) +
                                                               gz * nxy + (int64_t)gy * nx + gx);
            v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                int xx = gx + t, yy = gy, zz = gz;
                v[t] = 0.f;
                if (periodic) {
                    xx = wrap(xx, nx);
                    yy = wrap(yy, ny);
                    zz = wrap(zz, nz);
                } else if ((unsigned)xx >= (unsigned)nx || (unsigned)yy >= (unsigned)ny ||
                           (unsigned)zz >= (unsigned)nz) {
                    continue;
                }
                v[t] = to_acc(u[zz * nxy + (int64_t)yy * nx + xx]);
            }
        }
        const int o = wz * PY + wy * PX + wx;
        *reinterpret_cast<float4 *>(&uw[o]) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(&aw[o]) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    }
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x = x0 + tx, y = y0 + ty;
    if (x < nx && y < ny) {
#pragma unroll 2
        for (int k = 0; k < TZ; ++k) {
            const int zc = z0 + k;
            if (zc >= nz) break;
            const int64_t z = zc * nxy + (int64_t)y * nx + x;
            const char4 b[3] = {offs[3 * z], offs[3 * z + 1], offs[3 * z + 2]};
            int c[6][3];
            selling_offsets(b, c);
            float w[6];
            if (F16W) {
                weights6_f16_scaled(wbase, z, scale, w);
            } else {
                load_weights<float, 6>(wbase, wt, z, w);
#pragma unroll
                for (int q = 0; q < 6; ++q) w[q] *= scale;
            }
            const int zw = (k + H3) * PY + (ty + H3) * PX + tx + XL;
            const float uz = uw[zw];
            float own = 0.f;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float wq = w[q];
                if (abs(c[q][0]) <= H3 && abs(c[q][1]) <= H3 && abs(c[q][2]) <= H3) {
                    const int d = c[q][2] * PY + c[q][1] * PX + c[q][0];
#pragma unroll
                    for (int sg = -1; sg <= 1; sg += 2) {
                        if (!inside) {
                            const int xn = x + sg * c[q][0], yn = y + sg * c[q][1], zn = zc + sg * c[q][2];
                            if ((unsigned)xn >= (unsigned)nx || (unsigned)yn >= (unsigned)ny ||
                                (unsigned)zn >= (unsigned)nz)
                                continue;
                        }
                        const int zn = zw + sg * d;
                        if (!in_bounds(zn, B::CELLS, err)) continue;
                        const float f = wq * (uz - uw[zn]);
                        own += f;
                        atomicAdd(&aw[zn], -f);
                    }
                } else if (wq != 0.f) {
#pragma unroll
                    for (int sg = -1; sg <= 1; sg += 2) {
                        int xn = x + sg * c[q][0], yn = y + sg * c[q][1], zn = zc + sg * c[q][2];
                        if (periodic) {
                            xn = wrap(xn, nx);
                            yn = wrap(yn, ny);
                            zn = wrap(zn, nz);
                        } else if ((unsigned)xn >= (unsigned)nx || (unsigned)yn >= (unsigned)ny ||
                                   (unsigned)zn >= (unsigned)nz) {
                            continue;
                        }
                        const int64_t zz = zn * nxy + (int64_t)yn * nx + xn;
                        if (!in_bounds(zz, nxy * nz, err)) continue;
                        const float f = wq * (uz - to_acc(u[zz]));
                        own += f;
                        red_add(acc + zz, -f);
                    }
                }
            }
            atomicAdd(&aw[zw], own);
        }
    }
    __syncthreads();
    // flush the window (4 cells per step)
    const bool vec_ok = (nx % 4) == 0 && ((uintptr_t)acc % 16) == 0;
    for (int c4 = threadIdx.x; c4 < WZ * WY * Q; c4 += NT) {
        const int wz = c4 / (WY * Q), rem = c4 - wz * (WY * Q);
        const int wy = rem / Q, wx = (rem - wy * Q) * 4;
        const float4 v = *reinterpret_cast<const float4 *>(&aw[wz * PY + wy * PX + wx]);
        if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
        int gz = z0 - H3 + wz, gy = y0 - H3 + wy;
        const int gx = wx0 + wx;
        if (periodic) {
            gz = wrap(gz, nz);
            gy = wrap(gy, ny);
        } else if ((unsigned)gz >= (unsigned)nz || (unsigned)gy >= (unsigned)ny) {
            continue;
        }
        float *row = acc + gz * nxy + (int64_t)gy * nx;
        if (vec_ok && !periodic && gx >= 0 && gx + 3 < nx) {
            red_add_v4(row + gx, v.x, v.y, v.z, v.w);
        } else {
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (vv[t] == 0.f) continue;
                int xx = gx + t;
                if (periodic) xx = wrap(xx, nx);
                else if (xx < 0 || xx >= nx) continue;
                red_add(row + xx, vv[t]);
            }
        }
    }
}

// Point (x, y, zc) of a 3D grid: its own edges into a register, the
// opposite contributions and the own sum pushed to Au in L2.
template <typename UT, typename AT>
__device__ __forceinline__ void point3d(int nx, int ny, int nz, int bc, AT scale, const char4 *__restrict__ offs,
                                        const void *__restrict__ wbase, adlbr_dtype wt,
                                        const UT *__restrict__ u, AT *__restrict__ Au, int x, int y, int zc,
                                        int *err = nullptr) {
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
            if (!in_bounds(zz, (int64_t)nx * ny * nz, err)) continue;
            const AT flux = wq * (uz - to_acc(u[zz]));
            acc += flux;
            red_add(Au + zz, -flux);
        }
    }
    red_add(Au + z, acc);
}

}  // namespace op
}  // namespace adlbr

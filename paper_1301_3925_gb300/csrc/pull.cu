// Gather ("pull") form of the 2D operator A u = (1/2) grad E_h(u) (Eq. def:E*,
// h = 1), for stencils with F16 weights that are applied more than once.
//
// The operator is a sum over the directed edges (y, e), e in V(y) = {+-e_i(y)},
// each adding gamma_y(e) (u(y) - u(y+e)) at y and the opposite at y + e
// (pairs leaving the grid dropped, Sec. 1, or wrapped).  Row z of A therefore
// holds z's own six edges and the edges of other points that end at z.  Most
// of the latter are reciprocal: when the neighbour y = z + d (d = +-e_i(z))
// has +-d among its own superbase offsets, at slot j, the pair (z, y) carries
// the two weights w_i(z) + w_j(y) in both rows.  The remaining incoming
// edges -- y -> z with d = z - y not in V(z) -- are listed per point
// ("extras").
//
// So every row is a gather and the result is written once, with no atomic
// operation and no pre-zeroed output.  A one-off table moves all weight
// bookkeeping out of the application: each point's record holds its own
// three weights and, per direction, the reciprocal neighbour weight w_j(y),
// all as F16 values at the point's own power-of-two scale; each extra holds
// its source offset and weight the same way.  A neighbour weight is an F16
// value at the neighbour's scale, so it is exact at the point's scale unless
// it falls below the F16 normal range there (a weight under 2^-14 of the
// point's largest, rounded to the nearest F16 subnormal).  The gather thus
// computes the scatter's operator up to the order of the FP32 additions.
//
// Table (built once per stencil set, pull_build):
//   recw[z]  uint4: halves w0, w1, w2 (z's weights), rho0..rho4;
//   reco[z]  uint2: x = rho5 | (int8 scale exponent s_z) << 16 | count << 24,
//                   y = the superbase offsets e0, e1 as four int8 (e2 = -e0-e1);
//            rho_q, q = 2 i + (s < 0), is the weight of the pair (z, z + s e_i)
//            in the neighbour's stencil (0 if it has no such offset); value
//            = half * 2^s_z.
//   ext[]    the extras, one uint32 each: int8 dx, int8 dy (source z + d),
//            the source's weight as a half at z's scale in bits 16..31;
//            stored point after point in grid order, each point's list sorted
//            (deterministic).
//   seg[s]   index in ext of the first extra of row segment s (32 points of a
//            row, x = 32 k .. 32 k + 31); seg[nseg] = total.
#include <cuda.h>

#include <cstring>
#include <new>
#include <type_traits>

#include "internal.cuh"
#include "tma.cuh"

namespace adlbr {

namespace {

constexpr int SEG = 32;          // points per row segment (one warp)
constexpr int SCAN_T = 256;      // scan block: threads
constexpr int SCAN_I = 16;       //             items per thread
constexpr int SCAN_B = SCAN_T * SCAN_I;

// pull flags (device word of the table)
constexpr int PF_RANGE = 1;      // an offset coordinate beyond the int8 range
constexpr int PF_COUNT = 2;      // a point with more than 255 extras

__device__ __forceinline__ int wrapc(int c, int n) {
    c %= n;
    return c < 0 ? c + n : c;
}

// Is +-(dx, dy) one of the superbase offsets of o (e0, e1, e2 = -e0-e1)?
// Returns the slot or 3.
__device__ __forceinline__ int slot_of(short4 o, int dx, int dy) {
    const int f[3][2] = {{o.x, o.y}, {o.z, o.w}, {-o.x - o.z, -o.y - o.w}};
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if ((f[j][0] == dx && f[j][1] == dy) || (f[j][0] == -dx && f[j][1] == -dy)) return j;
    return 3;
}

// F16 weight record of a point (3 halves, meta: zero mask, scale exponent)
__device__ __forceinline__ unsigned rec_half(uint2 r, int j) {
    return j == 0 ? (r.x & 0xffffu) : (j == 1 ? (r.x >> 16) : (r.y & 0xffffu));
}
__device__ __forceinline__ int rec_exp(uint2 r) { return (int)(int8_t)(r.y >> 24); }
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((127 + s) << 23); }
// weight j of y re-expressed as a half at scale 2^s (exact when representable)
__device__ __forceinline__ unsigned half_at_scale(uint2 ry, int j, int s) {
    const float v = h2f_bits((uint16_t)rec_half(ry, j));       // weight / 2^s_y
    const int d = rec_exp(ry) - s;                               // |d| <= 240
    const float t = __fmul_rn(__fmul_rn(v, pow2f(d / 2)), pow2f(d - d / 2));
    return f2h_bits(t);
}

// Pass 1, one thread per point z: the record (own weights, reciprocal
// weights, offsets), and one count at every neighbour that must list one of
// z's edges as an extra.
__global__ void __launch_bounds__(256) pull_records2d(int nx, int ny, int periodic, const short4 *__restrict__ offs,
                                                      const uint2 *__restrict__ w, uint4 *__restrict__ recw,
                                                      uint2 *__restrict__ reco, uint8_t *__restrict__ pushm,
                                                      int *__restrict__ cnt, int *flag) {
    const int64_t N = (int64_t)nx * ny;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int y = (int)(i / nx), x = (int)(i - (int64_t)y * nx);
    const short4 o = offs[i];
    const int e[3][2] = {{o.x, o.y}, {o.z, o.w}, {-o.x - o.z, -o.y - o.w}};
    bool fits = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) fits = fits && abs(e[k][0]) <= 127 && abs(e[k][1]) <= 127;
    if (!fits) atomicOr(flag, PF_RANGE);
    const uint2 wr = w[i];
    const int sz = rec_exp(wr);
    const unsigned zm = (wr.y >> 16) & 0xffu;
    unsigned rho[6], push = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        rho[q] = 0;
        const int k = q >> 1, s = (q & 1) ? -1 : 1;
        const int dx = s * e[k][0], dy = s * e[k][1];
        int xn = x + dx, yn = y + dy;
        if (periodic) {
            xn = wrapc(xn, nx);
            yn = wrapc(yn, ny);
        } else if ((unsigned)xn >= (unsigned)nx || (unsigned)yn >= (unsigned)ny) {
            continue;
        }
        const int64_t zn = (int64_t)yn * nx + xn;
        const int j = slot_of(offs[zn], dx, dy);
        if (j != 3) {
            rho[q] = half_at_scale(w[zn], j, sz);
        } else if (!((zm >> k) & 1u)) {
            push |= 1u << q;
            atomicAdd(&cnt[zn], 1);
        }
    }
    recw[i] = make_uint4(wr.x, (wr.y & 0xffffu) | rho[0] << 16, rho[1] | rho[2] << 16, rho[3] | rho[4] << 16);
    const unsigned px = (unsigned)(uint8_t)(int8_t)e[0][0] | (unsigned)(uint8_t)(int8_t)e[0][1] << 8 |
                        (unsigned)(uint8_t)(int8_t)e[1][0] << 16 | (unsigned)(uint8_t)(int8_t)e[1][1] << 24;
    reco[i] = make_uint2(rho[5] | (unsigned)(uint8_t)(int8_t)sz << 16, px);
    pushm[i] = (uint8_t)push;
}

// Exclusive scan of cnt, part 1: every block scans SCAN_B consecutive counts
// and writes its total.
__global__ void __launch_bounds__(SCAN_T) scan_blocks(int64_t N, const int *__restrict__ cnt,
                                                      uint32_t *__restrict__ start, uint32_t *__restrict__ blk) {
    __shared__ uint32_t wsum[SCAN_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_I;
    uint32_t v[SCAN_I], tot = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        v[k] = base + k < N ? (uint32_t)cnt[base + k] : 0u;
        tot += v[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t wpre = 0, btot = 0;
    for (int k = 0; k < SCAN_T / 32; ++k) {
        if (k < w) wpre += wsum[k];
        btot += wsum[k];
    }
    uint32_t run = wpre + inc - tot;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        if (base + k < N) start[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) blk[blockIdx.x] = btot;
}

// Part 2: exclusive scan of the block totals (one block); blk[nb] = total.
__global__ void __launch_bounds__(1024) scan_top(int nb, uint32_t *blk) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? blk[b] : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int k = 0; k < 32; ++k) {
            if (k < w) wpre += wsum[k];
            tot += wsum[k];
        }
        const uint32_t c = carry;
        if (b < nb) blk[b] = c + wpre + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) blk[nb] = carry;
}

// Part 3: final starts; the count goes into the record and the segment
// starts are written.
__global__ void __launch_bounds__(256) scan_finish(int nx, int64_t N, int nb, uint32_t *__restrict__ start,
                                                   const uint32_t *__restrict__ blk, const int *__restrict__ cnt,
                                                   uint2 *__restrict__ reco, uint32_t *__restrict__ seg, int nseg_x,
                                                   int *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) seg[(int64_t)nseg_x * (N / nx)] = blk[nb];
    if (i >= N) return;
    const uint32_t s = start[i] + blk[i / SCAN_B];
    start[i] = s;
    const int c = cnt[i];
    if (c > 255) atomicOr(flag, PF_COUNT);
    reco[i].x |= (uint32_t)min(c, 255) << 24;
    const int y = (int)(i / nx), x = (int)(i - (int64_t)y * nx);
    if (x % SEG == 0) seg[(int64_t)y * nseg_x + x / SEG] = s;
}

// Pass 2, one thread per source y: writes each of y's push edges, with its
// weight at the far end's scale, into the far end's list (cnt counts down to
// zero again).
__global__ void __launch_bounds__(256) pull_fill2d(int nx, int ny, int periodic, const short4 *__restrict__ offs,
                                                   const uint2 *__restrict__ w, const uint8_t *__restrict__ pushm,
                                                   const uint32_t *__restrict__ start, int *__restrict__ cnt,
                                                   uint32_t *__restrict__ ext, int64_t cap) {
    const int64_t N = (int64_t)nx * ny;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned push = pushm[i];
    if (!push) return;
    const int y = (int)(i / nx), x = (int)(i - (int64_t)y * nx);
    const short4 o = offs[i];
    const uint2 wr = w[i];
    const int e[3][2] = {{o.x, o.y}, {o.z, o.w}, {-o.x - o.z, -o.y - o.w}};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (!((push >> q) & 1u)) continue;
        const int k = q >> 1, s = (q & 1) ? -1 : 1;
        const int dx = s * e[k][0], dy = s * e[k][1];
        int xn = x + dx, yn = y + dy;
        if (periodic) {
            xn = wrapc(xn, nx);
            yn = wrapc(yn, ny);
        }
        const int64_t zn = (int64_t)yn * nx + xn;
        const int64_t pos = (int64_t)start[zn] + atomicSub(&cnt[zn], 1) - 1;
        if (pos < 0 || pos >= cap) continue;   // only with an unusable table (flagged)
        const unsigned h = half_at_scale(wr, k, rec_exp(w[zn]));
        ext[pos] = (uint32_t)(uint8_t)(int8_t)(-dx) | (uint32_t)(uint8_t)(int8_t)(-dy) << 8 | h << 16;
    }
}

// Pass 3: each point's list in ascending order (the fill order depends on
// atomic scheduling; the sorted order does not).
__global__ void __launch_bounds__(256) pull_sort(int64_t N, const uint2 *__restrict__ reco,
                                                 const uint32_t *__restrict__ start, uint32_t *__restrict__ ext) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = (int)(reco[i].x >> 24);
    if (n < 2) return;
    uint32_t *p = ext + start[i];
    for (int a = 1; a < n; ++a) {
        const uint32_t v = p[a];
        int b = a - 1;
        while (b >= 0 && p[b] > v) {
            p[b + 1] = p[b];
            --b;
        }
        p[b + 1] = v;
    }
}

// ---------------------------------------------------------------- gather
constexpr int H = 8;   // window halo (points): 95% of the kappa <= 100 CED edges fit

// half bits -> float (exact; every table half is finite)
__device__ __forceinline__ float hf(unsigned h) { return __uint_as_float((h & 0xffffu) << 13) * 0x1p112f; }

template <int TW, int TH, int NT>
struct PullTile {
    static constexpr int WW = TW + 2 * H, WH = TH + 2 * H;
    static constexpr int CELLS = WW * WH;
    static constexpr int NW = NT / 32;          // warps
    static constexpr int SX = TW / 32;          // warps across the tile
    static constexpr int RG = NW / SX;          // row groups
    static constexpr int PASSES = TH / RG;      // rows per warp
    static constexpr int LQ = 64;               // long-edge queue per warp
    // shared-memory room for the tile's extras: 3.5 per point (the CED
    // stencils have 2.1 on average); a tile with more reads them from L2
    static constexpr int EXT_CAP = TW * TH * 7 / 2;
    static_assert(TW % 32 == 0 && NW % SX == 0 && TH % RG == 0 && TH <= 32 && PASSES <= 16, "tile");
    static constexpr size_t SMEM = (size_t)CELLS * 4 + (size_t)EXT_CAP * 4 + (size_t)NW * PASSES * 32 * 4 +
                                   (size_t)NW * LQ * 8;
};

// 1D bulk copy global -> shared completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tma::smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(tma::smem_u32(bar))
        : "memory");
}

// The term of a long edge (beyond the halo) of point (xt, y): own direction q
// (extra == false) or the extra entry v; in units of the point's weight
// scale (the caller multiplies by 2^s_z).
template <typename UT>
__device__ __forceinline__ float long_term(int nx, int ny, int periodic, const uint4 *__restrict__ recw,
                                           const uint2 *__restrict__ reco, const UT *__restrict__ u, int xt, int y,
                                           float uz, bool extra, uint32_t v, int q, int *err) {
    int dx, dy;
    float c;
    const int64_t z = (int64_t)y * nx + xt;
    if (extra) {
        dx = (int)(int8_t)(v & 0xffu);
        dy = (int)(int8_t)((v >> 8) & 0xffu);
        c = hf(v >> 16);
    } else {
        const uint4 rw = recw[z];
        const uint2 ro = reco[z];
        const int i = q >> 1;
        const int e0 = (int)(int8_t)(ro.y & 0xffu), f0 = (int)(int8_t)((ro.y >> 8) & 0xffu);
        const int e1 = (int)(int8_t)((ro.y >> 16) & 0xffu), f1 = (int)(int8_t)(ro.y >> 24);
        const int ex = i == 0 ? e0 : (i == 1 ? e1 : -e0 - e1), ey = i == 0 ? f0 : (i == 1 ? f1 : -f0 - f1);
        dx = (q & 1) ? -ex : ex;
        dy = (q & 1) ? -ey : ey;
        const unsigned wi = i == 0 ? rw.x : (i == 1 ? rw.x >> 16 : rw.y);
        const unsigned rq = q == 0 ? rw.y >> 16
                          : q == 1 ? rw.z
                          : q == 2 ? rw.z >> 16
                          : q == 3 ? rw.w
                          : q == 4 ? rw.w >> 16
                                   : ro.x;
        c = hf(wi) + hf(rq);
    }
    int xn = xt + dx, yn = y + dy;
    if (periodic) {
        xn = wrapc(xn, nx);
        yn = wrapc(yn, ny);
    }
    const int64_t zn = (int64_t)yn * nx + xn;
    if (!in_bounds(zn, (int64_t)nx * ny, err)) return 0.f;
    return c * (uz - to_acc(u[zn]));
}

// out[z] = a u(z) + b (A u)(z) over a TW x TH tile per CTA.
//  * Staged in shared memory before any arithmetic: u over the tile plus an
//    H-point halo (one TMA copy for FP32 u on a non-periodic grid, else
//    plain loads) and the tile's extras (one bulk copy per tile row).
//  * A warp covers 32 consecutive points of a row per pass: each point adds
//    its six pair terms (own weight + reciprocal weight) and its extras.
//  * Terms whose neighbour lies beyond the halo go to a per-warp queue and
//    are evaluated together after the last pass, so that a warp waits for L2
//    once per tile rather than once per row.
template <typename UT, typename OT, int TW, int TH, int NT, bool TMA>
__global__ void __launch_bounds__(NT, 4) pull2d_kernel(int nx, int ny, int periodic, const uint4 *__restrict__ recw,
                                                       const uint2 *__restrict__ reco,
                                                       const uint32_t *__restrict__ ext,
                                                       const uint32_t *__restrict__ seg, int nseg_x, int64_t n_ext,
                                                       const UT *__restrict__ u, OT *__restrict__ out, float a, float b,
                                                       const int *__restrict__ skip,
                                                       const __grid_constant__ CUtensorMap umap, int *err) {
    using PT = PullTile<TW, TH, NT>;
    constexpr int WW = PT::WW, SX = PT::SX, RG = PT::RG, PASSES = PT::PASSES, LQ = PT::LQ;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *uw = reinterpret_cast<float *>(smem_raw);                           // WH x WW values
    uint32_t *xs = reinterpret_cast<uint32_t *>(uw + PT::CELLS);               // the tile's extras
    float *lacc = reinterpret_cast<float *>(xs + PT::EXT_CAP);                 // [warp][pass][lane]
    uint2 *lq = reinterpret_cast<uint2 *>(lacc + PT::NW * PASSES * 32);        // [warp][LQ]
    __shared__ uint64_t bar;
    __shared__ int row_off[TH];       // per tile row: position of its extras in xs, minus
    __shared__ uint32_t row_a[TH];    // the index in ext of the first one copied
    __shared__ int ext_global;        // the tile's extras did not fit: read them from L2
    __shared__ int lq_n[PT::NW];
    if (skip && *skip) return;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cx0 = (warp % SX) * 32, ry = warp / SX;
    const int cx = cx0 + lane, x = x0 + cx;
    if (warp == 0) {
        // the extras of tile row `lane` are ext[seg[s0] .. seg[s1]), copied
        // from a 16-byte aligned start with a size rounded up to 16 bytes
        uint32_t a0 = 0, n = 0;
        const int yr = y0 + lane;
        if (lane < TH && yr < ny) {
            const int64_t s0 = (int64_t)yr * nseg_x + x0 / SEG;
            const int64_t s1 = min(s0 + TW / SEG, (int64_t)(yr + 1) * nseg_x);
            a0 = seg[s0] & ~3u;
            n = ((seg[s1] + 3u) & ~3u) - a0;
        }
        uint32_t inc = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        const bool fits = total <= (uint32_t)PT::EXT_CAP;
        if (lane < TH) {
            row_off[lane] = (int)(inc - n);
            row_a[lane] = a0;
        }
        if (lane == 0) {
            ext_global = fits ? 0 : 1;
            tma::bar_init(&bar, 1);
            const unsigned win = TMA ? PT::CELLS * 4u : 0u;
            tma::bar_expect_tx(&bar, win + (fits ? total * 4u : 0u));
            if constexpr (TMA) tma::load_2d(uw, &umap, x0 - H, y0 - H, &bar);
        }
        __syncwarp();
        if (fits && n > 0) bulk_load(xs + (inc - n), ext + a0, n * 4u, &bar);
    }
    if (lane == 0) lq_n[warp] = 0;
    if constexpr (!TMA) {
        for (int c = threadIdx.x; c < PT::CELLS; c += NT) {
            const int wy = c / WW, wx = c - wy * WW;
            int gx = x0 - H + wx, gy = y0 - H + wy;
            bool in = true;
            if (periodic) {
                gx = wrapc(gx, nx);
                gy = wrapc(gy, ny);
            } else {
                in = (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny;
            }
            uw[c] = in ? to_acc(u[(int64_t)gy * nx + gx]) : 0.f;
        }
    }
    // the first pass's records and segment start (later ones one pass ahead)
    uint4 rwn = make_uint4(0u, 0u, 0u, 0u);
    uint2 ron = make_uint2(0u, 0u);
    uint32_t sbn = 0;
    {
        const int y = y0 + ry;
        if (x < nx && y < ny) {
            rwn = recw[(int64_t)y * nx + x];
            ron = reco[(int64_t)y * nx + x];
        }
        if (y < ny) sbn = seg[(int64_t)y * nseg_x + (x0 + cx0) / SEG];
    }
    __syncthreads();   // barrier initialised, row table, queue counts and plain staging visible
    __shared__ int landed;
    if (!tma::bar_wait_block(&bar, 0, &landed)) {
        // a copy has not landed: record it, and wait longer before the block
        // leaves, so that it does not exit while its shared memory is still
        // being written
        if (threadIdx.x == 0) {
            if (err) atomicOr(err, ERRBIT_TIMEOUT);
            for (int t = 0; t < 4; ++t)
                if (tma::bar_wait(&bar, 0)) break;
        }
        __syncthreads();
        return;
    }
    const bool from_l2 = ext_global != 0;
    // every short own edge of every point stays in the grid (or wraps)
    const bool inside = periodic || (x0 >= H && y0 >= H && x0 + TW + H <= nx && y0 + TH + H <= ny);
    float *myacc = lacc + warp * PASSES * 32;
    uint2 *myq = lq + warp * LQ;
#pragma unroll 1
    for (int k = 0; k < PASSES; ++k) {
        const int ly = ry + k * RG, y = y0 + ly;
        const uint4 rw = rwn;
        const uint2 ro = ron;
        const uint32_t sb = sbn;
        if (k + 1 < PASSES) {   // next pass's records and segment start
            const int y1 = y + RG;
            if (x < nx && y1 < ny) {
                rwn = recw[(int64_t)y1 * nx + x];
                ron = reco[(int64_t)y1 * nx + x];
            }
            sbn = y1 < ny ? seg[(int64_t)y1 * nseg_x + (x0 + cx0) / SEG] : 0u;
        }
        if (y >= ny) break;   // warp-uniform
        const unsigned cnt = ro.x >> 24;
        uint32_t pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += t;
        }
        float acc = 0.f;
        if (x < nx) {
            const int zw = (ly + H) * WW + cx + H;
            const float uz = uw[zw];
            const float w[3] = {hf(rw.x), hf(rw.x >> 16), hf(rw.y)};
            const float rho[6] = {hf(rw.y >> 16), hf(rw.z), hf(rw.z >> 16), hf(rw.w), hf(rw.w >> 16), hf(ro.x)};
            const int e0 = (int)(int8_t)(ro.y & 0xffu), f0 = (int)(int8_t)((ro.y >> 8) & 0xffu);
            const int e1 = (int)(int8_t)((ro.y >> 16) & 0xffu), f1 = (int)(int8_t)(ro.y >> 24);
            const int ox[3] = {e0, e1, -e0 - e1}, oy[3] = {f0, f1, -f0 - f1};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const bool shrt = abs(ox[i]) <= H && abs(oy[i]) <= H;
                const int lin = oy[i] * WW + ox[i];
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int q = 2 * i + s;
                    const int dx = s ? -ox[i] : ox[i], dy = s ? -oy[i] : oy[i];
                    if (!(inside && shrt) && !periodic &&
                        ((unsigned)(x + dx) >= (unsigned)nx || (unsigned)(y + dy) >= (unsigned)ny))
                        continue;   // the pair leaves the grid (Neumann)
                    if (shrt) {
                        if (!in_bounds(zw + (s ? -lin : lin), PT::CELLS, err)) continue;
                        acc = __fmaf_rn(w[i] + rho[q], uz - uw[zw + (s ? -lin : lin)], acc);
                    } else {
                        const int slot = atomicAdd(&lq_n[warp], 1);
                        if (slot < LQ)
                            myq[slot] = make_uint2((uint32_t)k << 26 | (uint32_t)lane << 21 | (uint32_t)q, 0u);
                        else
                            acc += long_term<UT>(nx, ny, periodic, recw, reco, u, x, y, uz, false, 0u, q, err);
                    }
                }
            }
            const uint32_t eg = sb + pre - cnt;
            const int es = row_off[ly] + (int)(eg - row_a[ly]);
            for (unsigned t = 0; t < cnt; ++t) {
                if (!(from_l2 ? in_bounds((int64_t)eg + t, n_ext, err) : in_bounds(es + (int)t, PT::EXT_CAP, err)))
                    continue;
                const uint32_t v = from_l2 ? ext[eg + t] : xs[es + t];
                const int dx = (int)(int8_t)(v & 0xffu), dy = (int)(int8_t)((v >> 8) & 0xffu);
                if (abs(dx) <= H && abs(dy) <= H) {
                    if (!in_bounds(zw + dy * WW + dx, PT::CELLS, err)) continue;
                    acc = __fmaf_rn(hf(v >> 16), uz - uw[zw + dy * WW + dx], acc);
                } else {
                    const int slot = atomicAdd(&lq_n[warp], 1);
                    if (slot < LQ)
                        myq[slot] = make_uint2(0x80000000u | (uint32_t)k << 26 | (uint32_t)lane << 21, v);
                    else
                        acc += long_term<UT>(nx, ny, periodic, recw, reco, u, x, y, uz, true, v, 0, err);
                }
            }
            acc *= pow2f((int)(int8_t)((ro.x >> 16) & 0xffu));   // the point's weight scale
        }
        myacc[k * 32 + lane] = acc;
    }
    __syncwarp();
    // the queued long-edge terms, one per lane
    const int nq = min(lq_n[warp], LQ);
    for (int i = lane; i < nq; i += 32) {
        const uint2 item = myq[i];
        const int k = (item.x >> 26) & 15, tl = (item.x >> 21) & 31;
        const int ly = ry + k * RG, y = y0 + ly, xt = x0 + cx0 + tl;
        const float uz = uw[(ly + H) * WW + cx0 + tl + H];
        const float t = long_term<UT>(nx, ny, periodic, recw, reco, u, xt, y, uz, (item.x >> 31) != 0, item.y,
                                      (int)(item.x & 7u), err);
        const int sz = (int)(int8_t)((reco[(int64_t)y * nx + xt].x >> 16) & 0xffu);
        atomicAdd(&myacc[k * 32 + tl], t * pow2f(sz));
    }
    __syncwarp();
    // write the rows
#pragma unroll 1
    for (int k = 0; k < PASSES; ++k) {
        const int ly = ry + k * RG, y = y0 + ly;
        if (y >= ny) break;
        if (x < nx)
            out[(int64_t)y * nx + x] =
                from_acc<OT>(__fmaf_rn(b, myacc[k * 32 + lane], a * uw[(ly + H) * WW + cx + H]));
    }
}

constexpr int PTW = 64, PTH = 32, PNT = 256;

template <typename UT, typename OT>
adlbr_status launch_pull_u(const adlbr_stencils *s, const UT *u, OT *out, float a, float b, const int *skip,
                           cudaStream_t st) {
    using PT = PullTile<PTW, PTH, PNT>;
    const PullTable &T = *s->pull;
    const int nx = (int)s->n[0], ny = (int)s->n[1];
    const size_t smem = PT::SMEM;
    dim3 grid(blocks_for(nx, PTW), blocks_for(ny, PTH));
    CUtensorMap um;
    memset(&um, 0, sizeof(um));
    const bool tma_ok = std::is_same<UT, float>::value && s->bc != ADLBR_PERIODIC &&
                        tma::encode_2d_f32(&um, reinterpret_cast<const float *>(u), nx, ny, PT::WW, PT::WH);
    if (tma_ok) {
        auto k = pull2d_kernel<UT, OT, PTW, PTH, PNT, true>;
        static bool attr = false;
        if (!attr) {
            ADLBR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = true;
        }
        k<<<grid, PNT, smem, st>>>(nx, ny, 0, T.recw, T.reco, T.ext, T.seg, T.nseg_x, T.cap + 4, u, out, a, b,
                                   skip, um, s->err);
    } else {
        auto k = pull2d_kernel<UT, OT, PTW, PTH, PNT, false>;
        static bool attr = false;
        if (!attr) {
            ADLBR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = true;
        }
        k<<<grid, PNT, smem, st>>>(nx, ny, s->bc == ADLBR_PERIODIC, T.recw, T.reco, T.ext, T.seg, T.nseg_x,
                                   T.cap + 4, u, out, a, b, skip, um, s->err);
    }
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace

// ---------------------------------------------------------------- host side
bool pull_supported(const adlbr_stencils *s) {
    // extras are counted in uint32: at most 6 per point
    return s->dim == 2 && s->scheme == ADLBR_SCHEME_ADLBR && s->w_t == ADLBR_F16 && s->N <= (int64_t)1 << 29;
}

void pull_free(adlbr_stencils *s) {
    PullTable *T = s->pull;
    if (!T) return;
    cudaFree(T->recw);
    cudaFree(T->reco);
    cudaFree(T->ext);
    cudaFree(T->seg);
    cudaFree(T->cnt);
    cudaFree(T->start);
    cudaFree(T->blk);
    cudaFree(T->pushm);
    cudaFree(T->flag);
    cudaFreeHost(T->flag_host);
    delete T;
    s->pull = nullptr;
}

adlbr_status pull_build(adlbr_stencils *s, cudaStream_t st) {
    if (!pull_supported(s)) return fail(ADLBR_E_ARG, "the gather form needs a 2D handle with F16 weights");
    const int64_t N = s->N;
    const int nx = (int)s->n[0], ny = (int)s->n[1];
    PullTable *T = s->pull;
    if (!T) {
        T = new (std::nothrow) PullTable();
        if (!T) return fail(ADLBR_E_INTERNAL, "out of host memory");
        s->pull = T;
        T->nseg_x = (nx + SEG - 1) / SEG;
        T->nseg = (int64_t)T->nseg_x * ny;
        T->cap = 6 * N;
        T->nblk = (int)((N + SCAN_B - 1) / SCAN_B);
        cudaError_t e = cudaMalloc(&T->recw, N * sizeof(uint4));
        if (e == cudaSuccess) e = cudaMalloc(&T->reco, N * sizeof(uint2));
        if (e == cudaSuccess) e = cudaMalloc(&T->ext, (T->cap + 4) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&T->seg, (T->nseg + 1) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&T->cnt, N * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&T->start, N * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&T->blk, (T->nblk + 1) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&T->pushm, N);
        if (e == cudaSuccess) e = cudaMalloc(&T->flag, sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&T->flag_host, sizeof(int));
        if (e != cudaSuccess) {
            pull_free(s);
            return cuda_fail(e, "allocating the gather table");
        }
    }
    T->built = false;
    T->usable = false;
    ADLBR_CUDA(cudaMemsetAsync(T->cnt, 0, N * sizeof(int), st));
    ADLBR_CUDA(cudaMemsetAsync(T->flag, 0, sizeof(int), st));
    const int periodic = s->bc == ADLBR_PERIODIC;
    const unsigned nb = blocks_for(N, 256);
    const short4 *offs = (const short4 *)s->offs;
    const uint2 *w = (const uint2 *)s->w;
    pull_records2d<<<nb, 256, 0, st>>>(nx, ny, periodic, offs, w, T->recw, T->reco, T->pushm, T->cnt, T->flag);
    scan_blocks<<<T->nblk, SCAN_T, 0, st>>>(N, T->cnt, T->start, T->blk);
    scan_top<<<1, 1024, 0, st>>>(T->nblk, T->blk);
    scan_finish<<<nb, 256, 0, st>>>(nx, N, T->nblk, T->start, T->blk, T->cnt, T->reco, T->seg, T->nseg_x, T->flag);
    pull_fill2d<<<nb, 256, 0, st>>>(nx, ny, periodic, offs, w, T->pushm, T->start, T->cnt, T->ext, T->cap);
    pull_sort<<<nb, 256, 0, st>>>(N, T->reco, T->start, T->ext);
    ADLBR_CUDA(cudaGetLastError());
    ADLBR_CUDA(cudaMemcpyAsync(T->flag_host, T->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    ADLBR_CUDA(cudaStreamSynchronize(st));
    T->built = true;
    T->usable = *T->flag_host == 0;
    return ADLBR_OK;
}

bool pull_ready(const adlbr_stencils *s) { return s->pull && s->pull->built && s->pull->usable; }

// out = a u + b A u through the gather form (pull_ready(s) must hold).
adlbr_status launch_pull(const adlbr_stencils *s, const void *u, adlbr_dtype u_t, void *out, adlbr_dtype out_t,
                         double a, double b, const int *skip, cudaStream_t st) {
    ADLBR_NVTX("operator");
    const float fa = (float)a, fb = (float)b;
    if (out_t == ADLBR_F32) {
        switch (u_t) {
        case ADLBR_F32: return launch_pull_u<float, float>(s, (const float *)u, (float *)out, fa, fb, skip, st);
        case ADLBR_F16: return launch_pull_u<__half, float>(s, (const __half *)u, (float *)out, fa, fb, skip, st);
        case ADLBR_BF16:
            return launch_pull_u<__nv_bfloat16, float>(s, (const __nv_bfloat16 *)u, (float *)out, fa, fb, skip, st);
        default: break;
        }
    } else if (out_t == u_t) {
        switch (u_t) {
        case ADLBR_F16: return launch_pull_u<__half, __half>(s, (const __half *)u, (__half *)out, fa, fb, skip, st);
        case ADLBR_BF16:
            return launch_pull_u<__nv_bfloat16, __nv_bfloat16>(s, (const __nv_bfloat16 *)u, (__nv_bfloat16 *)out,
                                                               fa, fb, skip, st);
        default: break;
        }
    }
    return fail(ADLBR_E_ARG, "gather form: unsupported vector types %d -> %d", (int)u_t, (int)out_t);
}

adlbr_status choose_gather(adlbr_stencils *s, int uses, bool *gather, cudaStream_t st) {
    *gather = false;
    s->applies_since_build += uses;
    // the scatter form is the default (ADLBR_OP_AUTO): it measured faster on
    // every workload; the gather form runs when it is asked for
    if (s->op_form != ADLBR_OP_GATHER || !pull_supported(s)) return ADLBR_OK;
    if (!(s->pull && s->pull->built))
        if (adlbr_status e = pull_build(s, st)) return e;
    *gather = s->pull->usable;
    return ADLBR_OK;
}

adlbr_status launch_operator(adlbr_stencils *s, const void *u, adlbr_dtype u_t, void *out, double a, double b,
                             cudaStream_t st) {
    bool gather = false;
    if (u_t != ADLBR_F64)
        if (adlbr_status e = choose_gather(s, 1, &gather, st)) return e;
    if (gather) return launch_pull(s, u, u_t, out, ADLBR_F32, a, b, nullptr, st);
    const size_t es = u_t == ADLBR_F64 ? sizeof(double) : sizeof(float);
    if (a == 0.0) {
        ADLBR_CUDA(cudaMemsetAsync(out, 0, (size_t)s->N * es, st));
    } else if (a == 1.0 && (u_t == ADLBR_F64 || u_t == ADLBR_F32)) {
        ADLBR_CUDA(cudaMemcpyAsync(out, u, (size_t)s->N * es, cudaMemcpyDeviceToDevice, st));
    } else {
        return fail(ADLBR_E_INTERNAL, "scatter operator: unsupported initial term");
    }
    return launch_accumulate(s, u, out, u_t, b, nullptr, st);
}

}  // namespace adlbr

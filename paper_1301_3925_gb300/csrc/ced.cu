// Coherence-enhancing diffusion (Sec. 4.4, Eq. parabolique): the tensor
// stage D(J_rho(grad u_sigma)),
//   u_sigma = K_sigma * u,  J_rho = K_rho * (grad u_sigma grad u_sigma^T),
//   D = alpha v1 v1^T + lambda2 v2 v2^T,
//   lambda2 = alpha + (1 - alpha) exp(-C / (mu1 - mu2)^2),
// followed (adlbr_ced_stencils) by the AD-LBR stencil construction of D.
//
// sigma and rho are standard deviations; kernels are truncated at
// int(3 s + 0.5) and normalised; every stage reflects its own input about the
// border (u(-1) = u(0)): the Gaussians and the centred-difference gradient.
//
// Kernels: one fused tile kernel (all stages in shared memory, below), and
// the separable form it reproduces bit for bit, used where the fused windows
// do not fit: Gaussian passes staged through shared memory (a row segment
// plus halo for the x pass, a column band plus halo for the y pass), the
// gradient and outer product in one pass, and the 2x2 eigen-decomposition
// fused into the epilogue of the last (y) pass.
#include <algorithm>
#include <type_traits>
#include <cstdlib>
#include <cstring>

#include "ced_common.cuh"
#include "stencil2d.cuh"

namespace adlbr {

using ced::d_from_j;
using ced::kMaxR;
using ced::make_taps;
using ced::radius_of;
using ced::reflect;
using ced::Taps;

namespace {

// Each thread produces RB consecutive outputs along the blur direction from
// RB + 2r staged values (register blocking), so a 25-tap pass reads about
// 7 values from shared memory per output instead of 25.
constexpr int RB = 4;
constexpr int TXT = 128;            // x pass: threads per block
constexpr int TX = TXT * RB;        // x pass: outputs per block (one row segment)

// out[c][y][x] = sum_k taps[|k|] in[c][y][reflect(x + k)]
template <int C>
__global__ void __launch_bounds__(TXT) blur_x_kernel(int nx, int ny, int64_t N, int r, Taps tp,
                                                     const float *__restrict__ in,
                                                     float *__restrict__ out) {
    extern __shared__ float smx[];  // C * (TX + 2r)
    const int x0 = blockIdx.x * TX, y = blockIdx.y;
    const int W = TX + 2 * r;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *row = in + c * N + (int64_t)y * nx;
        for (int j = threadIdx.x; j < W; j += TXT) smx[c * W + j] = row[reflect(x0 - r + j, nx)];
    }
    __syncthreads();
    const int xb = x0 + RB * threadIdx.x;
    if (xb >= nx) return;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *s = smx + c * W + RB * threadIdx.x + r;  // s[j] = in[xb + j]
        float acc[RB];
#pragma unroll
        for (int o = 0; o < RB; ++o) acc[o] = __fmul_rn(tp.t[0], s[o]);
        for (int k = 1; k <= r; ++k) {
            float lo[RB], hi[RB];
#pragma unroll
            for (int o = 0; o < RB; ++o) {
                lo[o] = s[o - k];
                hi[o] = s[o + k];
            }
#pragma unroll
            for (int o = 0; o < RB; ++o) acc[o] = __fmaf_rn(tp.t[k], __fadd_rn(lo[o], hi[o]), acc[o]);
        }
        float *dst = out + c * N + (int64_t)y * nx + xb;
#pragma unroll
        for (int o = 0; o < RB; ++o)
            if (xb + o < nx) dst[o] = acc[o];
    }
}

constexpr int BX = 32, BY = 32;  // y pass tile; 8 rows of threads, RB rows each

// y pass; EPI 0: plain store; EPI 1: the channels are (Jxx, Jxy, Jyy) and the
// epilogue writes D(J) (three planes) instead.
template <int C, int EPI>
__global__ void __launch_bounds__(BX * 8) blur_y_kernel(int nx, int ny, int64_t N, int r, Taps tp,
                                                        const float *__restrict__ in,
                                                        float *__restrict__ out, float alpha,
                                                        float Cc) {
    extern __shared__ float smy[];  // C * (BY + 2r) * BX
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int H = BY + 2 * r;
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int x = x0 + tx;
    const bool xin = x < nx;
#pragma unroll
    for (int c = 0; c < C; ++c)
        for (int j = ty; j < H; j += 8) {
            int yy = reflect(y0 - r + j, ny);
            smy[(c * H + j) * BX + tx] = xin ? in[c * N + (int64_t)yy * nx + x] : 0.f;
        }
    __syncthreads();
    if (!xin) return;
    const int oy0 = RB * ty;  // this thread's rows: oy0 .. oy0 + RB - 1
    float v[C][RB];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *s = smy + (c * H + oy0 + r) * BX + tx;  // s[j * BX] = row oy0 + j
#pragma unroll
        for (int o = 0; o < RB; ++o) v[c][o] = __fmul_rn(tp.t[0], s[o * BX]);
        for (int k = 1; k <= r; ++k) {
            float lo[RB], hi[RB];
#pragma unroll
            for (int o = 0; o < RB; ++o) {
                lo[o] = s[(o - k) * BX];
                hi[o] = s[(o + k) * BX];
            }
#pragma unroll
            for (int o = 0; o < RB; ++o) v[c][o] = __fmaf_rn(tp.t[k], __fadd_rn(lo[o], hi[o]), v[c][o]);
        }
    }
#pragma unroll
    for (int o = 0; o < RB; ++o) {
        const int y = y0 + oy0 + o;
        if (y >= ny) break;
        const int64_t z = (int64_t)y * nx + x;
        if (EPI == 0) {
#pragma unroll
            for (int c = 0; c < C; ++c) out[c * N + z] = v[c][o];
        } else {
            float dxx, dxy, dyy;
            d_from_j(v[0][o], v[1][o], v[2][o], alpha, Cc, dxx, dxy, dyy);
            out[z] = dxx;
            out[N + z] = dxy;
            out[2 * N + z] = dyy;
        }
    }
}

// (gx^2, gx gy, gy^2) of the centred differences of us, reflected border.
__global__ void grad_outer_kernel(int nx, int ny, int64_t N, const float *__restrict__ us,
                                  float *__restrict__ P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const float *row = us + (int64_t)y * nx;
    const float gx = __fmul_rn(0.5f, __fsub_rn(row[reflect(x + 1, nx)], row[reflect(x - 1, nx)]));
    const float gy = __fmul_rn(0.5f, __fsub_rn(us[(int64_t)reflect(y + 1, ny) * nx + x],
                                                us[(int64_t)reflect(y - 1, ny) * nx + x]));
    const int64_t z = (int64_t)y * nx + x;
    P[z] = __fmul_rn(gx, gx);
    P[N + z] = __fmul_rn(gx, gy);
    P[2 * N + z] = __fmul_rn(gy, gy);
}

adlbr_status separable_tensor(int nx, int ny, const float *u, float *D, int rs, int rr, const Taps &ts,
                             const Taps &tr, float alpha, float C, void *scratch, cudaStream_t st) {
    const int64_t N = (int64_t)nx * ny;
    float *A = (float *)scratch;  // 3N
    float *B = A + 3 * N;         // 3N
    dim3 gx(blocks_for(nx, TX), ny), gy(blocks_for(nx, BX), blocks_for(ny, BY));
    blur_x_kernel<1><<<gx, TXT, (TX + 2 * rs) * sizeof(float), st>>>(nx, ny, N, rs, ts, u, A);
    blur_y_kernel<1, 0><<<gy, BX * 8, (BY + 2 * rs) * BX * sizeof(float), st>>>(nx, ny, N, rs, ts, A,
                                                                                   B, 0.f, 0.f);
    grad_outer_kernel<<<dim3(blocks_for(nx, 256), ny), 256, 0, st>>>(nx, ny, N, B, A);
    blur_x_kernel<3><<<gx, TXT, 3 * (TX + 2 * rr) * sizeof(float), st>>>(nx, ny, N, rr, tr, A, B);
    size_t smy = 3 * (BY + 2 * rr) * BX * sizeof(float);
    ADLBR_CUDA(cudaFuncSetAttribute(blur_y_kernel<3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smy));
    blur_y_kernel<3, 1><<<gy, BX * 8, smy, st>>>(nx, ny, N, rr, tr, B, D, alpha, C);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

// ---- fused tile kernel ---------------------------------------------------
// One CTA computes D on a FT x FT output tile from a u tile with a halo of
// R + S + 1 (R, S the radii of K_rho, K_sigma), all intermediate planes in
// shared memory:
//   u (reflected loads) -x-> bx -y-> u_sigma -grad, outer-> P -x-> Px -y, D(J)-> D.
// Every value is computed with the operations, in the order, of the
// separable kernels above, and every plane is held on an extended window
// whose cells outside the grid carry the value the separable kernels would
// read there (their reflected index): for the symmetric blurs of reflected
// inputs this holds by construction (the taps pair the same two values); P,
// whose xy component is odd about the border, is evaluated at the reflected
// cell.  So the fused kernel reproduces the separable result bit for bit.
// Tiles are full: the last tile of a row or column is shifted back into the
// grid (its overlap with the previous tile is recomputed and rewritten with
// the same values).
constexpr int FT = 64;
// Threads per CTA: 768 (24 warps) for compile-time radii, whose register
// windows fit in 85 registers (measured 0.287 against 0.304 ms with 512 at
// 4096^2, sigma 1, rho 4); 512 for the run-time-radius form, whose windows are
// sized for the largest radius.
template <int S_, int R_>
constexpr int fused_threads() { return S_ > 0 && R_ > 0 ? 768 : 512; }

// Window geometry for radii (R, S): P window PH x PW (pitch PP), u_sigma
// window SH x SW, x-blurred u BH x BW, u window UH x UW; odd pitches keep the
// lanes of the x passes (one row each) on distinct banks.
struct FusedGeom {
    int R, S, PH, PW, PP, SH, SW, SP, BH, BW, BP, UH, UW, UP, XP, nU, offB, offU1, offP;
    size_t bytes;
};

__host__ __device__ constexpr FusedGeom fused_geom(int R, int S) {
    FusedGeom g{};
    g.R = R, g.S = S;
    g.PH = g.PW = FT + 2 * R, g.PP = g.PW | 1;
    g.SH = g.SW = g.PW + 2, g.SP = g.SW | 1;
    g.BH = g.SH + 2 * S, g.BW = g.SW, g.BP = g.BW | 1;
    g.UH = g.BH, g.UW = g.SW + 2 * S, g.UP = g.UW | 1;
    g.XP = FT + 1;
    // layout [U0][B][U1][P]: the u window of the next tile loads into one U
    // buffer while the other serves as u, then u_sigma, and Px spans it and B
    // (both orders are contiguous)
    int nU = g.UH * g.UP > g.SH * g.SP ? g.UH * g.UP : g.SH * g.SP;
    const int nB = g.BH * g.BP, nP = 3 * g.PH * g.PP, nX = 3 * g.PH * g.XP;
    if (nU + nB < nX) nU = nX - nB;
    g.nU = nU, g.offB = nU, g.offU1 = nU + nB, g.offP = 2 * nU + nB;
    g.bytes = (size_t)(g.offP + nP) * sizeof(float);
    return g;
}

// One output group of a symmetric blur: RB consecutive outputs from the
// RB + 2r values v (v[r + o] is the centre of output o), in the operation
// order of the separable kernels.
template <int RR, int NB = RB>
__device__ __forceinline__ void blur_group(const float (&v)[NB + 2 * RR], const Taps &tp, int r,
                                           float (&acc)[NB]) {
#pragma unroll
    for (int o = 0; o < NB; ++o) acc[o] = __fmul_rn(tp.t[0], v[RR + o]);
#pragma unroll
    for (int k = 1; k <= RR; ++k) {
        if (k > r) break;
#pragma unroll
        for (int o = 0; o < NB; ++o) acc[o] = __fmaf_rn(tp.t[k], __fadd_rn(v[RR + o - k], v[RR + o + k]), acc[o]);
    }
}

// rows per thread in the last (y) pass of the run-time-radius form (512
// groups); the compile-time form gives every one of its 768 threads one
// group of 6 or 5 rows (0.2585 against 0.262 ms with 512 groups of 8)
constexpr int RBY = 8;
// outputs per thread in the first three passes of the fused kernel: 8 reads
// 2r + 8 staged values per 8 outputs (0.267 against 0.286 ms with 4 at
// 4096^2, sigma 1, rho 4; 16 in the P x pass alone: 0.269)
constexpr int RBF = 8;
// outputs per thread in the two sigma passes with compile-time radii: 12,
// so that the x pass has exactly one 12-column group per thread (96 rows x 8
// groups = 768) and the y pass one round (90 columns x 8 groups); with 8,
// half the threads took a second group while the rest waited at the
// barrier (0.262 against 0.270 ms at 4096^2, bit-identical)
constexpr int RBS_FIXED = 12;

// S_, R_ > 0: radii fixed at compile time (all loops unrolled, windows in
// registers, constant index arithmetic); 0: taken from g at run time, with
// the register windows sized for the largest radius kMaxR.
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Asynchronous copy of the (reflected) u window of the tile at (x0, y0), in
// kParts parts issued between the passes of the previous tile (part = -1:
// all at once).  Interior windows are split by rows; a window that needs
// reflection is copied whole by part 0.  The last part commits the group.
constexpr int kParts = 4;
template <int S_, int R_>
__device__ __forceinline__ void load_u_window(const FusedGeom &g, int nx, int ny, int x0, int y0,
                                              const float *__restrict__ u, float *U, int part = -1) {
    const int uox = x0 - g.R - 1 - g.S, uoy = y0 - g.R - 1 - g.S;
    const bool interior = uox >= 0 && uoy >= 0 && uox + g.UW <= nx && uoy + g.UH <= ny;
    constexpr int FNT = fused_threads<S_, R_>();
    if (interior) {
        // no reflection: a warp per row, each lane copying every 32nd column
        // from one row base (constant offsets, no per-element index math:
        // 0.249 against 0.260 ms at 4096^2, sigma 1, rho 4)
        const int r0 = part < 0 ? 0 : part * g.UH / kParts, r1 = part < 0 ? g.UH : (part + 1) * g.UH / kParts;
        for (int r = r0 + threadIdx.x / 32; r < r1; r += FNT / 32) {
            const float *src = u + (int64_t)(uoy + r) * nx + uox;
            float *dst = U + r * g.UP;
#pragma unroll 4
            for (int c = threadIdx.x % 32; c < g.UW; c += 32) cp_async4(dst + c, src + c);
        }
        if (part < 0 || part == kParts - 1) cp_async_commit();
        return;
    }
    if (part > 0) return;
    for (int i = threadIdx.x; i < g.UH * g.UW; i += FNT) {
        const int r = i / g.UW, c = i - r * g.UW;
        const int gy = reflect(uoy + r, ny);
        const int gx = reflect(uox + c, nx);
        cp_async4(U + r * g.UP + c, u + (int64_t)gy * nx + gx);
    }
    cp_async_commit();
}

// S_, R_ > 0: radii fixed at compile time (all loops unrolled, windows in
// registers, constant index arithmetic); 0: taken from g at run time, with
// the register windows sized for the largest radius kMaxR.
// Persistent: CTA b processes tiles b, b + gridDim.x, ...; the u window of
// the next tile is copied asynchronously while the current one is computed.
template <int S_, int R_>
__global__ void __launch_bounds__(fused_threads<S_, R_>(), 1) ced_fused_kernel(int nx, int ny, int64_t N, FusedGeom gr, Taps ts,
                                                           Taps tr, const float *__restrict__ u,
                                                           float *__restrict__ D, float alpha, float Cc) {
    constexpr bool fixed = S_ > 0 && R_ > 0;
    constexpr int FNT = fused_threads<S_, R_>();
    constexpr FusedGeom gc = fused_geom(R_ > 0 ? R_ : 1, S_ > 0 ? S_ : 1);
    const FusedGeom &g = fixed ? gc : gr;
    constexpr int SR = fixed ? S_ : kMaxR, RR = fixed ? R_ : kMaxR;   // register window radii
    extern __shared__ float sm[];
    float *B = sm + g.offB, *P = sm + g.offP;
    const int R = g.R, S = g.S;
    const int tiles_x = (nx + FT - 1) / FT, tiles = tiles_x * ((ny + FT - 1) / FT);
    int tile = blockIdx.x;
    if (tile >= tiles) return;
    auto origin = [&](int t, int &x0, int &y0) {
        x0 = min((t % tiles_x) * FT, nx - FT);
        y0 = min((t / tiles_x) * FT, ny - FT);
    };
    {
        int x0, y0;
        origin(tile, x0, y0);
        load_u_window<S_, R_>(g, nx, ny, x0, y0, u, sm);
    }
    for (int it = 0; tile < tiles; tile += gridDim.x, ++it) {
    float *U = (it & 1) ? sm + g.offU1 : sm;
    float *US = U, *PX = (it & 1) ? B : sm;   // u_sigma over u; Px over u and bx
    int x0, y0;
    origin(tile, x0, y0);
    // window origins (grid coordinates of local (0, 0))
    const int pox = x0 - R, poy = y0 - R;            // P
    const int sox = pox - 1, soy = poy - 1;          // u_sigma; bx has its columns
    const int uox = sox - S, uoy = soy - S;          // u; bx has its rows
    const bool interior = uox >= 0 && uoy >= 0 && uox + g.UW <= nx && uoy + g.UH <= ny;
    cp_async_wait_all();
    __syncthreads();   // u of this tile is in place; the previous tile is done
    // the next tile's window, copied in parts between the passes below
    const bool has_next = tile + (int)gridDim.x < tiles;
    int nx0 = 0, ny0 = 0;
    if (has_next) origin(tile + gridDim.x, nx0, ny0);
    float *Un = (it & 1) ? sm : sm + g.offU1;
    auto next_part = [&](int k) {
        if (has_next) load_u_window<S_, R_>(g, nx, ny, nx0, ny0, u, Un, k);
    };
    next_part(0);
    constexpr int RBS = fixed ? RBS_FIXED : RBF;
    // 2. bx = x pass of u (lanes along rows, RBS outputs per thread)
    {
        const int groups = (g.BW + RBS - 1) / RBS;
        for (int i = threadIdx.x; i < g.BH * groups; i += FNT) {
            const int r = i % g.BH, c0 = (i / g.BH) * RBS;
            const float *s = U + r * g.UP + c0 + S - SR;
            float v[RBS + 2 * SR], acc[RBS];
#pragma unroll
            for (int j = 0; j < RBS + 2 * SR; ++j) v[j] = (fixed || (j >= SR - S && j < SR + S + RBS)) ? s[j] : 0.f;
            blur_group<SR, RBS>(v, ts, S, acc);
#pragma unroll
            for (int o = 0; o < RBS; ++o)
                if (c0 + o < g.BW) B[r * g.BP + c0 + o] = acc[o];
        }
    }
    __syncthreads();
    next_part(1);
    // 3. u_sigma = y pass of bx (lanes along columns, RBS rows per thread)
    {
        const int groups = (g.SH + RBS - 1) / RBS;
        for (int i = threadIdx.x; i < g.SW * groups; i += FNT) {
            const int c = i % g.SW, r0 = (i / g.SW) * RBS;
            const float *s = B + (r0 + S - SR) * g.BP + c;
            float v[RBS + 2 * SR], acc[RBS];
#pragma unroll
            for (int j = 0; j < RBS + 2 * SR; ++j)
                v[j] = (fixed || (j >= SR - S && j < SR + S + RBS)) ? s[j * g.BP] : 0.f;
            blur_group<SR, RBS>(v, ts, S, acc);
#pragma unroll
            for (int o = 0; o < RBS; ++o)
                if (r0 + o < g.SH) US[(r0 + o) * g.SP + c] = acc[o];
        }
    }
    __syncthreads();
    next_part(2);
    // 4. P = outer product of the centred differences, at the reflected cell
    if (fixed && interior && g.PW * (g.PH / 11) <= FNT && g.PH % 11 == 0) {
        // no reflection: P cell (r, c) is u_sigma cell (r + 1, c + 1); each
        // thread walks 11 rows of one column, keeping the two u_sigma values
        // above the current row in registers (fewer instructions than the
        // indexed loop; no time change measured at 4096^2)
        if (threadIdx.x < g.PW * (g.PH / 11)) {
            const int c = threadIdx.x % g.PW, r0 = (threadIdx.x / g.PW) * 11;
            const float *s = US + r0 * g.SP + c + 1;
            float up = s[0], mid = s[g.SP];
#pragma unroll
            for (int j = 0; j < 11; ++j) {
                const float *m = s + (j + 1) * g.SP;
                const float down = m[g.SP];
                const float gx = __fmul_rn(0.5f, __fsub_rn(m[1], m[-1]));
                const float gy = __fmul_rn(0.5f, __fsub_rn(down, up));
                const int r = r0 + j;
                P[r * g.PP + c] = __fmul_rn(gx, gx);
                P[(g.PH + r) * g.PP + c] = __fmul_rn(gx, gy);
                P[(2 * g.PH + r) * g.PP + c] = __fmul_rn(gy, gy);
                up = mid;
                mid = down;
            }
        }
    } else {
    for (int i = threadIdx.x; i < g.PH * g.PW; i += FNT) {
        const int r = i / g.PW, c = i - r * g.PW;
        const int ly = (interior ? poy + r : reflect(poy + r, ny)) - soy;
        const int lx = (interior ? pox + c : reflect(pox + c, nx)) - sox;
        const float *s = US + ly * g.SP + lx;
        const float gx = __fmul_rn(0.5f, __fsub_rn(s[1], s[-1]));
        const float gy = __fmul_rn(0.5f, __fsub_rn(s[g.SP], s[-g.SP]));
        P[r * g.PP + c] = __fmul_rn(gx, gx);
        P[(g.PH + r) * g.PP + c] = __fmul_rn(gx, gy);
        P[(2 * g.PH + r) * g.PP + c] = __fmul_rn(gy, gy);
    }
    }
    __syncthreads();
    next_part(3);
    // 5. Px = x pass of P over the FT output columns (lanes along rows)
    {
        constexpr int groups = FT / RBF;
        for (int i = threadIdx.x; i < g.PH * groups; i += FNT) {
            const int r = i % g.PH, c0 = (i / g.PH) * RBF;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float *s = P + (ch * g.PH + r) * g.PP + c0 + R - RR;
                float v[RBF + 2 * RR], acc[RBF];
#pragma unroll
                for (int j = 0; j < RBF + 2 * RR; ++j)
                    v[j] = (fixed || (j >= RR - R && j < RR + R + RBF)) ? s[j] : 0.f;
                blur_group<RR, RBF>(v, tr, R, acc);
#pragma unroll
                for (int o = 0; o < RBF; ++o) PX[(ch * g.PH + r) * g.XP + c0 + o] = acc[o];
            }
        }
    }
    __syncthreads();
    // 6. y pass of Px and D(J) (lanes along columns, NB rows per thread)
    {
        auto y_group = [&](auto nb, int c, int r0) {
            constexpr int NB = decltype(nb)::value;
            float J[3][NB];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float *s = PX + (ch * g.PH + r0 + R - RR) * g.XP + c;
                float v[NB + 2 * RR];
#pragma unroll
                for (int j = 0; j < NB + 2 * RR; ++j)
                    v[j] = (fixed || (j >= RR - R && j < RR + R + NB)) ? s[j * g.XP] : 0.f;
                blur_group<RR, NB>(v, tr, R, J[ch]);
            }
#pragma unroll
            for (int o = 0; o < NB; ++o) {
                const int64_t z = (int64_t)(y0 + r0 + o) * nx + x0 + c;
                float dxx, dxy, dyy;
                d_from_j(J[0][o], J[1][o], J[2][o], alpha, Cc, dxx, dxy, dyy);
                D[z] = dxx;
                D[N + z] = dxy;
                D[2 * N + z] = dyy;
            }
        };
        if constexpr (fixed && FNT == 768 && FT == 64) {
            // every thread takes one group: warps 0-7 six rows each (rows
            // 0..23), warps 8-23 five rows each (rows 24..63)
            if (threadIdx.x < 256)
                y_group(std::integral_constant<int, 6>(), threadIdx.x % FT, (threadIdx.x / FT) * 6);
            else
                y_group(std::integral_constant<int, 5>(), (threadIdx.x - 256) % FT,
                        24 + ((threadIdx.x - 256) / FT) * 5);
        } else {
            constexpr int groups = FT / RBY;
            for (int i = threadIdx.x; i < FT * groups; i += FNT)
                y_group(std::integral_constant<int, RBY>(), i % FT, (i / FT) * RBY);
        }
    }
    }
}

// Kernel choice: the fused tile kernel where it applies, else the separable
// passes.  ADLBR_CED_PATH=separable in the environment forces the separable
// passes (the two are bit-identical; the tests compare them).
int ced_path() {
    const char *e = getenv("ADLBR_CED_PATH");
    return (e && strcmp(e, "separable") == 0) ? 1 : 0;
}

// The fused kernel needs full tiles, reflections that stay inside the
// windows (grid sides >= FT) and windows that fit in shared memory.
bool fused_ok(int nx, int ny, int R, int S) {
    if (nx < FT || ny < FT) return false;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    return fused_geom(R, S).bytes <= (size_t)optin;
}

template <int S_, int R_>
adlbr_status launch_fused(int nx, int ny, const FusedGeom &g, const float *u, float *D, const Taps &ts,
                          const Taps &tr, float alpha, float C, cudaStream_t st) {
    ADLBR_CUDA(cudaFuncSetAttribute(ced_fused_kernel<S_, R_>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.bytes));
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        ADLBR_CUDA(cudaGetDevice(&dev));
        ADLBR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int tiles = (int)(blocks_for(nx, FT) * blocks_for(ny, FT));
    const int grid = std::min(tiles, sms);
    ced_fused_kernel<S_, R_><<<grid, fused_threads<S_, R_>(), g.bytes, st>>>(nx, ny, (int64_t)nx * ny, g, ts, tr, u, D,
                                                         alpha, C);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status fused_tensor(int nx, int ny, const float *u, float *D, int rs, int rr, const Taps &ts,
                          const Taps &tr, float alpha, float C, cudaStream_t st) {
    const FusedGeom g = fused_geom(rr, rs);
    if (rs == 3 && rr == 12)   // sigma = 1, rho = 4
        return launch_fused<3, 12>(nx, ny, g, u, D, ts, tr, alpha, C, st);
    return launch_fused<0, 0>(nx, ny, g, u, D, ts, tr, alpha, C, st);
}

adlbr_status check_params(double sigma, double rho, double alpha, double C) {
    if (!(sigma > 0) || !(rho > 0) || !(alpha > 0 && alpha <= 1) || !(C >= 0))
        return fail(ADLBR_E_ARG, "bad CED parameters");
    if (radius_of(sigma) > kMaxR || radius_of(rho) > kMaxR)
        return fail(ADLBR_E_ARG, "Gaussian radius above %d", kMaxR);
    return ADLBR_OK;
}

}  // namespace

size_t ced_tensor_scratch_bytes(int64_t N) { return (size_t)N * sizeof(float) * 6; }

adlbr_status launch_ced_tensor(int nx, int ny, const float *u, float *D, double sigma, double rho,
                               double alpha, double C, void *scratch, cudaStream_t st) {
    ADLBR_NVTX("tensor");
    if (adlbr_status e = check_params(sigma, rho, alpha, C)) return e;
    const int rs = radius_of(sigma), rr = radius_of(rho);
    if (ced_path() != 1 && fused_ok(nx, ny, rr, rs))
        return fused_tensor(nx, ny, u, D, rs, rr, make_taps(sigma), make_taps(rho), (float)alpha,
                            (float)C, st);
    return separable_tensor(nx, ny, u, D, rs, rr, make_taps(sigma), make_taps(rho), (float)alpha,
                            (float)C, scratch, st);
}

adlbr_status launch_ced_build(adlbr_stencils *s, const float *u, double sigma, double rho,
                              double alpha, double C, void *scratch, float *Dtmp, cudaStream_t st) {
    if (s->dim == 3) {
        if (adlbr_status e = launch_ced_tensor3d((int)s->n[0], (int)s->n[1], (int)s->n[2], u, Dtmp, sigma, rho,
                                                 alpha, C, scratch, st))
            return e;
        return launch_build3d(s, Dtmp, ADLBR_F32, st);
    }
    if (adlbr_status e = launch_ced_tensor((int)s->n[0], (int)s->n[1], u, Dtmp, sigma, rho, alpha, C,
                                           scratch, st))
        return e;
    return launch_build2d(s, Dtmp, ADLBR_F32, st);
}

}  // namespace adlbr

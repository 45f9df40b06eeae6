// Internal declarations shared by the translation units of libadlbr.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include <nvtx3/nvToolsExt.h>

#include "../../include/adlbr.h"

namespace adlbr {

// ---------------------------------------------------------------- errors
adlbr_status fail(adlbr_status st, const char *fmt, ...);
adlbr_status cuda_fail(cudaError_t e, const char *what);

#define ADLBR_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Sticky per-handle error bits written by device code (atomicOr).
enum : int {
    ERRBIT_NONFINITE = 1 << 0,
    ERRBIT_NOT_SPD = 1 << 1,
    ERRBIT_RANGE = 1 << 2,
    ERRBIT_NOT_CONVERGED = 1 << 3,
    ERRBIT_TIMEOUT = 1 << 4,   // a bounded device-side wait gave up
    ERRBIT_BOUNDS = 1 << 5,    // a check of the bounds-checked build failed
};

// Index guard.  In the bounds-checked build (-DADLBR_BOUNDS_CHECK) an index
// outside [0, n) records ERRBIT_BOUNDS in *err (when err is given) and the
// caller skips the access; in the normal build the guard is the constant
// true and costs nothing.
#ifdef ADLBR_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, int *err) {
    if ((uint64_t)i < (uint64_t)n) return true;
    if (err) atomicOr(err, ERRBIT_BOUNDS);
    return false;
}
#else
constexpr bool kBoundsCheck = false;
__device__ __forceinline__ constexpr bool in_bounds(int64_t, int64_t, int *) { return true; }
#endif

// NVTX range over one entry point or stage (tensor, build, operator, solve),
// for timelines and for ncu's --nvtx filters.  Header-only NVTX v3: without
// an attached tool a push and a pop cost a few nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define ADLBR_NVTX(name) ::adlbr::NvtxRange adlbr_nvtx_range_(name)

}  // namespace adlbr

// ---------------------------------------------------------------- handle
// Storage layout in HBM (one record per grid point, SoA planes):
//   2D  offs : short4  (e0.x, e0.y, e1.x, e1.y) of the obtuse superbase
//              (e0, e1, e2 = -e0 - e1);
//       w    : 4 lanes (w0, w1, w2, meta), gamma(+-e_i) = w_i;
//   3D  offs : 3 x char4 (e1, e2, e3; e0 = -e1 - e2 - e3), 12 bytes;
//       w    : 8 lanes (w01, w02, w03, w12, w13, w23, meta, 0), w_ij the
//              weight of the Selling offset e_k x e_l, {k,l} = {0..3}\{i,j}.
// Lane types: F64 double, F32 float, F16 half (+ power-of-two scale).
// meta: bit i (i < K) set when weight i is exactly zero; for F16 the high
//       byte holds the signed exponent s of the per-point scale 2^s.
namespace adlbr {
// Table of the gather ("pull") form of a 2D operator (pull.cu).
struct PullTable {
    uint4 *recw = nullptr;      // per point: own and reciprocal weights (halves)
    uint2 *reco = nullptr;      // per point: last reciprocal weight, scale, count, int8 offsets
    uint32_t *ext = nullptr;    // extras (capacity cap + 4)
    uint32_t *seg = nullptr;    // per 32-point row segment: first extra (nseg + 1)
    int *cnt = nullptr;         // build temporaries
    uint32_t *start = nullptr;
    uint32_t *blk = nullptr;
    uint8_t *pushm = nullptr;
    int *flag = nullptr;        // device: the table does not fit its format
    int *flag_host = nullptr;
    int64_t nseg = 0, cap = 0;
    int nseg_x = 0, nblk = 0;
    bool built = false;         // matches the handle's current stencils
    bool usable = false;        // built and within the format's ranges
};
}  // namespace adlbr

struct adlbr_stencils {
    int dim;
    int bc;
    int64_t n[3];
    int64_t N;
    adlbr_dtype w_t;
    int device;
    void *offs;        // device
    void *offs3;       // device, 2D general stencils (A-NN) only: the third offset, short2 per point
    int scheme;        // adlbr_scheme
    void *w;           // device
    int *err;          // device, sticky error bits
    int *err_host;     // pinned host mirror
    // lazily allocated solver workspaces (CG; learned-preconditioner solver)
    void *ws;
    size_t ws_bytes;
    void *ws_nn;
    size_t ws_nn_bytes;
    // operator form (adlbr_operator_form) and the gather table
    int op_form;
    int applies_since_build;
    // a 2D AD-LBR build has stored stencils in offs: the fused build-and-step
    // kernel starts each point from its previous stencil (certified)
    int built;
    adlbr::PullTable *pull;
};

namespace adlbr {

inline int K_of(int dim) { return dim == 2 ? 3 : 6; }
inline size_t offs_bytes_per_point(int dim) { return dim == 2 ? 8 : 12; }
inline size_t w_lane_bytes(adlbr_dtype t) { return t == ADLBR_F64 ? 8 : (t == ADLBR_F32 ? 4 : 2); }
inline size_t w_bytes_per_point(int dim, adlbr_dtype t) { return (dim == 2 ? 4 : 8) * w_lane_bytes(t); }

// ---------------------------------------------------------------- value types
template <typename T> struct UTraits;
template <> struct UTraits<double> { using acc = double; };
template <> struct UTraits<float> { using acc = float; };
template <> struct UTraits<__half> { using acc = float; };
template <> struct UTraits<__nv_bfloat16> { using acc = float; };

// FP16 / BF16 <-> FP32 conversions in integer and FP32 arithmetic.  On GB300
// the hardware conversion instructions issue to the narrow FP64 pipe (ncu
// shows it busy in a kernel whose only non-FP32 work is half -> float), so the
// hot paths convert with bit operations instead.
__device__ __forceinline__ float h2f_bits(uint16_t h) {
    const uint32_t mag = (uint32_t)(h & 0x7fffu) << 13;  // exponent, mantissa in FP32 position
    float f = __fmul_rn(__uint_as_float(mag), 0x1p112f);  // rebias 15 -> 127 (subnormals too)
    if ((h & 0x7c00u) == 0x7c00u) f = __uint_as_float(0x7f800000u | mag);  // inf / nan
    return __uint_as_float(__float_as_uint(f) | ((uint32_t)(h & 0x8000u) << 16));
}
// Round to nearest even; finite inputs beyond the FP16 range give infinity.
__device__ __forceinline__ uint16_t f2h_bits(float f) {
    const uint32_t x = __float_as_uint(f);
    const uint32_t sign = (x >> 16) & 0x8000u;
    const float a = fabsf(f);
    if (!(a < 65520.f)) return (uint16_t)(sign | (a != a ? 0x7e00u : 0x7c00u));
    const uint32_t b = __float_as_uint(__fmul_rn(a, 0x1p-112f));  // exponent rebias 127 -> 15
    const uint32_t r = (b + 0x0fffu + ((b >> 13) & 1u)) >> 13;
    return (uint16_t)(sign | r);
}
__device__ __forceinline__ float bf2f_bits(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t f2bf_bits(float f) {
    const uint32_t x = __float_as_uint(f);
    if ((x & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((x >> 16) | 0x40u);  // nan
    return (uint16_t)((x + 0x7fffu + ((x >> 16) & 1u)) >> 16);
}

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__half v) { return h2f_bits(__half_as_ushort(v)); }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return bf2f_bits(__bfloat16_as_ushort(v)); }

template <typename T> __device__ __forceinline__ T from_acc(typename UTraits<T>::acc v);
template <> __device__ __forceinline__ double from_acc<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_acc<__half>(float v) {
    return __ushort_as_half(f2h_bits(v));
}
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float v) {
    return __ushort_as_bfloat16(f2bf_bits(v));
}

// The three half-stencil offsets of 2D point z.  An AD-LBR stencil stores the
// superbase (e0, e1) and e2 = -e0 - e1 (Corollary
// ObtuseSuperBaseFromReducedBasis2); a general stencil (the A-NN scheme of
// Remark rem:WG) stores e2 in its own plane offs3.
__device__ __forceinline__ void offsets2d(short4 o, const short2 *__restrict__ offs3, int64_t z, int (&ex)[3],
                                          int (&ey)[3]) {
    ex[0] = o.x, ey[0] = o.y, ex[1] = o.z, ey[1] = o.w;
    if (offs3) {
        const short2 t = offs3[z];
        ex[2] = t.x, ey[2] = t.y;
    } else {
        ex[2] = -o.x - o.z, ey[2] = -o.y - o.w;
    }
}

// Selling offsets of a 3D superbase (e0 = -e1-e2-e3): pair q = (i, j) gets
// e_k x e_l with {k, l} the complement, q in (01, 02, 03, 12, 13, 23).
__device__ __forceinline__ void selling_offsets(const char4 (&b)[3], int (&c)[6][3]) {
    int e[4][3];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        e[k][0] = b[k - 1].x;
        e[k][1] = b[k - 1].y;
        e[k][2] = b[k - 1].z;
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) e[0][t] = -e[1][t] - e[2][t] - e[3][t];
    constexpr int PK[6] = {2, 1, 1, 0, 0, 0};
    constexpr int PL[6] = {3, 3, 2, 3, 2, 1};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int *a = e[PK[q]], *bb = e[PL[q]];
        c[q][0] = a[1] * bb[2] - a[2] * bb[1];
        c[q][1] = a[2] * bb[0] - a[0] * bb[2];
        c[q][2] = a[0] * bb[1] - a[1] * bb[0];
    }
}

// ---------------------------------------------------------------- weights
// Reads the K weights of point i (widened to Acc) and the zero mask.
template <typename Acc, int K>
__device__ __forceinline__ unsigned load_weights(const void *wbase, adlbr_dtype wt, int64_t i,
                                                 Acc (&w)[K]) {
    constexpr int L = (K == 3) ? 4 : 8;
    if (wt == ADLBR_F16) {
        const uint4 *p = reinterpret_cast<const uint4 *>(wbase);
        if (L == 4) {
            uint2 r = reinterpret_cast<const uint2 *>(wbase)[i];
            __half h[4];
            *reinterpret_cast<uint2 *>(h) = r;
            uint16_t meta = *reinterpret_cast<uint16_t *>(&h[3]);
            int s = (int)(int8_t)(meta >> 8);
            float sc = __int_as_float((127 + s) << 23);
#pragma unroll
            for (int k = 0; k < K; ++k) w[k] = (Acc)(h2f_bits(__half_as_ushort(h[k])) * sc);
            return meta & 0xffu;
        } else {
            uint4 r = p[i];
            __half h[8];
            *reinterpret_cast<uint4 *>(h) = r;
            uint16_t meta = *reinterpret_cast<uint16_t *>(&h[6]);
            int s = (int)(int8_t)(meta >> 8);
            float sc = __int_as_float((127 + s) << 23);
#pragma unroll
            for (int k = 0; k < K; ++k) w[k] = (Acc)(h2f_bits(__half_as_ushort(h[k])) * sc);
            return meta & 0xffu;
        }
    } else if (wt == ADLBR_F32) {
        const float *p = reinterpret_cast<const float *>(wbase) + i * L;
        float v[L];
        if (L == 4) {
            *reinterpret_cast<float4 *>(v) = *reinterpret_cast<const float4 *>(p);
        } else {
            *reinterpret_cast<float4 *>(v) = *reinterpret_cast<const float4 *>(p);
            *reinterpret_cast<float4 *>(v + 4) = *reinterpret_cast<const float4 *>(p + 4);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = (Acc)v[k];
        return (unsigned)v[K];
    } else {
        const double *p = reinterpret_cast<const double *>(wbase) + i * L;
        double v[L];
#pragma unroll
        for (int k = 0; k < L; k += 2)
            *reinterpret_cast<double2 *>(v + k) = *reinterpret_cast<const double2 *>(p + k);
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = (Acc)v[k];
        return (unsigned)v[K];
    }
}

// ---------------------------------------------------------------- launch helpers
// Number of SMs of the current device (queried once per device).
int sm_count();
// Blocks of the grid-stride vector and reduction kernels: 8 per SM.
inline int vec_blocks() { return 8 * sm_count(); }

inline unsigned blocks_for(int64_t n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

// API-level validation helpers (api.cu)
adlbr_status check_handle(const adlbr_stencils *s);

// kernels' host launchers
// Every build launcher first marks the handle's stencils as changed: the
// gather table (if any) no longer matches them.
void stencils_changed(adlbr_stencils *s);
adlbr_status launch_build2d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st);
adlbr_status launch_build3d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st);
// the A-NN comparison scheme (Sec. 4.1, Remark rem:WG), 2D (ann.cu)
adlbr_status launch_build_ann2d(adlbr_stencils *s, const void *D, adlbr_dtype D_t, cudaStream_t st);
adlbr_status launch_export(const adlbr_stencils *s, int16_t *offs, void *w, cudaStream_t st);
adlbr_status launch_apply(const adlbr_stencils *s, const void *u, void *Au, adlbr_dtype u_t,
                          cudaStream_t st);
size_t ced_tensor_scratch_bytes(int64_t N);
size_t ced_tensor3d_scratch_bytes(int64_t N);
adlbr_status launch_ced_tensor3d(int nx, int ny, int nz, const float *u, float *D, double sigma, double rho,
                                 double alpha, double C, void *scratch, cudaStream_t st);
adlbr_status launch_eed_tensor3d(int nx, int ny, int nz, const float *u, float *D, double sigma, double rho,
                                 double C, void *scratch, cudaStream_t st);
adlbr_status launch_ced_tensor(int nx, int ny, const float *u, float *D, double sigma, double rho,
                               double alpha, double C, void *scratch, cudaStream_t st);
// CED tensor stage fused with the 2D stencil construction into handle s
// (Dtmp, 3N floats, is only used by the fallback path for unusual radii).
adlbr_status launch_ced_build(adlbr_stencils *s, const float *u, double sigma, double rho,
                              double alpha, double C, void *scratch, float *Dtmp, cudaStream_t st);
adlbr_status unet_create(int cin, int c1, int c2, int c3, int B, int H, int W, adlbr_unet **out);
adlbr_status unet_destroy(adlbr_unet *n);
adlbr_status unet_forward(adlbr_unet *n, const float *params, const float *xin, float *yout,
                          cudaStream_t st);
adlbr_status unet_backward(adlbr_unet *n, const float *params, const float *gy, float *gparams,
                           float *gx, cudaStream_t st);
adlbr_status unet_adam(float *params, const float *grads, float *m, float *v, int64_t n, double lr,
                       double b1, double b2, double eps, int t, cudaStream_t st);
int64_t unet_num_params(const adlbr_unet *n);
adlbr_status unet_set_tensor_cores(adlbr_unet *n, int on);
// The tensor-core forward's BF16 channels-last input buffer ([B][H][W][cp],
// cp = cin rounded up to 16), or nullptr when the network runs on FP32 cores.
// unet_tc_prepare packs the BF16 weights of params; unet_forward_from_input
// then runs the tensor-core forward on the input buffer and the packed
// weights as they stand (a caller whose parameters and some input channels
// do not change between forwards sets them up once).
__nv_bfloat16 *unet_tc_input(adlbr_unet *n, int *cp);
adlbr_status unet_tc_prepare(adlbr_unet *n, const float *params, cudaStream_t st);
adlbr_status unet_forward_from_input(adlbr_unet *n, const float *params, float *yout, cudaStream_t st);
// tensor-core 3x3 convolution + bias + ReLU (unet_tc.cu)
size_t conv_tc_pack_elems(int Co, int Ci);
struct ConvPackTable {   // the 3x3 layers packed by one conv_tc_pack launch
    int n;
    int co[10], ci[10];
    int64_t w_off[10];   // weights in the flat parameter vector
    int64_t out_off[10]; // packed BF16 elements, 8-element aligned
};
adlbr_status conv_tc_pack(const ConvPackTable &T, const float *params, __nv_bfloat16 *out, cudaStream_t st);
bool conv_tc_supported(int Co, int Ci);
// y (BF16 [B][H][W][Co]) = ReLU(bias + conv3x3([x0 | x1])), x0 [B][H][W][C0],
// x1 [B][H][W][C1] (C1 = 0: no second input), C0 + C1 = the packed Kp
adlbr_status conv_tc(int B, int H, int W, const __nv_bfloat16 *x0, int C0, const __nv_bfloat16 *x1, int C1,
                     int Co, const __nv_bfloat16 *wpack, const float *bias, __nv_bfloat16 *y, cudaStream_t st);
adlbr_status tc_to_nhwc(int B, int C, int Cp, int64_t HW, const float *x, __nv_bfloat16 *y, cudaStream_t st);
adlbr_status tc_pool(int B, int H2, int W2, int C, const __nv_bfloat16 *x, __nv_bfloat16 *y, cudaStream_t st);
adlbr_status tc_up(int B, int H, int W, int C, const __nv_bfloat16 *x, __nv_bfloat16 *y, cudaStream_t st);
adlbr_status tc_out1x1(int64_t n, int C, const __nv_bfloat16 *x, const float *w, const float *bias, float *y,
                       cudaStream_t st);
void unet_shape(const adlbr_unet *n, int *cin, int *B, int *H, int *W);
adlbr_status run_fcg(adlbr_stencils *s, const float *b, float *x, double dt, double rtol, int maxit,
                     const adlbr_nn_precond *nn, int *iters_out, double *relres_out, cudaStream_t st);
adlbr_status nn_pairs(adlbr_stencils *s, const float *b, double dt, double rtol, int maxit, int every,
                      int max_pairs, const adlbr_nn_precond *nn, float *feats, float *targets,
                      float *xbuf, int *n_pairs, cudaStream_t st);
adlbr_status max_diag(adlbr_stencils *s, double *out, cudaStream_t st);
adlbr_status nn_apply(adlbr_stencils *s, const adlbr_nn_precond *nn, double dt, const float *r,
                      float *z, cudaStream_t st);
adlbr_status mse_grad(const float *y, const float *t, int64_t n, float *gy, double *loss,
                      cudaStream_t st);
adlbr_status run_cg(adlbr_stencils *s, const float *b, float *x, double dt, double rtol, int maxit,
                    int *iters_out, double *relres_out, cudaStream_t st);
typedef adlbr_status (*CgHook)(void *ctx, const float *r, const float *x, int iter, cudaStream_t st);
adlbr_status run_cg_hooked(adlbr_stencils *s, const float *b, float *x, double dt, double rtol,
                           int maxit, int *iters_out, double *relres_out, int every, CgHook hook,
                           void *ctx, cudaStream_t st);
// Records whether the last implicit solve of the calling thread ended with
// its true relative residual at or below rtol (adlbr_last_residual_met).
void set_last_residual_met(bool met);
// CG preconditioned by the diagonal 1 + dt A_zz (same stopping test as run_cg)
adlbr_status run_pcg_jacobi(adlbr_stencils *s, const float *b, float *x, double dt, double rtol, int maxit,
                            int *iters_out, double *relres_out, cudaStream_t st);
// inv_d = 1 / (1 + dt A_zz) (nnpc.cu)
adlbr_status launch_jacobi_inverse(const adlbr_stencils *s, double dt, float *inv_d, cudaStream_t st);
// acc += scale * A u (accumulation type: double for F64 u, float otherwise);
// a kernel launched with skip != NULL returns at once when *skip != 0.
adlbr_status launch_accumulate(const adlbr_stencils *s, const void *u, void *acc, adlbr_dtype u_t,
                               double scale, const int *skip, cudaStream_t st);
// acc = scale A u with the stencils of the FP32 tensor D built (and stored
// in s) by the same kernel: 2D AD-LBR handles with F16 weights, FP32 u on a
// non-periodic grid that takes a TMA window, not set to the gather form.
// *done = false (nothing enqueued) for any other case.
adlbr_status launch_build_accumulate2d(adlbr_stencils *s, const float *D, const float *u, float *acc,
                                       double scale, bool *done, cudaStream_t st);
// acc (double) += scale * A u for FP32 u: the FP64-accumulated operator used to
// measure true residuals.
adlbr_status launch_accumulate_f64(const adlbr_stencils *s, const float *u, double *acc, double scale,
                                   cudaStream_t st);
// u <- u - acc ; acc <- 0
// A fixed sequence of launches recorded into a CUDA graph and replayed with
// cudaGraphLaunch on the caller's stream.  The recording runs on a private
// stream (capture is not allowed on the legacy default stream, which a
// caller may pass); nothing executes during it.
struct ChunkGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    template <typename F>
    adlbr_status capture(F &&enqueue) {
        cudaStream_t cs = nullptr;
        ADLBR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        adlbr_status e = ADLBR_OK;
        if (ce == cudaSuccess) {
            e = enqueue(cs);
            ce = cudaStreamEndCapture(cs, &graph);
        }
        cudaStreamDestroy(cs);
        if (e != ADLBR_OK) return e;
        ADLBR_CUDA(ce);
        ADLBR_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        return ADLBR_OK;
    }
    ~ChunkGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

adlbr_status launch_finalize(const adlbr_stencils *s, void *u, void *acc, adlbr_dtype u_t,
                             cudaStream_t st);

// ---- gather (pull) form of the operator (pull.cu)
bool pull_supported(const adlbr_stencils *s);
// Builds the table for the handle's current stencils (synchronises st once).
adlbr_status pull_build(adlbr_stencils *s, cudaStream_t st);
void pull_free(adlbr_stencils *s);
bool pull_ready(const adlbr_stencils *s);
// out = a u + b A u by the gather form (requires pull_ready(s)); out is
// F32, or u's own type for F16 / BF16 u.  Must not alias u.
adlbr_status launch_pull(const adlbr_stencils *s, const void *u, adlbr_dtype u_t, void *out, adlbr_dtype out_t,
                         double a, double b, const int *skip, cudaStream_t st);
// Decides the form of the next operator applications on s: true = gather
// (building the table first when needed).  `uses` is the number of
// applications the caller is about to make with the current stencils.
adlbr_status choose_gather(adlbr_stencils *s, int uses, bool *gather, cudaStream_t st);
// out = a u + b A u by whichever form choose_gather picks (the scatter form
// initialises out with a u, by a memset or a copy, and accumulates).
adlbr_status launch_operator(adlbr_stencils *s, const void *u, adlbr_dtype u_t, void *out, double a, double b,
                             cudaStream_t st);

}  // namespace adlbr

// C-ABI entry points of libadlbr.so (see include/adlbr.h).
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace adlbr {

static thread_local char g_msg[512] = "";
static thread_local int g_residual_met = 0;

void set_last_residual_met(bool met) { g_residual_met = met ? 1 : 0; }

adlbr_status fail(adlbr_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

adlbr_status cuda_fail(cudaError_t e, const char *what) {
    return fail(ADLBR_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int sm_count() {
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        cache[dev] = n;
    }
    return cache[dev];
}

adlbr_status check_handle(const adlbr_stencils *s) {
    if (!s) return fail(ADLBR_E_ARG, "null stencil handle");
    return ADLBR_OK;
}

static bool valid_grid(const adlbr_grid *g) {
    if (!g || (g->dim != 2 && g->dim != 3)) return false;
    if (g->bc != ADLBR_NEUMANN && g->bc != ADLBR_PERIODIC) return false;
    for (int k = 0; k < g->dim; ++k)
        if (g->n[k] <= 0 || g->n[k] > 65535) return false;
    return true;
}

static int64_t npoints(const adlbr_grid *g) {
    return g->n[0] * g->n[1] * (g->dim == 3 ? g->n[2] : 1);
}

void stencils_changed(adlbr_stencils *s) {
    if (s->pull) s->pull->built = false;
    s->applies_since_build = 0;
}

// *ps == NULL: allocates a handle for grid g, weight type w_t and scheme.
// *ps != NULL: checks that it matches (and takes g's boundary rule).
static adlbr_status acquire_handle(const adlbr_grid *g, adlbr_dtype w_t, adlbr_stencils **ps,
                                   int scheme = ADLBR_SCHEME_ADLBR) {
    adlbr_stencils *s = *ps;
    if (s) {
        bool same = s->dim == g->dim && s->w_t == w_t && s->n[0] == g->n[0] && s->n[1] == g->n[1] &&
                    (g->dim == 2 || s->n[2] == g->n[2]) && s->scheme == scheme;
        if (!same) return fail(ADLBR_E_SHAPE, "handle does not match the grid / weight type / scheme");
        if (s->bc != g->bc) pull_free(s);
        s->bc = g->bc;
        return ADLBR_OK;
    }
    s = new (std::nothrow) adlbr_stencils();
    if (!s) return fail(ADLBR_E_INTERNAL, "out of host memory");
    s->dim = g->dim;
    s->bc = g->bc;
    s->n[0] = g->n[0];
    s->n[1] = g->n[1];
    s->n[2] = g->dim == 3 ? g->n[2] : 1;
    s->N = npoints(g);
    s->w_t = w_t;
    s->scheme = scheme;
    cudaGetDevice(&s->device);
    size_t ob = offs_bytes_per_point(s->dim) * (size_t)s->N;
    size_t wb = w_bytes_per_point(s->dim, w_t) * (size_t)s->N;
    cudaError_t e = cudaMalloc(&s->offs, ob);
    if (e == cudaSuccess && scheme == ADLBR_SCHEME_ANN) e = cudaMalloc(&s->offs3, sizeof(short2) * (size_t)s->N);
    if (e == cudaSuccess) e = cudaMalloc(&s->w, wb);
    if (e == cudaSuccess) e = cudaMalloc(&s->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&s->err_host, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        adlbr_stencils_destroy(s);
        return cuda_fail(e, "allocating stencil storage");
    }
    *ps = s;
    return ADLBR_OK;
}

}  // namespace adlbr

using namespace adlbr;

// Stencils of D into s, then one explicit step of u (FP32) with acc as the
// accumulator: one fused kernel where the handle allows it.
static adlbr_status build_then_step(adlbr_stencils *s, const void *D, adlbr_dtype D_t, float *u, float *acc,
                                    double dt, cudaStream_t stream) {
    bool fused = false;
    if (D_t == ADLBR_F32)
        if (adlbr_status st = launch_build_accumulate2d(s, (const float *)D, u, acc, dt, &fused, stream)) return st;
    if (fused) return launch_finalize(s, u, acc, ADLBR_F32, stream);
    adlbr_status st = s->dim == 2 ? launch_build2d(s, D, D_t, stream) : launch_build3d(s, D, D_t, stream);
    if (st != ADLBR_OK) return st;
    return adlbr_step_explicit(s, u, acc, ADLBR_F32, dt, 1, stream);
}

extern "C" {

const char *adlbr_version(void) {
    return kBoundsCheck ? "adlbr-gb300 0.1 (sm_103a, bounds-checked)" : "adlbr-gb300 0.1 (sm_103a)";
}

const char *adlbr_last_error(void) { return g_msg; }

int adlbr_last_residual_met(void) { return g_residual_met; }

adlbr_status adlbr_build_stencils(const adlbr_grid *g, const void *D, adlbr_dtype D_t,
                                  adlbr_dtype w_t, adlbr_stencils **out, cudaStream_t stream) {
    return adlbr_build_stencils_scheme(g, D, D_t, w_t, ADLBR_SCHEME_ADLBR, out, stream);
}

adlbr_status adlbr_build_stencils_scheme(const adlbr_grid *g, const void *D, adlbr_dtype D_t,
                                         adlbr_dtype w_t, int scheme, adlbr_stencils **out,
                                         cudaStream_t stream) {
    ADLBR_NVTX("adlbr_build_stencils_scheme");
    if (!out || !D) return fail(ADLBR_E_ARG, "null argument");
    if (!valid_grid(g)) return fail(ADLBR_E_SHAPE, "invalid grid");
    if (D_t != ADLBR_F32 && D_t != ADLBR_F64) return fail(ADLBR_E_ARG, "D must be F32 or F64");
    if (w_t != ADLBR_F32 && w_t != ADLBR_F64 && w_t != ADLBR_F16)
        return fail(ADLBR_E_ARG, "weights must be F64, F32 or F16");
    if (scheme != ADLBR_SCHEME_ADLBR && scheme != ADLBR_SCHEME_ANN)
        return fail(ADLBR_E_ARG, "unknown scheme %d", scheme);
    if (scheme == ADLBR_SCHEME_ANN && g->dim != 2) return fail(ADLBR_E_SHAPE, "the A-NN scheme is 2D");
    adlbr_stencils *s = *out;
    if (adlbr_status e = acquire_handle(g, w_t, &s, scheme)) return e;
    adlbr_status st = scheme == ADLBR_SCHEME_ANN ? launch_build_ann2d(s, D, D_t, stream)
                      : s->dim == 2              ? launch_build2d(s, D, D_t, stream)
                                                 : launch_build3d(s, D, D_t, stream);
    if (st != ADLBR_OK) {
        if (!*out) adlbr_stencils_destroy(s);
        return st;
    }
    *out = s;
    return ADLBR_OK;
}

adlbr_status adlbr_stencils_check(adlbr_stencils *s, cudaStream_t stream) {
    if (adlbr_status st = check_handle(s)) return st;
    ADLBR_CUDA(cudaMemcpyAsync(s->err_host, s->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    ADLBR_CUDA(cudaMemsetAsync(s->err, 0, sizeof(int), stream));
    ADLBR_CUDA(cudaStreamSynchronize(stream));
    int bits = *s->err_host;
    if (bits & ERRBIT_NONFINITE) return fail(ADLBR_E_NONFINITE, "non-finite tensor entries");
    if (bits & ERRBIT_NOT_SPD) return fail(ADLBR_E_NOT_SPD, "tensor not positive definite");
    if (bits & ERRBIT_RANGE) return fail(ADLBR_E_RANGE, "stencil offset out of storage range");
    if (bits & ERRBIT_NOT_CONVERGED) return fail(ADLBR_E_NOT_CONVERGED, "reduction did not converge");
    if (bits & ERRBIT_TIMEOUT) return fail(ADLBR_E_TIMEOUT, "a device-side wait for a tile copy gave up");
    if (bits & ERRBIT_BOUNDS)
        return fail(ADLBR_E_INTERNAL, "an index or stencil-radius check of the bounds-checked build failed");
    return ADLBR_OK;
}

adlbr_status adlbr_stencils_scheme(const adlbr_stencils *s, int *scheme) {
    if (adlbr_status st = check_handle(s)) return st;
    if (!scheme) return fail(ADLBR_E_ARG, "null output");
    *scheme = s->scheme;
    return ADLBR_OK;
}

adlbr_status adlbr_stencils_grid(const adlbr_stencils *s, adlbr_grid *g) {
    if (adlbr_status st = check_handle(s)) return st;
    if (!g) return fail(ADLBR_E_ARG, "null grid");
    g->dim = s->dim;
    g->bc = s->bc;
    g->n[0] = s->n[0];
    g->n[1] = s->n[1];
    g->n[2] = s->n[2];
    return ADLBR_OK;
}

adlbr_status adlbr_stencils_export(const adlbr_stencils *s, int16_t *offs, void *w,
                                   cudaStream_t stream) {
    ADLBR_NVTX("adlbr_stencils_export");
    if (adlbr_status st = check_handle(s)) return st;
    if (!offs || !w) return fail(ADLBR_E_ARG, "null output");
    return launch_export(s, offs, w, stream);
}

adlbr_status adlbr_stencils_destroy(adlbr_stencils *s) {
    if (!s) return ADLBR_OK;
    // bounds-checked build: a failed check that no adlbr_stencils_check
    // collected is reported here (the copy waits for the device)
    int bits = 0;
    if (kBoundsCheck && s->err && cudaMemcpy(&bits, s->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        bits = 0;
    if (s->offs) cudaFree(s->offs);
    if (s->offs3) cudaFree(s->offs3);
    if (s->w) cudaFree(s->w);
    if (s->err) cudaFree(s->err);
    if (s->err_host) cudaFreeHost(s->err_host);
    if (s->ws) cudaFree(s->ws);
    if (s->ws_nn) cudaFree(s->ws_nn);
    pull_free(s);
    delete s;
    if (bits & ERRBIT_BOUNDS)
        return fail(ADLBR_E_INTERNAL, "an index or stencil-radius check of the bounds-checked build failed");
    return ADLBR_OK;
}

adlbr_status adlbr_apply(const adlbr_stencils *s, const void *u, void *Au, adlbr_dtype u_t,
                         cudaStream_t stream) {
    ADLBR_NVTX("adlbr_apply");
    if (adlbr_status st = check_handle(s)) return st;
    if (!u || !Au) return fail(ADLBR_E_ARG, "null vector");
    if (u == Au) return fail(ADLBR_E_ARG, "Au must not alias u");
    if (u_t < ADLBR_F64 || u_t > ADLBR_BF16) return fail(ADLBR_E_ARG, "bad u dtype");
    // the handle's gather table is a cache: building it does not change the operator
    return launch_operator(const_cast<adlbr_stencils *>(s), u, u_t, Au, 0.0, 1.0, stream);
}

adlbr_status adlbr_stencils_set_operator(adlbr_stencils *s, int form) {
    if (adlbr_status st = check_handle(s)) return st;
    if (form != ADLBR_OP_AUTO && form != ADLBR_OP_SCATTER && form != ADLBR_OP_GATHER)
        return fail(ADLBR_E_ARG, "unknown operator form %d", form);
    s->op_form = form;
    return ADLBR_OK;
}

adlbr_status adlbr_stencils_get_operator(const adlbr_stencils *s, int *form, int *gather_ready) {
    if (adlbr_status st = check_handle(s)) return st;
    if (form) *form = s->op_form;
    if (gather_ready) *gather_ready = pull_ready(s) ? 1 : 0;
    return ADLBR_OK;
}

adlbr_status adlbr_build_step_explicit(const adlbr_grid *g, const void *D, adlbr_dtype D_t, adlbr_dtype w_t,
                                       adlbr_stencils **out, float *u, void *scratch, double dt,
                                       cudaStream_t stream) {
    ADLBR_NVTX("adlbr_build_step_explicit");
    if (!out || !D || !u || !scratch) return fail(ADLBR_E_ARG, "null argument");
    if (!valid_grid(g)) return fail(ADLBR_E_SHAPE, "invalid grid");
    if (D_t != ADLBR_F32 && D_t != ADLBR_F64) return fail(ADLBR_E_ARG, "D must be F32 or F64");
    if (w_t != ADLBR_F32 && w_t != ADLBR_F64 && w_t != ADLBR_F16)
        return fail(ADLBR_E_ARG, "weights must be F64, F32 or F16");
    if (!(dt >= 0.0)) return fail(ADLBR_E_ARG, "bad dt");
    const bool fresh = *out == nullptr;
    adlbr_stencils *s = *out;
    if (adlbr_status e = acquire_handle(g, w_t, &s)) return e;
    adlbr_status st = build_then_step(s, D, D_t, u, (float *)scratch, dt, stream);
    if (st != ADLBR_OK) {
        if (fresh) adlbr_stencils_destroy(s);
        return st;
    }
    *out = s;
    return ADLBR_OK;
}

size_t adlbr_step_scratch_bytes(const adlbr_stencils *s, adlbr_dtype u_t) {
    if (!s) return 0;
    return (size_t)s->N * (u_t == ADLBR_F64 ? sizeof(double) : sizeof(float));
}

adlbr_status adlbr_step_explicit(const adlbr_stencils *s, void *u, void *scratch, adlbr_dtype u_t,
                                 double dt, int nsteps, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_step_explicit");
    if (adlbr_status st = check_handle(s)) return st;
    if (!u || !scratch) return fail(ADLBR_E_ARG, "null buffer");
    if (nsteps < 0 || !(dt >= 0.0)) return fail(ADLBR_E_ARG, "bad dt / nsteps");
    if (u_t < ADLBR_F64 || u_t > ADLBR_BF16) return fail(ADLBR_E_ARG, "bad u dtype");
    if (nsteps == 0) return ADLBR_OK;
    adlbr_stencils *sm = const_cast<adlbr_stencils *>(s);   // gather table: a cache
    bool gather = false;
    if (u_t != ADLBR_F64)
        if (adlbr_status st = choose_gather(sm, nsteps, &gather, stream)) return st;
    if (gather) {
        // u^{n+1} = u^n - dt A u^n written to the other buffer (u, scratch in turn)
        void *src = u, *dst = scratch;
        for (int k = 0; k < nsteps; ++k) {
            if (adlbr_status st = launch_pull(s, src, u_t, dst, u_t, 1.0, -dt, nullptr, stream)) return st;
            void *t = src;
            src = dst;
            dst = t;
        }
        if (src != u) {
            const size_t es = u_t == ADLBR_F32 ? 4 : 2;
            ADLBR_CUDA(cudaMemcpyAsync(u, src, (size_t)s->N * es, cudaMemcpyDeviceToDevice, stream));
        }
        return ADLBR_OK;
    }
    // per step: scratch <- 0, scratch += dt A u, u -= scratch
    for (int k = 0; k < nsteps; ++k) {
        ADLBR_CUDA(cudaMemsetAsync(scratch, 0, adlbr_step_scratch_bytes(s, u_t), stream));
        if (adlbr_status st = launch_accumulate(s, u, scratch, u_t, dt, nullptr, stream)) return st;
        if (adlbr_status st = launch_finalize(s, u, scratch, u_t, stream)) return st;
    }
    return ADLBR_OK;
}

adlbr_status adlbr_step_implicit(adlbr_stencils *s, const void *rhs, void *x, double dt,
                                 double rtol, int maxit, int precond, const void *nn,
                                 int *iters_out, double *relres_out, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_step_implicit");
    if (adlbr_status st = check_handle(s)) return st;
    if (!rhs || !x) return fail(ADLBR_E_ARG, "null vector");
    if (!(dt >= 0.0) || !(rtol > 0.0) || maxit < 1) return fail(ADLBR_E_ARG, "bad dt / rtol / maxit");
    set_last_residual_met(false);
    if (precond == 1)
        return run_fcg(s, (const float *)rhs, (float *)x, dt, rtol, maxit,
                       (const adlbr_nn_precond *)nn, iters_out, relres_out, stream);
    if (precond == 2)
        return run_pcg_jacobi(s, (const float *)rhs, (float *)x, dt, rtol, maxit, iters_out, relres_out, stream);
    if (precond != 0) return fail(ADLBR_E_ARG, "unknown preconditioner %d", precond);
    return run_cg(s, (const float *)rhs, (float *)x, dt, rtol, maxit, iters_out, relres_out, stream);
}

adlbr_status adlbr_nn_training_pairs(adlbr_stencils *s, const float *rhs, double dt, double rtol,
                                     int maxit, int every, int max_pairs,
                                     const adlbr_nn_precond *nn, float *feats, float *targets,
                                     float *xbuf, int *n_pairs, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_nn_training_pairs");
    if (adlbr_status st = check_handle(s)) return st;
    if (!rhs || !feats || !targets || !xbuf) return fail(ADLBR_E_ARG, "null buffer");
    if (!(dt >= 0.0) || !(rtol > 0.0) || maxit < 1) return fail(ADLBR_E_ARG, "bad dt / rtol / maxit");
    return nn_pairs(s, rhs, dt, rtol, maxit, every, max_pairs, nn, feats, targets, xbuf, n_pairs,
                    stream);
}

adlbr_status adlbr_nn_precondition(adlbr_stencils *s, const adlbr_nn_precond *nn, double dt,
                                   const float *r, float *z, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_nn_precondition");
    if (adlbr_status st = check_handle(s)) return st;
    if (!r || !z) return fail(ADLBR_E_ARG, "null buffer");
    return nn_apply(s, nn, dt, r, z, stream);
}

adlbr_status adlbr_stencils_max_diag(adlbr_stencils *s, double *out, cudaStream_t stream) {
    if (adlbr_status st = check_handle(s)) return st;
    if (!out) return fail(ADLBR_E_ARG, "null output");
    return max_diag(s, out, stream);
}

adlbr_status adlbr_mse_grad(const float *y, const float *t, int64_t n, float *gy,
                            double *loss_out, cudaStream_t stream) {
    if (!y || !t || !gy || n < 1) return fail(ADLBR_E_ARG, "bad argument");
    return mse_grad(y, t, n, gy, loss_out, stream);
}

// CED scratch: tensor temporaries, then D (3 or 6 planes), then the explicit
// step's accumulator (N floats).
static size_t ced_temp_bytes(const adlbr_grid *g, int64_t N) {
    return g->dim == 2 ? ced_tensor_scratch_bytes(N) : ced_tensor3d_scratch_bytes(N);
}
static int ced_planes(const adlbr_grid *g) { return g->dim == 2 ? 3 : 6; }

size_t adlbr_ced_scratch_bytes(const adlbr_grid *g) {
    if (!valid_grid(g)) return 0;
    const int64_t N = npoints(g);
    return ced_temp_bytes(g, N) + (size_t)N * sizeof(float) * (ced_planes(g) + 1);
}

adlbr_status adlbr_ced_tensor(const adlbr_grid *g, const float *u, float *D, double sigma,
                              double rho, double alpha, double C, void *scratch,
                              cudaStream_t stream) {
    ADLBR_NVTX("adlbr_ced_tensor");
    if (!valid_grid(g)) return fail(ADLBR_E_SHAPE, "CED needs a valid 2D or 3D grid");
    if (!u || !D || !scratch) return fail(ADLBR_E_ARG, "null buffer");
    if (g->dim == 3)
        return launch_ced_tensor3d((int)g->n[0], (int)g->n[1], (int)g->n[2], u, D, sigma, rho, alpha, C,
                                   scratch, stream);
    return launch_ced_tensor((int)g->n[0], (int)g->n[1], u, D, sigma, rho, alpha, C, scratch, stream);
}

adlbr_status adlbr_eed_tensor(const adlbr_grid *g, const float *u, float *D, double sigma, double rho, double C,
                              void *scratch, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_eed_tensor");
    if (!valid_grid(g) || g->dim != 3) return fail(ADLBR_E_SHAPE, "edge-enhancing diffusion needs a valid 3D grid");
    if (!u || !D || !scratch) return fail(ADLBR_E_ARG, "null buffer");
    return launch_eed_tensor3d((int)g->n[0], (int)g->n[1], (int)g->n[2], u, D, sigma, rho, C, scratch, stream);
}

adlbr_status adlbr_ced_stencils(adlbr_stencils **s, const adlbr_grid *g, const float *u,
                                void *scratch, double sigma, double rho, double alpha, double C,
                                adlbr_dtype w_t, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_ced_stencils");
    if (!s) return fail(ADLBR_E_ARG, "null handle pointer");
    if (!valid_grid(g)) return fail(ADLBR_E_SHAPE, "CED needs a valid 2D or 3D grid");
    if (!u || !scratch) return fail(ADLBR_E_ARG, "null buffer");
    if (w_t != ADLBR_F32 && w_t != ADLBR_F64 && w_t != ADLBR_F16)
        return fail(ADLBR_E_ARG, "weights must be F64, F32 or F16");
    const int64_t N = npoints(g);
    float *D = (float *)((char *)scratch + ced_temp_bytes(g, N));
    const bool fresh = *s == nullptr;
    if (adlbr_status st = acquire_handle(g, w_t, s)) return st;
    adlbr_status st = launch_ced_build(*s, u, sigma, rho, alpha, C, scratch, D, stream);
    if (st != ADLBR_OK && fresh) {
        adlbr_stencils_destroy(*s);
        *s = nullptr;
    }
    return st;
}

adlbr_status adlbr_ced_step(adlbr_stencils **s, const adlbr_grid *g, float *u, void *scratch,
                            double sigma, double rho, double alpha, double C, double dt,
                            int nsteps, adlbr_dtype w_t, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_ced_step");
    if (!s) return fail(ADLBR_E_ARG, "null handle pointer");
    if (!valid_grid(g)) return fail(ADLBR_E_SHAPE, "CED needs a valid 2D or 3D grid");
    if (!u || !scratch) return fail(ADLBR_E_ARG, "null buffer");
    if (nsteps < 0 || !(dt >= 0.0)) return fail(ADLBR_E_ARG, "bad dt / nsteps");
    const int64_t N = npoints(g);
    float *D = (float *)((char *)scratch + ced_temp_bytes(g, N));
    float *acc = D + ced_planes(g) * N;
    if (w_t != ADLBR_F32 && w_t != ADLBR_F64 && w_t != ADLBR_F16)
        return fail(ADLBR_E_ARG, "weights must be F64, F32 or F16");
    const bool fresh = *s == nullptr;
    if (adlbr_status st = acquire_handle(g, w_t, s)) return st;
    for (int k = 0; k < nsteps; ++k) {
        // tensor stage, stencil construction, one explicit step; in 2D the
        // construction and the operator run as one kernel where the handle
        // allows it (F16 weights, a TMA window)
        adlbr_status st =
            g->dim == 2
                ? launch_ced_tensor((int)g->n[0], (int)g->n[1], u, D, sigma, rho, alpha, C, scratch, stream)
                : launch_ced_tensor3d((int)g->n[0], (int)g->n[1], (int)g->n[2], u, D, sigma, rho, alpha, C,
                                      scratch, stream);
        if (st == ADLBR_OK) st = build_then_step(*s, D, ADLBR_F32, u, acc, dt, stream);
        if (st != ADLBR_OK) {
            if (fresh) {
                adlbr_stencils_destroy(*s);
                *s = nullptr;
            }
            return st;
        }
    }
    return ADLBR_OK;
}

}  // extern "C"

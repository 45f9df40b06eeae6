// Implicit step (I + dt A) x = b by conjugate gradients (Sec. 4.2: the
// discretised Eq. elliptic is solved by Conjugate Gradient; here with
// lambda = dt and b = u^n).
//
// Vectors are FP32; every dot product and norm is accumulated with exact
// products in float-float within threads and warps and in FP64 across warps
// and blocks, by a deterministic two-level reduction (one partial per block,
// the last block to finish sums the partials in block order).  The CG scalars
// alpha, beta and |r|^2 live in device memory and are produced by that last
// block, so an iteration needs no host round trip; the host polls a
// convergence flag every few iterations.  Once the flag is set every kernel
// returns immediately, so the reported iteration count is exact.
//
// Per iteration, with q = p on entry: q += dt A p (so q = (I + dt A) p), then
//   K2  <p, q> ; last block: alpha = rr / <p,q>
//   K3  x += alpha p ; r -= alpha q ; <r, r> ; last block: beta, flag
//   K4  p <- r + beta p ; q <- p
// JAC (CG preconditioned by the diagonal d = 1 + dt A_zz, z = r / d, held as
// 1 / d): alpha = <r,z> / <p,q>, K3 also sums <r,z>, beta = <r,z>_new /
// <r,z>_old, K4 sets p <- z + beta p.  The stopping test stays |r| <= rtol |b|.
// (no kernel stores a constant over a value it has just loaded: such a
// store waits for the load and a vector pass with one runs at a fraction of
// the HBM rate on this GPU)
#include <cmath>
#include <cstddef>

#include "internal.cuh"
#include "reduce.cuh"

namespace adlbr {

namespace {


struct CgState {
    double rr, rr_new, pq, alpha, beta, bb, tol2, rz;
    int conv, iters, max_iters;  // conv: 0 running, 1 converged, 2 iteration limit, 3 non-finite
    unsigned int count;          // last-block ticket
};

// (Re)start from the true residual: r = b - (x + dt A x) evaluated in FP64
// (acc holds dt A x accumulated in FP64 -- or in FP32 for the first round,
// AT = float), rounded once to FP32; p = r.
// rr_new = |r|^2 of the FP64 residual, rr = |r|^2 of its FP32 copy, bb = |b|^2;
// conv = 1 when the true residual already meets the tolerance.
template <bool JAC, typename AT>
__global__ void __launch_bounds__(RT) cg_restart_kernel(int64_t N, const float *__restrict__ b,
                                                        const float *__restrict__ x,
                                                        const AT *__restrict__ acc,
                                                        const float *__restrict__ inv_d,
                                                        float *__restrict__ r, float *__restrict__ p,
                                                        double *partials, double *partials2,
                                                        double *partials3, double *partials4, CgState *S) {
    double s_true = 0.0, s_rr = 0.0, s_bb = 0.0, s_rz = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < N; i += (int64_t)gridDim.x * RT) {
        const double bi = b[i];
        const double ri = bi - ((double)x[i] + (double)acc[i]);
        const float rf = (float)ri;
        r[i] = rf;
        const float zf = JAC ? rf * inv_d[i] : rf;
        p[i] = zf;
        s_true += ri * ri;
        s_rr += (double)rf * rf;
        s_bb += bi * bi;
        if (JAC) s_rz += (double)rf * zf;
    }
    const double pt = block_sum(s_true);
    const double pr = block_sum(s_rr);
    const double pb = block_sum(s_bb);
    const double pz = block_sum(s_rz);
    if (threadIdx.x == 0) {
        partials2[blockIdx.x] = pr;
        partials3[blockIdx.x] = pb;
        partials4[blockIdx.x] = pz;
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = pt;
        __threadfence();
        last = atomicAdd(&S->count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, rr = 0.0, bb = 0.0, rz = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += RT) {
        a += ((volatile double *)partials)[k];
        rr += ((volatile double *)partials2)[k];
        bb += ((volatile double *)partials3)[k];
        rz += ((volatile double *)partials4)[k];
    }
    a = block_sum(a);
    rr = block_sum(rr);
    bb = block_sum(bb);
    rz = block_sum(rz);
    if (threadIdx.x == 0) {
        S->count = 0;
        S->rr_new = a;
        S->rr = rr;
        S->rz = JAC ? rz : rr;
        S->bb = bb;
        S->iters = 0;
        S->conv = (a <= S->tol2 * bb) ? 1 : 0;
    }
}

// alpha = rr / <p, q>.  V4: four consecutive elements per step (16-byte
// loads; every vector 16-byte aligned and N a multiple of 4).
template <bool V4>
__global__ void __launch_bounds__(RT) cg_k2(int64_t N, const float *__restrict__ p,
                                            const float *__restrict__ q, double *partials, CgState *S) {
    if (S->conv) return;
    FFAcc s;
    const int64_t i0 = (int64_t)blockIdx.x * RT + threadIdx.x, stride = (int64_t)gridDim.x * RT;
    if constexpr (V4) {
        // two accumulators, so that the four products of a load do not form
        // one dependent chain (one chain left fewer loads in flight: 15.3
        // against 13.8 us per launch for the scalar pass at 2048^2)
        const float4 *p4 = reinterpret_cast<const float4 *>(p), *q4 = reinterpret_cast<const float4 *>(q);
        FFAcc s2;
#pragma unroll 2
        for (int64_t i = i0; i < N / 4; i += stride) {
            const float4 a = p4[i], b = q4[i];
            ff_add_prod(s, a.x, b.x);
            ff_add_prod(s2, a.y, b.y);
            ff_add_prod(s, a.z, b.z);
            ff_add_prod(s2, a.w, b.w);
        }
        ff_add(s, s2.hi);
        s.lo = __fadd_rn(s.lo, s2.lo);
    } else {
        for (int64_t i = i0; i < N; i += stride) ff_add_prod(s, p[i], q[i]);
    }
    double part = block_sum_ff(s);
    double tot;
    if (finish_reduction(part, partials, &S->count, tot)) {
        S->pq = tot;
        S->alpha = S->rz / tot;   // rz = rr without preconditioner
    }
}

// x += alpha p ; r -= alpha q ; rr_new = <r, r> (JAC: and <r, z>) ; beta ; flag
template <bool JAC, bool V4>
__global__ void __launch_bounds__(RT) cg_k3(int64_t N, float *__restrict__ x, const float *__restrict__ p,
                                            float *__restrict__ r, const float *__restrict__ q,
                                            const float *__restrict__ inv_d, double *partials,
                                            double *partials2, CgState *S) {
    if (S->conv) return;
    const float alpha = (float)S->alpha;
    FFAcc s, sz;
    const int64_t i0 = (int64_t)blockIdx.x * RT + threadIdx.x, stride = (int64_t)gridDim.x * RT;
    auto one = [&](float &xi, float pi, float &ri, float qi, float di) {
        xi += alpha * pi;
        ri = ri - alpha * qi;
        ff_add_prod(s, ri, ri);
        if (JAC) ff_add_prod(sz, ri, ri * di);
    };
    if constexpr (V4) {
        float4 *x4 = reinterpret_cast<float4 *>(x), *r4 = reinterpret_cast<float4 *>(r);
        const float4 *p4 = reinterpret_cast<const float4 *>(p), *q4 = reinterpret_cast<const float4 *>(q);
        const float4 *d4 = reinterpret_cast<const float4 *>(inv_d);
#pragma unroll 2
        for (int64_t i = i0; i < N / 4; i += stride) {
            float4 xv = x4[i], rv = r4[i];
            const float4 pv = p4[i], qv = q4[i];
            const float4 dv = JAC ? d4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            one(xv.x, pv.x, rv.x, qv.x, dv.x);
            one(xv.y, pv.y, rv.y, qv.y, dv.y);
            one(xv.z, pv.z, rv.z, qv.z, dv.z);
            one(xv.w, pv.w, rv.w, qv.w, dv.w);
            x4[i] = xv;
            r4[i] = rv;
        }
    } else {
        for (int64_t i = i0; i < N; i += stride) {
            float xi = x[i], ri = r[i];
            one(xi, p[i], ri, q[i], JAC ? inv_d[i] : 0.f);
            x[i] = xi;
            r[i] = ri;
        }
    }
    double part = block_sum_ff(s);
    double tot, rz = 0.0;
    bool fin;
    if (JAC) fin = finish_reduction2(part, block_sum_ff(sz), partials, partials2, &S->count, tot, rz);
    else fin = finish_reduction(part, partials, &S->count, tot);
    if (fin) {
        if (JAC) {
            S->beta = rz / S->rz;
            S->rz = rz;
        } else {
            S->beta = tot / S->rr;
            S->rz = tot;
        }
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

// p <- z + beta p (z = r, or r / d) ; q <- p (QP: for the scatter operator,
// which accumulates dt A p into q; the gather operator writes q itself)
template <bool JAC, bool QP, bool V4>
__global__ void __launch_bounds__(RT) cg_k4(int64_t N, const float *__restrict__ r, const float *__restrict__ inv_d,
                                            float *__restrict__ p, float *__restrict__ q, const CgState *S) {
    if (S->conv) return;
    const float beta = (float)S->beta;
    const int64_t i0 = (int64_t)blockIdx.x * RT + threadIdx.x, stride = (int64_t)gridDim.x * RT;
    if constexpr (V4) {
        const float4 *r4 = reinterpret_cast<const float4 *>(r), *d4 = reinterpret_cast<const float4 *>(inv_d);
        float4 *p4 = reinterpret_cast<float4 *>(p), *q4 = reinterpret_cast<float4 *>(q);
        for (int64_t i = i0; i < N / 4; i += stride) {
            const float4 rv = r4[i], pv = p4[i];
            float4 z = rv;
            if (JAC) {
                const float4 dv = d4[i];
                z = make_float4(rv.x * dv.x, rv.y * dv.y, rv.z * dv.z, rv.w * dv.w);
            }
            const float4 np = make_float4(z.x + beta * pv.x, z.y + beta * pv.y, z.z + beta * pv.z,
                                          z.w + beta * pv.w);
            p4[i] = np;
            if (QP) q4[i] = np;
        }
    } else {
        for (int64_t i = i0; i < N; i += stride) {
            const float zi = JAC ? r[i] * inv_d[i] : r[i];
            const float pi = zi + beta * p[i];
            p[i] = pi;
            if (QP) q[i] = pi;
        }
    }
}

}  // namespace

struct CgWorkspace {
    float *r, *p, *q, *z;
    double *acc64;  // aliases q and z (8 bytes per point), used between iterations
    float *inv_d;   // 1 / (1 + dt A_zz) of the Jacobi-preconditioned solve
    double *partials, *partials2, *partials3, *partials4;
    CgState *S;
};

static size_t cg_ws_bytes(int64_t N) {
    return 5 * (size_t)N * sizeof(float) + 4 * vec_blocks() * sizeof(double) + 256 + sizeof(CgState);
}

static adlbr_status cg_workspace(adlbr_stencils *s, CgWorkspace &W) {
    size_t need = cg_ws_bytes(s->N);
    if (!s->ws || s->ws_bytes < need) {
        if (s->ws) cudaFree(s->ws);
        s->ws = nullptr;
        ADLBR_CUDA(cudaMalloc(&s->ws, need));
        s->ws_bytes = need;
    }
    char *b = (char *)s->ws;
    W.r = (float *)b;
    W.p = W.r + s->N;
    W.q = W.p + s->N;
    W.z = W.q + s->N;
    W.acc64 = (double *)W.q;
    W.inv_d = W.z + s->N;
    W.partials = (double *)(W.inv_d + s->N);
    W.partials2 = W.partials + vec_blocks();
    W.partials3 = W.partials2 + vec_blocks();
    W.partials4 = W.partials3 + vec_blocks();
    uintptr_t a = (uintptr_t)(W.partials4 + vec_blocks());
    a = (a + 255) & ~(uintptr_t)255;
    W.S = (CgState *)a;
    return ADLBR_OK;
}

// The three vector kernels of one CG iteration after the operator.
template <bool V4>
static void cg_vec_iteration(int64_t N, float *x, const CgWorkspace &W, bool jac, bool gather, cudaStream_t cs) {
    cg_k2<V4><<<vec_blocks(), RT, 0, cs>>>(N, W.p, W.q, W.partials, W.S);
    if (jac) {
        cg_k3<true, V4><<<vec_blocks(), RT, 0, cs>>>(N, x, W.p, W.r, W.q, W.inv_d, W.partials, W.partials2, W.S);
        if (gather) cg_k4<true, false, V4><<<vec_blocks(), RT, 0, cs>>>(N, W.r, W.inv_d, W.p, W.q, W.S);
        else cg_k4<true, true, V4><<<vec_blocks(), RT, 0, cs>>>(N, W.r, W.inv_d, W.p, W.q, W.S);
    } else {
        cg_k3<false, V4><<<vec_blocks(), RT, 0, cs>>>(N, x, W.p, W.r, W.q, W.inv_d, W.partials, W.partials2, W.S);
        if (gather) cg_k4<false, false, V4><<<vec_blocks(), RT, 0, cs>>>(N, W.r, W.inv_d, W.p, W.q, W.S);
        else cg_k4<false, true, V4><<<vec_blocks(), RT, 0, cs>>>(N, W.r, W.inv_d, W.p, W.q, W.S);
    }
}

static const int *conv_flag(const CgState *S) {
    return (const int *)((const char *)S + offsetof(CgState, conv));
}

// CG on FP32 vectors with FP64 reductions, wrapped in iterative refinement:
// every (re)start measures the true residual b - (I + dt A) x with the
// operator accumulated in FP64, stops if it meets rtol, and otherwise runs CG
// on the FP32-rounded residual until the recursive residual meets rtol.
static adlbr_status cg_impl(adlbr_stencils *s, const float *b, float *x, double dt, double rtol, int maxit,
                            int *iters_out, double *relres_out, int every, CgHook hook, void *ctx, bool jac,
                            cudaStream_t st);

adlbr_status run_cg(adlbr_stencils *s, const float *b, float *x, double dt, double rtol, int maxit,
                    int *iters_out, double *relres_out, cudaStream_t st) {
    return cg_impl(s, b, x, dt, rtol, maxit, iters_out, relres_out, 8, nullptr, nullptr, false, st);
}

adlbr_status run_pcg_jacobi(adlbr_stencils *s, const float *b, float *x, double dt, double rtol, int maxit,
                            int *iters_out, double *relres_out, cudaStream_t st) {
    return cg_impl(s, b, x, dt, rtol, maxit, iters_out, relres_out, 8, nullptr, nullptr, true, st);
}

// As run_cg; when hook != NULL it is called (on the host, work enqueued on
// st) with the current residual and iterate every `every` iterations of the
// first CG round, while the solve has not converged.
adlbr_status run_cg_hooked(adlbr_stencils *s, const float *b, float *x, double dt, double rtol,
                           int maxit, int *iters_out, double *relres_out, int every, CgHook hook,
                           void *ctx, cudaStream_t st) {
    return cg_impl(s, b, x, dt, rtol, maxit, iters_out, relres_out, every, hook, ctx, false, st);
}

static adlbr_status cg_impl(adlbr_stencils *s, const float *b, float *x, double dt, double rtol, int maxit,
                            int *iters_out, double *relres_out, int every, CgHook hook, void *ctx, bool jac,
                            cudaStream_t st) {
    CgWorkspace W;
    if (adlbr_status e = cg_workspace(s, W)) return e;
    const int64_t N = s->N;
    bool gather = false;   // q = p + dt A p by the gather form of the operator
    if (adlbr_status e = choose_gather(s, 2, &gather, st)) return e;
    if (jac)
        if (adlbr_status e = launch_jacobi_inverse(s, dt, W.inv_d, st)) return e;
    CgState init = {};
    init.tol2 = rtol * rtol;
    CgState host = {};
    int total_iters = 0;
    double relres = INFINITY, prev = INFINITY;
    int round_iters = 0;   // CG iterations of the last round
    bool cg_converged = false;
    const int kMaxRestarts = 3;
    for (int restart = 0; restart <= kMaxRestarts; ++restart) {
        // The first residual only starts CG, so it takes the FP32 operator;
        // every later round measures the true residual with the operator
        // accumulated in FP64, and only those decide convergence.
        const bool first32 = restart == 0;
        init.max_iters = maxit - total_iters;
        ADLBR_CUDA(cudaMemcpyAsync(W.S, &init, sizeof(CgState), cudaMemcpyHostToDevice, st));
        if (first32) {
            float *acc32 = W.q;   // q is set from p below
            ADLBR_CUDA(cudaMemsetAsync(acc32, 0, N * sizeof(float), st));
            if (adlbr_status e = launch_accumulate(s, x, acc32, ADLBR_F32, dt, nullptr, st)) return e;
            if (jac)
                cg_restart_kernel<true, float><<<vec_blocks(), RT, 0, st>>>(
                    N, b, x, acc32, W.inv_d, W.r, W.p, W.partials, W.partials2, W.partials3, W.partials4, W.S);
            else
                cg_restart_kernel<false, float><<<vec_blocks(), RT, 0, st>>>(
                    N, b, x, acc32, W.inv_d, W.r, W.p, W.partials, W.partials2, W.partials3, W.partials4, W.S);
        } else {
            ADLBR_CUDA(cudaMemsetAsync(W.acc64, 0, N * sizeof(double), st));
            if (adlbr_status e = launch_accumulate_f64(s, x, W.acc64, dt, st)) return e;
            if (jac)
                cg_restart_kernel<true, double><<<vec_blocks(), RT, 0, st>>>(
                    N, b, x, W.acc64, W.inv_d, W.r, W.p, W.partials, W.partials2, W.partials3, W.partials4, W.S);
            else
                cg_restart_kernel<false, double><<<vec_blocks(), RT, 0, st>>>(
                    N, b, x, W.acc64, W.inv_d, W.r, W.p, W.partials, W.partials2, W.partials3, W.partials4, W.S);
        }
        ADLBR_CUDA(cudaGetLastError());
        // q = p (q aliases acc64, which the restart kernel has consumed)
        ADLBR_CUDA(cudaMemcpyAsync(W.q, W.p, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        ADLBR_CUDA(cudaMemcpyAsync(&host, W.S, sizeof(CgState), cudaMemcpyDeviceToHost, st));
        ADLBR_CUDA(cudaStreamSynchronize(st));
        if (!std::isfinite(host.bb) || !std::isfinite(host.rr_new)) {
            if (iters_out) *iters_out = total_iters;
            return fail(ADLBR_E_NONFINITE, "non-finite right-hand side or iterate in CG");
        }
        relres = host.bb > 0 ? std::sqrt(host.rr_new / host.bb) : 0.0;
        // stop when the true residual meets rtol, when refinement stopped
        // paying (x is FP32: the true residual floors near eps32 |I + dt A|),
        // or when the budget is spent
        if ((!first32 && relres <= rtol) || total_iters >= maxit || restart == kMaxRestarts) break;
        // (not after a round that ran no iteration: the first, FP32 residual
        // can already meet rtol where the FP64 one does not)
        if (restart > 0 && round_iters > 0 && (relres <= 10.0 * rtol || !(relres < 0.5 * prev))) break;
        prev = relres;
        const int chunk = every > 0 ? every : 8;
        // 16-byte vector passes when every vector allows them (the workspace
        // vectors are N floats apart, so N % 4 == 0 aligns them; x is the caller's)
        const bool v4 = N % 4 == 0 && (uintptr_t)x % 16 == 0;
        auto enqueue_chunk = [&](cudaStream_t cs) -> adlbr_status {
            for (int k = 0; k < chunk; ++k) {
                if (gather) {
                    if (adlbr_status e = launch_pull(s, W.p, ADLBR_F32, W.q, ADLBR_F32, 1.0, dt, conv_flag(W.S), cs))
                        return e;
                } else if (adlbr_status e = launch_accumulate(s, W.p, W.q, ADLBR_F32, dt, conv_flag(W.S), cs)) {
                    return e;
                }
                if (v4)
                    cg_vec_iteration<true>(N, x, W, jac, gather, cs);
                else
                    cg_vec_iteration<false>(N, x, W, jac, gather, cs);
            }
            ADLBR_CUDA(cudaGetLastError());
            return ADLBR_OK;
        };
        // Without a hook the chunk (4 kernels per iteration, each a no-op
        // once the device flag is set) is captured once as a CUDA graph and
        // replayed; the host reads the flag after every replay.
        ChunkGraph graph;
        if (!hook)
            if (adlbr_status e = graph.capture(enqueue_chunk)) return e;
        int it = 0;
        while (it < maxit - total_iters) {
            if (hook && restart == 0)
                if (adlbr_status e = hook(ctx, W.r, x, it, st)) return e;
            if (graph.exec) {
                ADLBR_CUDA(cudaGraphLaunch(graph.exec, st));
            } else if (adlbr_status e = enqueue_chunk(st)) {
                return e;
            }
            it += chunk;
            ADLBR_CUDA(cudaMemcpyAsync(&host, W.S, sizeof(CgState), cudaMemcpyDeviceToHost, st));
            ADLBR_CUDA(cudaStreamSynchronize(st));
            if (host.conv) break;
        }
        total_iters += host.iters;
        round_iters = host.iters;
        cg_converged = host.conv == 1;
        if (host.conv == 3) {
            if (iters_out) *iters_out = total_iters;
            return fail(ADLBR_E_NONFINITE, "CG residual became non-finite after %d iterations", total_iters);
        }
    }
    if (iters_out) *iters_out = total_iters;
    if (relres_out) *relres_out = relres;
    set_last_residual_met(relres <= rtol);
    if (!(relres <= rtol) && !cg_converged)
        return fail(ADLBR_E_NOT_CONVERGED, "CG stopped at relative residual %.3e after %d iterations",
                    relres, total_iters);
    return ADLBR_OK;
}

}  // namespace adlbr

// Operator application A u = (1/2) grad E_h(u) (Eq. def:E*, h = 1) and the
// canonical export of the stencils.
//
// The operator is a sum over the directed edges (z, e), e in V(z), of
// gamma_z(e) (u(z) - u(z+e)) added at z and subtracted at z+e.  Scatter
// formulation: one thread per point z gathers its own edges' contributions
// into a register and pushes the opposite contributions to the far ends
// with fire-and-forget atomics (red.global.add), which L2 performs.  Pairs
// that leave the grid are dropped (Neumann rule of Sec. 1) or wrapped.
#include "internal.cuh"

namespace adlbr {

namespace {

__device__ __forceinline__ int wrap(int c, int n) {
    c %= n;
    return c < 0 ? c + n : c;
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

template <typename UT>
__global__ void __launch_bounds__(256) apply2d_scatter(int nx, int ny, int bc,
                                                       const short4 *__restrict__ offs,
                                                       const void *__restrict__ wbase, adlbr_dtype wt,
                                                       const UT *__restrict__ u,
                                                       typename UTraits<UT>::acc *__restrict__ Au) {
    using AT = typename UTraits<UT>::acc;
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
        if (w[k] == (AT)0) continue;
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
            const AT flux = w[k] * (uz - to_acc(u[zn]));
            acc += flux;
            atomicAdd(Au + zn, -flux);
        }
    }
    atomicAdd(Au + z, acc);
}

template <typename UT>
__global__ void __launch_bounds__(128) apply3d_scatter(int nx, int ny, int nz, int bc,
                                                       const char4 *__restrict__ offs,
                                                       const void *__restrict__ wbase, adlbr_dtype wt,
                                                       const UT *__restrict__ u,
                                                       typename UTraits<UT>::acc *__restrict__ Au) {
    using AT = typename UTraits<UT>::acc;
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
        if (w[q] == (AT)0) continue;
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
            const AT flux = w[q] * (uz - to_acc(u[zz]));
            acc += flux;
            atomicAdd(Au + zz, -flux);
        }
    }
    atomicAdd(Au + z, acc);
}

// u <- u - dt * acc ; acc <- 0
template <typename UT>
__global__ void axpy_zero_kernel(int64_t N, UT *__restrict__ u,
                                 typename UTraits<UT>::acc *__restrict__ acc, double dt) {
    using AT = typename UTraits<UT>::acc;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    AT a = acc[i];
    acc[i] = (AT)0;
    u[i] = from_acc<UT>(to_acc(u[i]) - (AT)dt * a);
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
    // insertion sort (K <= 6)
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

template <typename UT>
static adlbr_status apply_t(const adlbr_stencils *s, const UT *u, typename UTraits<UT>::acc *Au,
                            cudaStream_t st) {
    using AT = typename UTraits<UT>::acc;
    ADLBR_CUDA(cudaMemsetAsync(Au, 0, (size_t)s->N * sizeof(AT), st));
    if (s->dim == 2) {
        const int threads = 256;
        dim3 grid(blocks_for(s->n[0], threads), (unsigned)s->n[1]);
        apply2d_scatter<UT><<<grid, threads, 0, st>>>((int)s->n[0], (int)s->n[1], s->bc,
                                                      (const short4 *)s->offs, s->w, s->w_t, u, Au);
    } else {
        const int threads = 128;
        dim3 grid(blocks_for(s->n[0], threads), (unsigned)s->n[1], (unsigned)s->n[2]);
        apply3d_scatter<UT><<<grid, threads, 0, st>>>((int)s->n[0], (int)s->n[1], (int)s->n[2],
                                                      s->bc, (const char4 *)s->offs, s->w, s->w_t,
                                                      u, Au);
    }
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

adlbr_status launch_apply(const adlbr_stencils *s, const void *u, void *Au, adlbr_dtype u_t,
                          cudaStream_t st) {
    switch (u_t) {
    case ADLBR_F64: return apply_t<double>(s, (const double *)u, (double *)Au, st);
    case ADLBR_F32: return apply_t<float>(s, (const float *)u, (float *)Au, st);
    case ADLBR_F16: return apply_t<__half>(s, (const __half *)u, (float *)Au, st);
    case ADLBR_BF16: return apply_t<__nv_bfloat16>(s, (const __nv_bfloat16 *)u, (float *)Au, st);
    }
    return fail(ADLBR_E_ARG, "bad u dtype %d", (int)u_t);
}

adlbr_status launch_axpy_zero(const adlbr_stencils *s, void *u, void *acc, adlbr_dtype u_t,
                              double dt, cudaStream_t st) {
    const int threads = 256;
    unsigned blocks = blocks_for(s->N, threads);
    switch (u_t) {
    case ADLBR_F64:
        axpy_zero_kernel<double><<<blocks, threads, 0, st>>>(s->N, (double *)u, (double *)acc, dt);
        break;
    case ADLBR_F32:
        axpy_zero_kernel<float><<<blocks, threads, 0, st>>>(s->N, (float *)u, (float *)acc, dt);
        break;
    case ADLBR_F16:
        axpy_zero_kernel<__half><<<blocks, threads, 0, st>>>(s->N, (__half *)u, (float *)acc, dt);
        break;
    case ADLBR_BF16:
        axpy_zero_kernel<__nv_bfloat16><<<blocks, threads, 0, st>>>(s->N, (__nv_bfloat16 *)u,
                                                                    (float *)acc, dt);
        break;
    default: return fail(ADLBR_E_ARG, "bad u dtype %d", (int)u_t);
    }
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

}  // namespace adlbr

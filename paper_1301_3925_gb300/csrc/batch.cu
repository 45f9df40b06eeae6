// Batched explicit steps over images and volumes of uneven sizes (not in the
// paper: the serving form of its explicit scheme, Sec. 4.4, u <- u - dt A u
// per item).
//
// A batch fixes its items (stencil handles, FP32 u buffers, time steps) and
// owns one accumulator array for all of them.  One step is
//   memset (all accumulators and the two tile counters)
//   -> one persistent kernel over the 2D tiles of every image
//      (op::tile2d), then one over the 3D blocks of every volume
//      (op::tile3d); tiles are handed out by an atomic counter, so uneven
//      items balance across the SMs.  Two kernels rather than one that takes
//      both: each is compiled for its own operator only, so it keeps the
//      register count, and the occupancy, of the single-grid kernel
//   -> one finalize kernel over chunks of every item (u -= acc).
// The step is recorded once as a CUDA graph and replayed.  The tile shapes
// (2D tile, 3D block) come from an autotuner that times each accumulate
// kernel for every candidate on the batch itself (the accumulate kernels
// write only the batch's accumulator, so tuning leaves u untouched).
#include <algorithm>
#include <cstring>
#include <vector>

#include "operator.cuh"

struct adlbr_batch_item {
    int dim, bc, nx, ny, nz;
    adlbr_dtype wt;
    const void *offs;
    const void *w;
    float *u;
    float *acc;
    float scale;
    int64_t N;
};

struct adlbr_batch_tile {
    int item, x0, y0, z0;
};

struct adlbr_batch_chunk {
    int item;
    int64_t start, len;
};

struct adlbr_batch {
    int device;
    int n_items;
    int cand2, cand3;            // chosen 2D tile and 3D block candidates
    double tuned_ms;             // its accumulate time
    int64_t points;
    adlbr_batch_item *items;     // device
    adlbr_batch_tile *tiles;     // device (for the chosen shapes): 2D tiles, then 3D blocks
    int n_tiles, n_tiles2;
    adlbr_batch_chunk *chunks;   // device
    int n_chunks;
    float *acc;                  // device, sum of N_i floats + tile counter
    size_t acc_bytes;
    unsigned *counter;           // two tile counters (2D, 3D), inside acc's allocation
    int grid2, grid3;            // persistent CTAs of the two accumulate kernels
    int sms;
    adlbr::ChunkGraph *graph;
    std::vector<adlbr_batch_item> host_items;
};

namespace adlbr {

namespace {

constexpr int BNT = 256;             // threads per CTA of the batched kernels
constexpr int kChunk = 1 << 16;      // finalize chunk (floats)

// candidates of the autotuner (each one an instantiation of its kernel)
struct Shape2 {
    int tw, th;        // 2D tile
};
struct Shape3 {
    int bx, by, bz;    // 3D block (bz planes per thread)
};
constexpr Shape2 kShapes2[] = {{64, 32}, {64, 16}, {32, 32}, {128, 16}};
constexpr Shape3 kShapes3[] = {{32, 8, 4}, {64, 4, 4}, {32, 8, 8}};
constexpr int kNum2 = sizeof(kShapes2) / sizeof(kShapes2[0]);
constexpr int kNum3 = sizeof(kShapes3) / sizeof(kShapes3[0]);

// The next tile of this kernel's range [first, last) from its counter, the
// same for every thread of the block (-1 once the range is exhausted).
__device__ __forceinline__ int next_tile(unsigned *counter, int first, int last) {
    __shared__ int next;
    __syncthreads();   // every thread has read `next` of the previous round
    if (threadIdx.x == 0) next = first + (int)atomicAdd(counter, 1u);
    __syncthreads();
    return next < last ? next : -1;
}

template <int TW, int TH>
__global__ void __launch_bounds__(BNT) batch_accumulate2d(const adlbr_batch_item *__restrict__ items,
                                                          const adlbr_batch_tile *__restrict__ tiles,
                                                          int n_tiles2, unsigned *counter) {
    constexpr int WX = 16;
    extern __shared__ __align__(16) float smem[];
    for (;;) {
        const int t = next_tile(counter, 0, n_tiles2);
        if (t < 0) return;
        const adlbr_batch_tile tl = tiles[t];
        const adlbr_batch_item it = items[tl.item];
        if (it.wt == ADLBR_F16)
            op::tile2d<float, TW, TH, BNT, WX, true>(it.nx, it.ny, it.bc, it.scale, (const short4 *)it.offs,
                                                     nullptr, it.w, it.wt, it.u, it.acc, tl.x0, tl.y0, smem);
        else
            op::tile2d<float, TW, TH, BNT, WX, false>(it.nx, it.ny, it.bc, it.scale, (const short4 *)it.offs,
                                                      nullptr, it.w, it.wt, it.u, it.acc, tl.x0, tl.y0, smem);
    }
}

template <int BX, int BY, int BZ>
__global__ void __launch_bounds__(BNT, 4) batch_accumulate3d(const adlbr_batch_item *__restrict__ items,
                                                             const adlbr_batch_tile *__restrict__ tiles,
                                                             int n_tiles2, int n_tiles, unsigned *counter) {
    static_assert(BX * BY == BNT, "one thread per (x, y) of a 3D block");
    extern __shared__ __align__(16) float smem[];
    for (;;) {
        const int t = next_tile(counter + 1, n_tiles2, n_tiles);
        if (t < 0) return;
        const adlbr_batch_tile tl = tiles[t];
        const adlbr_batch_item it = items[tl.item];
        if (it.wt == ADLBR_F16)
            op::tile3d<float, BX, BY, BZ, true>(it.nx, it.ny, it.nz, it.bc, it.scale, (const char4 *)it.offs,
                                                it.w, it.wt, it.u, it.acc, tl.x0, tl.y0, tl.z0, smem);
        else
            op::tile3d<float, BX, BY, BZ, false>(it.nx, it.ny, it.nz, it.bc, it.scale, (const char4 *)it.offs,
                                                 it.w, it.wt, it.u, it.acc, tl.x0, tl.y0, tl.z0, smem);
    }
}

__global__ void __launch_bounds__(BNT) batch_finalize_kernel(const adlbr_batch_item *__restrict__ items,
                                                             const adlbr_batch_chunk *__restrict__ chunks,
                                                             int n_chunks) {
    for (int c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const adlbr_batch_chunk ch = chunks[c];
        const adlbr_batch_item it = items[ch.item];
        float *u = it.u + ch.start;
        const float *a = it.acc + ch.start;
        if ((((uintptr_t)u | (uintptr_t)a) & 15) == 0 && (ch.len & 3) == 0) {
            float4 *u4 = reinterpret_cast<float4 *>(u);
            const float4 *a4 = reinterpret_cast<const float4 *>(a);
            for (int64_t i = threadIdx.x; i < ch.len / 4; i += BNT) {
                const float4 av = a4[i], uv = u4[i];
                u4[i] = make_float4(uv.x - av.x, uv.y - av.y, uv.z - av.z, uv.w - av.w);
            }
        } else {
            for (int64_t i = threadIdx.x; i < ch.len; i += BNT) u[i] -= a[i];
        }
    }
}

// Work list for shapes (s2, s3): the 2D items by TW x TH tiles, then the 3D
// items by BX x BY x BZ blocks, the largest items first in each part.
std::vector<adlbr_batch_tile> make_tiles(const std::vector<adlbr_batch_item> &items, const Shape2 &s2,
                                         const Shape3 &s3, int *n2) {
    std::vector<int> order(items.size());
    for (size_t i = 0; i < items.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return items[a].N > items[b].N; });
    std::vector<adlbr_batch_tile> out;
    for (int i : order) {
        const adlbr_batch_item &it = items[i];
        if (it.dim != 2) continue;
        for (int y = 0; y < it.ny; y += s2.th)
            for (int x = 0; x < it.nx; x += s2.tw) out.push_back({i, x, y, 0});
    }
    *n2 = (int)out.size();
    for (int i : order) {
        const adlbr_batch_item &it = items[i];
        if (it.dim != 3) continue;
        for (int z = 0; z < it.nz; z += s3.bz)
            for (int y = 0; y < it.ny; y += s3.by)
                for (int x = 0; x < it.nx; x += s3.bx) out.push_back({i, x, y, z});
    }
    return out;
}

// Persistent grid of a kernel: its resident blocks per SM times the SMs,
// at most one block per tile.
template <typename K>
adlbr_status persistent_grid(K kern, size_t smem, int tiles, int sms, int *grid) {
    ADLBR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ADLBR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BNT, smem));
    *grid = std::max(1, std::min(tiles, std::max(1, per_sm) * sms));
    return ADLBR_OK;
}

// prepare = true: set the kernel's shared-memory limit and compute its
// persistent grid (outside any graph capture); false: launch it.
template <int TW, int TH>
adlbr_status acc2_t(adlbr_batch *b, bool prepare, cudaStream_t st) {
    using T = op::Tile<TW, TH, BNT, 16>;
    const size_t smem = 2 * (size_t)T::P * T::WH * sizeof(float);
    auto kern = batch_accumulate2d<TW, TH>;
    if (prepare) return persistent_grid(kern, smem, b->n_tiles2, b->sms, &b->grid2);
    if (b->n_tiles2 > 0) {
        kern<<<b->grid2, BNT, smem, st>>>(b->items, b->tiles, b->n_tiles2, b->counter);
        ADLBR_CUDA(cudaGetLastError());
    }
    return ADLBR_OK;
}

template <int BX, int BY, int BZ>
adlbr_status acc3_t(adlbr_batch *b, bool prepare, cudaStream_t st) {
    const size_t smem = 2 * (size_t)op::Block3<BX, BY, BZ>::CELLS * sizeof(float);
    auto kern = batch_accumulate3d<BX, BY, BZ>;
    const int n3 = b->n_tiles - b->n_tiles2;
    if (prepare) return persistent_grid(kern, smem, n3, b->sms, &b->grid3);
    if (n3 > 0) {
        kern<<<b->grid3, BNT, smem, st>>>(b->items, b->tiles, b->n_tiles2, b->n_tiles, b->counter);
        ADLBR_CUDA(cudaGetLastError());
    }
    return ADLBR_OK;
}

adlbr_status acc2(adlbr_batch *b, int c, bool prepare, cudaStream_t st) {
    switch (c) {
    case 0: return acc2_t<64, 32>(b, prepare, st);
    case 1: return acc2_t<64, 16>(b, prepare, st);
    case 2: return acc2_t<32, 32>(b, prepare, st);
    case 3: return acc2_t<128, 16>(b, prepare, st);
    }
    return fail(ADLBR_E_ARG, "bad 2D shape candidate %d", c);
}

adlbr_status acc3(adlbr_batch *b, int c, bool prepare, cudaStream_t st) {
    switch (c) {
    case 0: return acc3_t<32, 8, 4>(b, prepare, st);
    case 1: return acc3_t<64, 4, 4>(b, prepare, st);
    case 2: return acc3_t<32, 8, 8>(b, prepare, st);
    }
    return fail(ADLBR_E_ARG, "bad 3D shape candidate %d", c);
}

adlbr_status upload_tiles(adlbr_batch *b, const std::vector<adlbr_batch_tile> &t, int n2, cudaStream_t st) {
    if (b->tiles) cudaFree(b->tiles);
    b->tiles = nullptr;
    ADLBR_CUDA(cudaMalloc(&b->tiles, std::max<size_t>(1, t.size()) * sizeof(adlbr_batch_tile)));
    ADLBR_CUDA(cudaMemcpyAsync(b->tiles, t.data(), t.size() * sizeof(adlbr_batch_tile),
                               cudaMemcpyHostToDevice, st));
    ADLBR_CUDA(cudaStreamSynchronize(st));
    b->n_tiles = (int)t.size();
    b->n_tiles2 = n2;
    return ADLBR_OK;
}

// Work list of candidates (c2, c3) on the device and the launch geometry of
// both kernels.
adlbr_status use_shapes(adlbr_batch *b, int c2, int c3, cudaStream_t st) {
    int n2 = 0;
    const std::vector<adlbr_batch_tile> t = make_tiles(b->host_items, kShapes2[c2], kShapes3[c3], &n2);
    if (adlbr_status e = upload_tiles(b, t, n2, st)) return e;
    if (adlbr_status e = acc2(b, c2, true, st)) return e;
    return acc3(b, c3, true, st);
}

// One step, enqueued on st (also what the graph records).
adlbr_status enqueue_step(adlbr_batch *b, cudaStream_t st) {
    ADLBR_CUDA(cudaMemsetAsync(b->acc, 0, b->acc_bytes, st));
    if (adlbr_status e = acc2(b, b->cand2, false, st)) return e;
    if (adlbr_status e = acc3(b, b->cand3, false, st)) return e;
    batch_finalize_kernel<<<std::max(1, std::min(b->n_chunks, 4 * b->sms)), BNT, 0, st>>>(
        b->items, b->chunks, b->n_chunks);
    ADLBR_CUDA(cudaGetLastError());
    return ADLBR_OK;
}

void free_batch(adlbr_batch *b) {
    if (!b) return;
    delete b->graph;
    if (b->items) cudaFree(b->items);
    if (b->tiles) cudaFree(b->tiles);
    if (b->chunks) cudaFree(b->chunks);
    if (b->acc) cudaFree(b->acc);
    delete b;
}

}  // namespace

}  // namespace adlbr

using namespace adlbr;

extern "C" {

adlbr_status adlbr_batch_create(int n_items, adlbr_stencils *const *s, float *const *u, const double *dt,
                                int autotune, adlbr_batch **out, cudaStream_t stream) {
    if (!out) return fail(ADLBR_E_ARG, "null output");
    *out = nullptr;
    if (n_items < 1 || !s || !u || !dt) return fail(ADLBR_E_ARG, "empty batch or null arrays");
    int dev = 0;
    ADLBR_CUDA(cudaGetDevice(&dev));
    adlbr_batch *b = new adlbr_batch();
    b->device = dev;
    b->n_items = n_items;
    if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) b->sms = 1;
    b->cand2 = b->cand3 = 0;
    b->tuned_ms = 0.0;
    // items and accumulator layout (each item's accumulator 16-byte aligned)
    int64_t off = 0;
    for (int i = 0; i < n_items; ++i) {
        const adlbr_stencils *h = s[i];
        if (!h || !u[i] || !(dt[i] >= 0.0)) {
            free_batch(b);
            return fail(ADLBR_E_ARG, "item %d: null handle / buffer or bad dt", i);
        }
        if (h->device != dev) {
            free_batch(b);
            return fail(ADLBR_E_ARG, "item %d lives on device %d, current device is %d", i, h->device, dev);
        }
        if (h->scheme != ADLBR_SCHEME_ADLBR) {
            free_batch(b);
            return fail(ADLBR_E_ARG, "item %d: the batched step takes AD-LBR stencils", i);
        }
        adlbr_batch_item it = {};
        it.dim = h->dim;
        it.bc = h->bc;
        it.nx = (int)h->n[0];
        it.ny = (int)h->n[1];
        it.nz = h->dim == 3 ? (int)h->n[2] : 1;
        it.wt = h->w_t;
        it.offs = h->offs;
        it.w = h->w;
        it.u = u[i];
        it.scale = (float)dt[i];
        it.N = h->N;
        it.acc = reinterpret_cast<float *>((uintptr_t)off);   // offset for now
        off += (h->N + 3) / 4 * 4;
        b->points += h->N;
        b->host_items.push_back(it);
    }
    b->acc_bytes = (size_t)off * sizeof(float) + 256;
    cudaError_t ce = cudaMalloc(&b->acc, b->acc_bytes);
    if (ce != cudaSuccess) {
        free_batch(b);
        return cuda_fail(ce, "cudaMalloc (batch accumulator)");
    }
    b->counter = reinterpret_cast<unsigned *>(b->acc + off);
    for (auto &it : b->host_items) it.acc = b->acc + (int64_t)(uintptr_t)it.acc;
    // finalize chunks
    std::vector<adlbr_batch_chunk> chunks;
    for (int i = 0; i < n_items; ++i)
        for (int64_t st = 0; st < b->host_items[i].N; st += kChunk)
            chunks.push_back({i, st, std::min<int64_t>(kChunk, b->host_items[i].N - st)});
    b->n_chunks = (int)chunks.size();
    adlbr_status e = ADLBR_OK;
#define BCHECK(x)                                   \
    do {                                            \
        cudaError_t c_ = (x);                       \
        if (c_ != cudaSuccess) {                    \
            free_batch(b);                          \
            return cuda_fail(c_, #x);                \
        }                                           \
    } while (0)
    BCHECK(cudaMalloc(&b->items, n_items * sizeof(adlbr_batch_item)));
    BCHECK(cudaMalloc(&b->chunks, chunks.size() * sizeof(adlbr_batch_chunk)));
    BCHECK(cudaMemcpyAsync(b->items, b->host_items.data(), n_items * sizeof(adlbr_batch_item),
                           cudaMemcpyHostToDevice, stream));
    BCHECK(cudaMemcpyAsync(b->chunks, chunks.data(), chunks.size() * sizeof(adlbr_batch_chunk),
                           cudaMemcpyHostToDevice, stream));
    BCHECK(cudaStreamSynchronize(stream));
    // autotune: time each accumulate kernel for every candidate shape (the
    // 2D kernel with the first 3D shape, then the 3D kernel with the best 2D
    // shape); the tuned time is the sum of the two best
    int best2 = 0, best3 = 0;
    if (autotune) {
        cudaEvent_t e0, e1;
        BCHECK(cudaEventCreate(&e0));
        BCHECK(cudaEventCreate(&e1));
        auto time_acc = [&](int c2, int c3, bool three, float *out_ms) -> adlbr_status {
            if (adlbr_status ee = use_shapes(b, c2, c3, stream)) return ee;
            float ms_min = 1e30f;
            for (int r = 0; r < 4; ++r) {   // the first round warms up
                cudaMemsetAsync(b->acc, 0, b->acc_bytes, stream);
                cudaEventRecord(e0, stream);
                adlbr_status ee = three ? acc3(b, c3, false, stream) : acc2(b, c2, false, stream);
                if (ee) return ee;
                cudaEventRecord(e1, stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) ms_min = std::min(ms_min, ms);
            }
            *out_ms = ms_min;
            return ADLBR_OK;
        };
        float best_ms2 = 1e30f, best_ms3 = 1e30f;
        for (int c = 0; c < kNum2 && e == ADLBR_OK; ++c) {
            float ms = 0.f;
            if ((e = time_acc(c, 0, false, &ms))) break;
            if (ms < best_ms2) best_ms2 = ms, best2 = c;
        }
        for (int c = 0; c < kNum3 && e == ADLBR_OK; ++c) {
            float ms = 0.f;
            if ((e = time_acc(best2, c, true, &ms))) break;
            if (ms < best_ms3) best_ms3 = ms, best3 = c;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->tuned_ms = best_ms2 + best_ms3;
        if (e != ADLBR_OK) {
            free_batch(b);
            return e;
        }
    }
    b->cand2 = best2;
    b->cand3 = best3;
    if ((e = use_shapes(b, best2, best3, stream))) {
        free_batch(b);
        return e;
    }
    // record one step as a graph
    b->graph = new ChunkGraph();
    e = b->graph->capture([&](cudaStream_t cs) { return enqueue_step(b, cs); });
    if (e != ADLBR_OK) {
        free_batch(b);
        return e;
    }
#undef BCHECK
    *out = b;
    return ADLBR_OK;
}

adlbr_status adlbr_batch_step(adlbr_batch *b, int nsteps, cudaStream_t stream) {
    ADLBR_NVTX("adlbr_batch_step");
    if (!b) return fail(ADLBR_E_ARG, "null batch");
    if (nsteps < 0) return fail(ADLBR_E_ARG, "bad nsteps");
    int dev = -1;
    ADLBR_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return fail(ADLBR_E_ARG, "current device %d is not the batch's device %d", dev, b->device);
    for (int k = 0; k < nsteps; ++k) ADLBR_CUDA(cudaGraphLaunch(b->graph->exec, stream));
    return ADLBR_OK;
}

adlbr_status adlbr_batch_config(const adlbr_batch *b, int *shape_out, double *tuned_ms, int64_t *points,
                                int *n_tiles) {
    if (!b) return fail(ADLBR_E_ARG, "null batch");
    if (shape_out) {
        const Shape2 &s2 = kShapes2[b->cand2];
        const Shape3 &s3 = kShapes3[b->cand3];
        shape_out[0] = s2.tw, shape_out[1] = s2.th;
        shape_out[2] = s3.bx, shape_out[3] = s3.by, shape_out[4] = s3.bz;
    }
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    if (points) *points = b->points;
    if (n_tiles) *n_tiles = b->n_tiles;
    return ADLBR_OK;
}

adlbr_status adlbr_batch_destroy(adlbr_batch *b) {
    free_batch(b);
    return ADLBR_OK;
}

}  // extern "C"

// Batched sweeps: many 2D grids of any size, each with its own stencil (star/box/diamond,
// radius 1-2), storage type and boundary, advanced `steps` time steps by ONE persistent
// cooperative kernel (the sweep of ForgeStencil Sec. 2.1, applied to every grid of a batch).
//
// Work: every grid is cut into output tiles; tile t of step group g reads the grid's previous
// buffer and writes the next one (in -> out/scratch ping-pong, arranged so the last group
// writes `out`).  A group fuses `fuse` steps in shared memory (the tile engine of the fused 2D
// kernel).  Between groups all blocks meet at a device-wide barrier.  Its wait is bounded by
// %globaltimer: a block that waits longer than the limit latches STENCIL_ERR_TIMEOUT, raises
// the abort flag and returns, and every other block leaves at its next wait.  Nothing traps.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/stencil.h"
#include "fused2d.cuh"
#include "internal.h"
#include "plan_internal.h"

namespace gst {

struct BatchGrid {
    const void *in;
    void *out;
    void *scratch;    // one grid-sized buffer (null when a single group suffices)
    int ny, nx;
    int code;         // kernel selector: dtype * 8 + shape * 2 + (radius - 1)
    int periodic;
    int coef_off;     // first coefficient in the batch's coefficient array
    int tiles_x;
};

struct BatchTile {
    int grid;
    int y0, x0;
};

struct BatchControl {
    unsigned int arrived;        // barrier arrivals (reset to 0 before every launch)
    int abort;                   // set by a block whose wait expired
    int err;                     // latched status
    int phantom;                 // extra arrivals a barrier waits for (fault injection only)
    unsigned long long limit_ns; // bounded-wait limit
};

struct BatchParams {
    const BatchGrid *grids;
    const BatchTile *tiles;
    const float *coefs;
    BatchControl *ctl;
    int ntiles;
    int groups;      // step groups
    int fuse;        // steps per group (the last group may be shorter)
    int steps;
    int tile_y, tile_x;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Device-wide barrier number k (1-based) with a bounded wait.  Returns false if the batch is
// aborting (this block must return).
__device__ bool grid_barrier(BatchControl *ctl, unsigned int k) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&ctl->arrived, 1u);
        const unsigned int target = k * gridDim.x + (unsigned int)ctl->phantom;
        const unsigned long long t0 = global_ns();
        int ok = 1;
        while (true) {
            const unsigned int a = *((volatile unsigned int *)&ctl->arrived);
            if (a >= target) break;
            if (*((volatile int *)&ctl->abort)) {
                ok = 0;
                break;
            }
            if (global_ns() - t0 > ctl->limit_ns) {
                atomicCAS(&ctl->err, 0, kErrTimeout);
                atomicExch(&ctl->abort, 1);
                ok = 0;
                break;
            }
            __nanosleep(256);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T, int SHAPE, int R>
__device__ void batch_tile(const BatchParams &P, const BatchGrid &G, const BatchTile &tl,
                           int group, float *buf) {
    constexpr int NPTS = OffsetTable<2, SHAPE, R>::count;
    float creg[NPTS];
#pragma unroll
    for (int i = 0; i < NPTS; ++i) creg[i] = __ldg(P.coefs + G.coef_off + i);
    const int g_total = P.groups;
    const int k = min(P.fuse, P.steps - group * P.fuse);
    const void *src = group == 0 ? G.in : (((g_total - group) % 2 == 0) ? G.out : G.scratch);
    void *dst = ((g_total - 1 - group) % 2 == 0) ? G.out : G.scratch;
    Fused2DTile t;
    t.ny = G.ny;
    t.nx = G.nx;
    t.periodic = G.periodic;
    t.y0 = tl.y0;
    t.x0 = tl.x0;
    t.th = min(P.tile_y, G.ny - tl.y0);
    t.tw = min(P.tile_x, G.nx - tl.x0);
    t.steps = k;
    fused2d_tile<T, SHAPE, R, true, 4>(static_cast<const T *>(src), static_cast<T *>(dst), t, buf,
                                       [&](int idx) { return creg[idx]; });
}

template <typename T>
__device__ __forceinline__ void batch_tile_dt(const BatchParams &P, const BatchGrid &G,
                                              const BatchTile &tl, int group, float *buf) {
    switch (G.code & 7) {
    case 0: batch_tile<T, kStar, 1>(P, G, tl, group, buf); break;
    case 1: batch_tile<T, kStar, 2>(P, G, tl, group, buf); break;
    case 2: batch_tile<T, kBox, 1>(P, G, tl, group, buf); break;
    case 3: batch_tile<T, kBox, 2>(P, G, tl, group, buf); break;
    case 4: batch_tile<T, kDiamond, 1>(P, G, tl, group, buf); break;
    case 5: batch_tile<T, kDiamond, 2>(P, G, tl, group, buf); break;
    default: break;
    }
}

__global__ void __launch_bounds__(128) batch_persistent_kernel(const BatchParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>(smem_raw);
    for (int g = 0; g < P.groups; ++g) {
        if (g > 0 && !grid_barrier(P.ctl, (unsigned int)g)) return;
        for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
            const BatchTile tl = P.tiles[t];
            const BatchGrid G = P.grids[tl.grid];
            switch (G.code >> 3) {
            case kF32: batch_tile_dt<float>(P, G, tl, g, buf); break;
            case kF16: batch_tile_dt<__half>(P, G, tl, g, buf); break;
            case kBF16: batch_tile_dt<__nv_bfloat16>(P, G, tl, g, buf); break;
            default: break;
            }
        }
    }
}

}  // namespace gst

using namespace gst;

struct stencil_batch_s {
    int n = 0, steps = 0, fuse = 1, groups = 0;
    int tile_y = 32, tile_x = 120;  // a halo row (<= 124 cells) is one pass of 32 lanes x 4
    int nblocks = 0, threads = 128;
    size_t smem = 0;
    BatchGrid *d_grids = nullptr;
    BatchTile *d_tiles = nullptr;
    float *d_coefs = nullptr;
    BatchControl *d_ctl = nullptr;
    std::vector<void *> scratch;
    int ntiles = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    BatchParams params{};
};

static void batch_free(stencil_batch_s *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void *p : b->scratch) cudaFree(p);
    cudaFree(b->d_grids);
    cudaFree(b->d_tiles);
    cudaFree(b->d_coefs);
    cudaFree(b->d_ctl);
    delete b;
}

// Enqueue the counter reset and the persistent kernel on `s` (captured or not).
static cudaError_t batch_enqueue(stencil_batch_s *b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->d_ctl, 0, 2 * sizeof(unsigned int), s);  // arrived, abort
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(b->nblocks);
    cfg.blockDim = dim3(b->threads);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_persistent_kernel, b->params);
}

extern "C" {

int stencil_batch_plan(stencil_batch *out, const stencil_batch_item *items, int n, int steps) {
    // the dispatch map's shape for the batch's storage type, when every grid has the same one
    BatchShape bs;
    if (items && n > 0 && items[0].plan) {
        const int dt = items[0].plan->dtype;
        bool same = true;
        for (int i = 1; i < n; ++i)
            if (!items[i].plan || items[i].plan->dtype != dt) same = false;
        if (same) bs = batch_shape_for(dt);
    }
    return stencil_batch_plan_tiles(out, items, n, steps, bs.tile_y, bs.tile_x, bs.fuse);
}

int stencil_batch_plan_tiles(stencil_batch *out, const stencil_batch_item *items, int n,
                             int steps, int tile_y, int tile_x, int fuse) {
    if (!out) return STENCIL_ERR_BADARG;
    *out = nullptr;
    if (!items || n < 1 || steps < 1) return STENCIL_ERR_BADARG;
    if (tile_y < 0 || tile_x < 0 || fuse < 0 || tile_y > 1024 || tile_x > 1024 || fuse > 64)
        return STENCIL_ERR_BADARG;
    stencil_batch_s *b = new (std::nothrow) stencil_batch_s();
    if (!b) return STENCIL_ERR_OOM;
    b->n = n;
    b->steps = steps;
    // defaults: one step per group (a barrier between steps), tiles of 32 x 120 cells
    if (tile_y > 0) b->tile_y = tile_y;
    if (tile_x > 0) b->tile_x = tile_x;
    b->fuse = fuse > 0 ? std::min(fuse, steps) : 1;
    b->groups = (steps + b->fuse - 1) / b->fuse;
    int max_r = 1;
    std::vector<BatchGrid> grids(n);
    std::vector<BatchTile> tiles;
    std::vector<float> coefs;
    for (int i = 0; i < n; ++i) {
        const stencil_plan_s *p = items[i].plan;
        if (!p || !items[i].in || !items[i].out) {
            delete b;
            return STENCIL_ERR_BADARG;
        }
        if (p->ndim != 2 || p->kind != STENCIL_CONST) {
            delete b;
            return STENCIL_ERR_UNSUPPORTED;
        }
        if (p->radius > 2) {
            delete b;
            return STENCIL_ERR_UNSUPPORTED;
        }
        const size_t bytes = (size_t)p->dims[1] * p->dims[2] * dtype_size(p->dtype);
        if (overlaps(items[i].in, items[i].out, bytes)) {
            delete b;
            return STENCIL_ERR_BADARG;
        }
        max_r = std::max(max_r, p->radius);
        BatchGrid &G = grids[i];
        G.in = items[i].in;
        G.out = items[i].out;
        G.scratch = nullptr;
        G.ny = (int)p->dims[1];
        G.nx = (int)p->dims[2];
        G.code = p->dtype * 8 + p->shape * 2 + (p->radius - 1);
        G.periodic = p->boundary == STENCIL_PERIODIC;
        G.coef_off = (int)coefs.size();
        G.tiles_x = (G.nx + b->tile_x - 1) / b->tile_x;
        coefs.insert(coefs.end(), p->cf.begin(), p->cf.end());
        if (b->groups > 1) {
            void *sp = nullptr;
            if (cudaMalloc(&sp, bytes) != cudaSuccess) {
                cudaGetLastError();
                batch_free(b);
                return STENCIL_ERR_OOM;
            }
            b->scratch.push_back(sp);
            G.scratch = sp;
        }
        const int tiles_y = (G.ny + b->tile_y - 1) / b->tile_y;
        for (int ty = 0; ty < tiles_y; ++ty)
            for (int tx = 0; tx < G.tiles_x; ++tx) tiles.push_back({i, ty * b->tile_y, tx * b->tile_x});
    }
    // large grids' tiles first so that the ragged end of each step is made of small work
    b->ntiles = (int)tiles.size();
    b->smem = fused2d_smem_bytes(b->tile_x, b->tile_y, max_r, b->fuse);
    if (b->smem > 227 * 1024) {  // the tile with its halo does not fit in shared memory
        batch_free(b);
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (cudaFuncSetAttribute(batch_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)b->smem) != cudaSuccess) {
        batch_free(b);
        return STENCIL_ERR_CUDA;
    }
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel, b->threads,
                                                      b->smem) != cudaSuccess ||
        per_sm < 1) {
        batch_free(b);
        return STENCIL_ERR_UNSUPPORTED;
    }
    b->nblocks = std::max(1, std::min(per_sm * sms, b->ntiles));
    if (cudaMalloc(&b->d_grids, sizeof(BatchGrid) * n) != cudaSuccess ||
        cudaMalloc(&b->d_tiles, sizeof(BatchTile) * tiles.size()) != cudaSuccess ||
        cudaMalloc(&b->d_coefs, sizeof(float) * coefs.size()) != cudaSuccess ||
        cudaMalloc(&b->d_ctl, sizeof(BatchControl)) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return STENCIL_ERR_OOM;
    }
    BatchControl ctl;
    std::memset(&ctl, 0, sizeof(ctl));
    ctl.limit_ns = 2000000000ull;  // 2 s
    if (cudaMemcpy(b->d_grids, grids.data(), sizeof(BatchGrid) * n, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(),
                   cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_coefs, coefs.data(), sizeof(float) * coefs.size(),
                   cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice)) {
        batch_free(b);
        return STENCIL_ERR_CUDA;
    }
    b->params.grids = b->d_grids;
    b->params.tiles = b->d_tiles;
    b->params.coefs = b->d_coefs;
    b->params.ctl = b->d_ctl;
    b->params.ntiles = b->ntiles;
    b->params.groups = b->groups;
    b->params.fuse = b->fuse;
    b->params.steps = b->steps;
    b->params.tile_y = b->tile_y;
    b->params.tile_x = b->tile_x;

    // capture the reset + persistent launch into a graph (falls back to direct launches when
    // this runtime cannot capture a cooperative kernel)
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cudaError_t e = batch_enqueue(b, cs);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (e == cudaSuccess && e2 == cudaSuccess && g &&
                cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
                b->graph = g;
            } else {
                if (g) cudaGraphDestroy(g);
                b->exec = nullptr;
            }
        }
        cudaGetLastError();
        cudaStreamDestroy(cs);
    }
    *out = b;
    return STENCIL_OK;
}

int stencil_batch_launch(stencil_batch b, void *stream) {
    if (!b) return STENCIL_ERR_BADARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, s) : batch_enqueue(b, s);
    count_launch();
    return e == cudaSuccess ? STENCIL_OK : STENCIL_ERR_CUDA;
}

int stencil_batch_status(stencil_batch b, void *stream) {
    if (!b) return STENCIL_ERR_BADARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return STENCIL_ERR_CUDA;
    BatchControl ctl;
    if (cudaMemcpy(&ctl, b->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
        return STENCIL_ERR_CUDA;
    if (ctl.err) {
        int zero = 0;
        cudaMemcpy(&b->d_ctl->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return ctl.err;
    }
    return STENCIL_OK;
}

int stencil_batch_set_wait_limit(stencil_batch b, double seconds, int phantom_arrivals) {
    if (!b || !(seconds > 0.0) || seconds > 3600.0 || phantom_arrivals < 0)
        return STENCIL_ERR_BADARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return STENCIL_ERR_CUDA;
    BatchControl ctl;
    if (cudaMemcpy(&ctl, b->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
        return STENCIL_ERR_CUDA;
    ctl.limit_ns = (unsigned long long)(seconds * 1e9);
    ctl.phantom = phantom_arrivals;
    if (cudaMemcpy(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice) != cudaSuccess)
        return STENCIL_ERR_CUDA;
    return STENCIL_OK;
}

int stencil_batch_info(stencil_batch b, int *ntiles, int *nblocks, int *graph_captured) {
    if (!b) return STENCIL_ERR_BADARG;
    if (ntiles) *ntiles = b->ntiles;
    if (nblocks) *nblocks = b->nblocks;
    if (graph_captured) *graph_captured = b->exec != nullptr;
    return STENCIL_OK;
}

int stencil_batch_destroy(stencil_batch b) {
    batch_free(b);
    return STENCIL_OK;
}

}  // extern "C"

// Host side of the C ABI declared in include/stencil.h: plan validation, the dispatch map,
// multi-step scheduling (ping-pong through a plan-owned scratch grid) and error reporting.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/stencil.h"
#include "internal.h"
#include "plan_internal.h"
#include "wavefront.h"

namespace gst {

static std::atomic<uint64_t> g_launches{0};
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------------------
// Offset sets (canonical order: lexicographic (dz, dy, dx), each -r..r).
// ---------------------------------------------------------------------------------------
static bool host_in_shape(int ndim, int shape, int r, int dz, int dy, int dx) {
    if (ndim == 2 && dz != 0) return false;
    int az = std::abs(dz), ay = std::abs(dy), ax = std::abs(dx);
    if (az > r || ay > r || ax > r) return false;
    if (shape == STENCIL_STAR) return ((dz != 0) + (dy != 0) + (dx != 0)) <= 1;
    if (shape == STENCIL_BOX) return true;
    return az + ay + ax <= r;
}

std::vector<int32_t> make_offsets(int ndim, int shape, int r) {
    std::vector<int32_t> out;
    const int zr = ndim == 3 ? r : 0;
    for (int dz = -zr; dz <= zr; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (host_in_shape(ndim, shape, r, dz, dy, dx)) {
                    if (ndim == 3) out.push_back(dz);
                    out.push_back(dy);
                    out.push_back(dx);
                }
    return out;
}

// ---------------------------------------------------------------------------------------
// Dispatch map
// ---------------------------------------------------------------------------------------
struct MapEntry {
    int key[8];  // ndim shape radius dtype boundary kind size_class geometry (-1: any)
    stencil_variant v;
};
static std::mutex g_map_mu;
static std::vector<MapEntry> g_map;
static BatchShape g_batch_map[3];  // per storage type; zeros: no entry

BatchShape batch_shape_for(int dtype) {
    std::lock_guard<std::mutex> lk(g_map_mu);
    return (dtype >= 0 && dtype < 3) ? g_batch_map[dtype] : BatchShape{};
}

int size_class_of(int64_t cells) {
    if (cells < (int64_t)1 << 16) return 0;
    if (cells < (int64_t)1 << 20) return 1;
    if (cells < (int64_t)1 << 24) return 2;
    return 3;
}

// Grid geometry class: 1 for a 3D slab thin in z (nz at most 1/8 of ny and of nx: few planes
// per tile column, so the z chunks and halo planes weigh differently), 0 otherwise.
int geometry_class_of(int ndim, const int64_t *d) {
    if (ndim == 3 && d[0] * 8 <= d[1] && d[0] * 8 <= d[2]) return 1;
    return 0;
}

// Built-in defaults (used when the map has no entry for a key).
static stencil_variant default_variant(const stencil_plan_s &p) {
    stencil_variant v;
    std::memset(&v, 0, sizeof(v));
    const int es = p.dtype == STENCIL_F32 ? 4 : 2;
    const int vx = 16 / es;
    v.family = STENCIL_FAMILY_STREAM;
    v.block_x = 128 / vx;  // 128-cell tiles in x
    v.block_y = 128 / v.block_x;  // 128 consumer threads
    v.vec_y = 1;
    // 3D: 64-plane chunks, so that the CTAs of neighbouring tiles walk the same planes at the
    // same time and share their halo rows in L2 (measured on GB300, 512^3 f32: an equal share
    // per resident CTA, whose pieces start at unrelated planes, took 1.8x as long)
    v.z_chunk = p.ndim == 3 ? 64 : 0;
    v.fuse = 1;
    if (p.kind != STENCIL_CONST) {
        // variable coefficients: one output row per thread, 64-plane z chunks
        v.block_y = (p.kind == STENCIL_DIVKGRAD ? 192 : 128) / v.block_x;
        v.z_chunk = 64;
        return v;
    }
    if (p.ndim == 3) {
        // two rows per thread while the partial-sum queue stays small
        if (stream_vy_compiled(3, p.shape, p.radius, 2) && p.radius <= 2) {
            v.vec_y = 2;
            v.block_y /= 2;
        }
    } else {
        v.vec_y = 2;
        v.block_y = 4;
        const int64_t cells = p.dims[1] * p.dims[2];
        if (cells <= ((int64_t)1 << 20)) {
            v.family = STENCIL_FAMILY_FUSED2D;
            v.fuse = 8;
            v.tile_x = 32;
            v.tile_y = 32;
            v.block_x = 256;
            v.block_y = 1;
            v.vec_y = 1;
        }
    }
    return v;
}

static bool lookup_map(const stencil_plan_s &p, stencil_variant *out) {
    std::lock_guard<std::mutex> lk(g_map_mu);
    const int key[8] = {p.ndim, p.shape, p.radius, p.dtype, p.boundary, p.kind,
                        size_class_of(p.dims[0] * p.dims[1] * p.dims[2]),
                        geometry_class_of(p.ndim, p.dims)};
    for (const MapEntry &e : g_map) {
        bool ok = true;
        for (int i = 0; i < 8; ++i)
            if (e.key[i] != key[i] && e.key[i] != -1) ok = false;
        if (ok) {
            *out = e.v;
            return true;
        }
    }
    return false;
}

int validate_variant(const stencil_plan_s &p, const stencil_variant &v) {
    if (p.kind != STENCIL_CONST) {
        // variable-coefficient kernels: 128-cell tiles, block_y rows of threads with one output
        // row each (div(k grad u): one or two), at most 224 threads, z chunks of z_chunk planes
        // (0: whole columns for the general sweeps, an equal share per resident CTA for
        // div(k grad u); -1, div(k grad u) only: aligned chunks per tile column)
        const bool vy_ok = v.vec_y == 1 || (v.vec_y == 2 && p.kind == STENCIL_DIVKGRAD);
        if (v.family != STENCIL_FAMILY_STREAM || !vy_ok || v.fuse != 1 ||
            v.block_x != (int)(128 / (16 / dtype_size(p.dtype))) || v.block_y < 1 ||
            v.block_x * v.block_y > 224 || (v.block_x * v.block_y) % 32 != 0 ||
            v.z_chunk < (p.kind == STENCIL_DIVKGRAD ? -1 : 0))
            return STENCIL_ERR_BADARG;
        return STENCIL_OK;
    }
    if (v.family == STENCIL_FAMILY_STREAM) {
        // tiles are 128 cells wide: one 16-byte vector of cells per thread along x
        if (v.block_x != (int)(128 / (16 / dtype_size(p.dtype))) || v.block_y < 1 ||
            v.block_x * v.block_y > stream_max_threads(p.ndim, p.shape, p.radius, v.vec_y, p.dtype) ||
            (v.block_x * v.block_y) % 32 != 0)
            return STENCIL_ERR_BADARG;
        if (!stream_vy_compiled(p.ndim, p.shape, p.radius, v.vec_y))
            return STENCIL_ERR_UNSUPPORTED;
        if (v.z_chunk < -1 || v.fuse != 1) return STENCIL_ERR_BADARG;
        if (v.stages != 0 && (v.stages < 2 || v.stages > 16)) return STENCIL_ERR_BADARG;
        return STENCIL_OK;
    }
    if (v.family == STENCIL_FAMILY_FUSED3D) {
        // two fused 3D steps: 128-cell tiles, two output rows per thread, at least 2R rows of
        // threads (the grown tile of the first step fits in three rows per thread)
        if (!fused3d_compiled(p.ndim, p.shape, p.radius)) return STENCIL_ERR_UNSUPPORTED;
        if (v.block_x != (int)(128 / (16 / dtype_size(p.dtype))) ||
            v.vec_y != (dtype_size(p.dtype) == 4 ? 2 : 1) ||
            v.block_y < 2 * p.radius || v.block_x * v.block_y > 224 ||
            (v.block_x * v.block_y) % 32 != 0 || v.fuse != 2 || v.z_chunk < 0)
            return STENCIL_ERR_BADARG;
        if (v.stages != 0 && (v.stages < 2 || v.stages > 16)) return STENCIL_ERR_BADARG;
        return STENCIL_OK;
    }
    if (v.family == STENCIL_FAMILY_TENSOR) {
        // the radius-2 box on the tensor cores: 16-bit storage, zero Dirichlet, rows a
        // multiple of 8 cells; tile_x = 16, 32 or 64 outputs per CTA, 5..12 plane slots
        if (!toeplitz_compiled(p.ndim, p.shape, p.radius, p.dtype) ||
            p.boundary != STENCIL_DIRICHLET0 || p.dims[2] % 8 != 0)
            return STENCIL_ERR_UNSUPPORTED;
        // vec_y: warps issuing the MMAs, each for every vec_y-th output plane (0 or 1, 2, or
        // 4 with 64-output tiles)
        const int mw = v.vec_y <= 1 ? 1 : v.vec_y, nb = v.tile_x / 16;
        if ((v.tile_x != 16 && v.tile_x != 32 && v.tile_x != 64) || v.fuse != 1 ||
            v.z_chunk < 0 || v.block_y < 0 || v.block_y > 1 ||
            (v.stages != 0 && (v.stages < 5 || v.stages > 12)) || v.vec_y < 0 ||
            (mw != 1 && mw != 2 && mw != 4) || (mw == 4 && nb != 4))
            return STENCIL_ERR_BADARG;
        return STENCIL_OK;
    }
    if (v.family == STENCIL_FAMILY_FUSED2D) {
        if (p.ndim != 2) return STENCIL_ERR_UNSUPPORTED;
        if (v.fuse < 1 || v.tile_x < 1 || v.tile_y < 1) return STENCIL_ERR_BADARG;
        if (v.block_x < 32 || v.block_x > 256 || v.block_x % 32 || v.block_y != 1)
            return STENCIL_ERR_BADARG;
        if (fused2d_smem_bytes(v.tile_x, v.tile_y, p.radius, v.fuse) > 227 * 1024)
            return STENCIL_ERR_UNSUPPORTED;
        return STENCIL_OK;
    }
    return STENCIL_ERR_BADARG;
}

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? STENCIL_OK : STENCIL_ERR_CUDA; }

int map_launch_rc(int rc) {
    if (rc == 0) return STENCIL_OK;
    if (rc == -1) return STENCIL_ERR_BADARG;
    if (rc == -2) return STENCIL_ERR_UNSUPPORTED;
    return STENCIL_ERR_CUDA;
}

size_t dtype_size(int dtype) { return dtype == STENCIL_F32 ? 4 : 2; }

int ensure_scratch(stencil_plan_s &p) {
    const size_t bytes = (size_t)p.dims[0] * p.dims[1] * p.dims[2] * dtype_size(p.dtype);
    if (p.scratch && p.scratch_bytes >= bytes) return STENCIL_OK;
    if (p.scratch) cudaFree(p.scratch);
    p.scratch = nullptr;
    p.scratch_bytes = 0;
    if (cudaMalloc(&p.scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return STENCIL_ERR_OOM;
    }
    p.scratch_bytes = bytes;
    return STENCIL_OK;
}

// One launch of `k` steps from src to dst with the plan's variant and coefficients (3D
// streaming plans: output planes [z_lo, z_hi) only, z_hi < 0 meaning all).
static int launch_group(stencil_plan_s &p, const float *cf, const void *src, void *dst, int k,
                        cudaStream_t s, int64_t z_lo = 0, int64_t z_hi = -1) {
    const stencil_variant &v = p.variant;
    if (v.family == STENCIL_FAMILY_FUSED2D) {
        Fused2DLaunch L;
        L.ny = p.dims[1];
        L.nx = p.dims[2];
        L.shape = p.shape;
        L.radius = p.radius;
        L.dtype = p.dtype;
        L.periodic = p.boundary == STENCIL_PERIODIC;
        L.coeffs = cf;
        L.in = src;
        L.out = dst;
        L.steps = k;
        L.tile_x = v.tile_x;
        L.tile_y = v.tile_y;
        L.block_threads = v.block_x;
        L.stream = s;
        return map_launch_rc(launch_fused2d(L));
    }
    StreamLaunch L;
    L.ndim = p.ndim;
    L.nz = p.dims[0];
    L.ny = p.dims[1];
    L.nx = p.dims[2];
    L.shape = p.shape;
    L.radius = p.radius;
    L.dtype = p.dtype;
    L.periodic = p.boundary == STENCIL_PERIODIC;
    L.coeffs = cf;
    L.in = src;
    L.out = dst;
    L.block_x = v.block_x;
    L.block_y = v.block_y;
    L.vec_y = v.vec_y;
    // a z sub-range (a slab of the host-buffer pipeline) holds too few planes to fill the GPU
    // with the tuned chunks: every resident CTA takes an equal share of it instead
    const bool slab = z_hi >= 0 && z_hi - z_lo < p.dims[0];
    L.z_chunk = slab ? 0 : v.z_chunk;
    L.stages = v.stages;
    L.z_lo = z_lo;
    L.z_hi = z_hi;
    L.err = status_word(p.status_slot);
    L.wait = p.wait;
    L.stream = s;
    p.launched = true;
    // a fused 3D plan runs pairs of steps on the fused kernel, an odd last step on the
    // streaming kernel with the same tile
    if (v.family == STENCIL_FAMILY_FUSED3D && k == 2 && !slab)
        return map_launch_rc(launch_fused3d(L));
    if (v.family == STENCIL_FAMILY_TENSOR)
        return map_launch_rc(launch_toeplitz(L, v.tile_x / 16, v.vec_y <= 1 ? 1 : v.vec_y));
    return map_launch_rc(launch_stream(L));
}

// Steps per launch of the plan's kernel family.
static int steps_per_launch(const stencil_plan_s &p) {
    if (p.variant.family == STENCIL_FAMILY_FUSED2D) return std::max(1, p.variant.fuse);
    if (p.variant.family == STENCIL_FAMILY_FUSED3D) return 2;
    return 1;
}

// `steps` sweeps in groups of variant.fuse; the groups alternate between `out` and the scratch
// grid so that the last one writes `out` and `in` is never written.
int run_steps(stencil_plan_s &p, const float *cf, const void *in, void *out, int steps,
              cudaStream_t s) {
    const int fuse = steps_per_launch(p);
    const int groups = (steps + fuse - 1) / fuse;
    if (groups > 1) {
        int rc = ensure_scratch(p);
        if (rc) return rc;
    }
    const void *src = in;
    int done = 0;
    for (int g = 0; g < groups; ++g) {
        const int k = std::min(fuse, steps - done);
        void *dst = ((groups - 1 - g) % 2 == 0) ? out : p.scratch;
        int rc = launch_group(p, cf, src, dst, k, s);
        if (rc) return rc;
        src = dst;
        done += k;
    }
    return STENCIL_OK;
}

bool overlaps(const void *a, const void *b, size_t n) {
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + n && y < x + n;
}

int check_apply_args(const stencil_plan_s *p, const void *in, const void *out, int steps) {
    if (!p || !in || !out || steps < 1) return STENCIL_ERR_BADARG;
    const size_t bytes = (size_t)p->dims[0] * p->dims[1] * p->dims[2] * dtype_size(p->dtype);
    if (overlaps(in, out, bytes)) return STENCIL_ERR_BADARG;
    return STENCIL_OK;
}

}  // namespace gst

using namespace gst;

// =========================================================================================
// C ABI
// =========================================================================================
// stencil_apply_host for 3D streaming plans, pipelined over z slabs: the input slabs are
// copied in on one stream; on the caller's stream a slab of output planes is swept as soon as
// the input planes it reads have landed; the finished output slabs are copied out on a third
// stream (several sweeps: the wavefront of host_wavefront above).  Both copy
// directions overlap the sweeps and each other.  Slab k reads input planes up to R beyond
// its end, so it waits for input slab k + 1; on a periodic grid slab 0 also reads the last
// planes, so it is swept last.
// Several sweeps of stencil_apply_host: the wavefront over z of wavefront.h, the input copied
// in on s_in as in the single sweep (slab k recorded by ev_in[k]), the sweeps in order on the
// caller's stream, alternating between the scratch grid and stage_out (the last one writes
// stage_out), the finished planes of the last sweep out on s_out.
static int host_wavefront(stencil_plan_s &h, char *hout, int steps, const int64_t *zb,
                          int nslab, cudaStream_t s) {
    constexpr int kMax = stencil_plan_s::kMaxSlabs;
    const size_t plane = (size_t)h.dims[1] * h.dims[2] * dtype_size(h.dtype);
    const char *dout = static_cast<const char *>(h.stage_out);
    auto check = [](cudaError_t e) { return e == cudaSuccess; };
    auto dst_of = [&](int t) -> void * { return ((steps - t) % 2 == 0) ? h.stage_out : h.scratch; };
    auto src_of = [&](int t) -> const void * { return t == 1 ? h.stage_in : dst_of(t - 1); };
    int nev = 0;
    const int rc = wavefront_schedule(
        h.dims[0], h.radius, h.boundary == STENCIL_PERIODIC, steps, zb, nslab,
        [&](int kind, int slab, int t, int64_t a, int64_t b) -> int {
            if (kind == kWaveWaitInput)
                return check(cudaStreamWaitEvent(s, h.ev_in[slab], 0)) ? STENCIL_OK
                                                                       : STENCIL_ERR_CUDA;
            if (kind == kWaveSweep)
                return launch_group(h, h.cf.data(), src_of(t), dst_of(t), 1, s, a, b);
            // the last sweep's planes [a, b) out to the host once the launches so far are done
            cudaEvent_t e = h.ev_out[nev++ % kMax];
            if (!check(cudaEventRecord(e, s)) || !check(cudaStreamWaitEvent(h.s_out, e, 0)) ||
                !check(cudaMemcpyAsync(hout + (size_t)a * plane, dout + (size_t)a * plane,
                                       (size_t)(b - a) * plane, cudaMemcpyDeviceToHost, h.s_out)))
                return STENCIL_ERR_CUDA;
            return STENCIL_OK;
        });
    if (rc) return rc;
    if (!check(cudaEventRecord(h.ev_done, h.s_out)) || !check(cudaStreamWaitEvent(s, h.ev_done, 0)))
        return STENCIL_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(s));
}

static int apply_host_pipelined(stencil_plan_s &h, const void *in_host, void *out_host,
                                int steps, cudaStream_t s) {
    constexpr int kMax = stencil_plan_s::kMaxSlabs;
    const int64_t nz = h.dims[0];
    const size_t plane = (size_t)h.dims[1] * h.dims[2] * dtype_size(h.dtype);
    const int R = h.radius;
    const bool periodic = h.boundary == STENCIL_PERIODIC;
    const int nslab = (int)std::min<int64_t>(kMax, nz / std::max(16, 2 * R));
    int64_t zb[kMax + 1];
    for (int k = 0; k <= nslab; ++k) zb[k] = nz * k / nslab;
    if (!h.s_in) {
        bool ok = cudaStreamCreateWithFlags(&h.s_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h.s_out, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&h.ev_start, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&h.ev_done, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; k < kMax && ok; ++k)
            ok = cudaEventCreateWithFlags(&h.ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h.ev_out[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return STENCIL_ERR_CUDA;
        }
    }
    if (steps > 1) {
        int rc = ensure_scratch(h);
        if (rc) return rc;
    }
    auto check = [](cudaError_t e) { return e == cudaSuccess; };
    // the copies start after whatever the caller queued before
    if (!check(cudaEventRecord(h.ev_start, s)) || !check(cudaStreamWaitEvent(h.s_in, h.ev_start, 0)) ||
        !check(cudaStreamWaitEvent(h.s_out, h.ev_start, 0)))
        return STENCIL_ERR_CUDA;
    const char *hin = static_cast<const char *>(in_host);
    char *hout = static_cast<char *>(out_host);
    char *din = static_cast<char *>(h.stage_in), *dout = static_cast<char *>(h.stage_out);
    for (int k = 0; k < nslab; ++k) {
        const size_t off = (size_t)zb[k] * plane, len = (size_t)(zb[k + 1] - zb[k]) * plane;
        if (!check(cudaMemcpyAsync(din + off, hin + off, len, cudaMemcpyHostToDevice, h.s_in)) ||
            !check(cudaEventRecord(h.ev_in[k], h.s_in)))
            return STENCIL_ERR_CUDA;
    }
    if (steps > 1) return host_wavefront(h, hout, steps, zb, nslab, s);
    const void *src = h.stage_in;
    for (int g = 0; g < steps; ++g) {
        void *dst = ((steps - 1 - g) % 2 == 0) ? h.stage_out : h.scratch;
        const bool first = g == 0, last = g == steps - 1;
        if (!first && !last) {
            int rc = launch_group(h, h.cf.data(), src, dst, 1, s);
            if (rc) return rc;
        } else {
            for (int j = 0; j < nslab; ++j) {
                // periodic grids sweep slab 0 last (it reads the last input planes)
                const int k = periodic ? (j + 1) % nslab : j;
                if (first) {
                    const int need = (periodic && k == 0) ? nslab - 1 : std::min(k + 1, nslab - 1);
                    if (!check(cudaStreamWaitEvent(s, h.ev_in[need], 0))) return STENCIL_ERR_CUDA;
                }
                int rc = launch_group(h, h.cf.data(), src, dst, 1, s, zb[k], zb[k + 1]);
                if (rc) return rc;
                if (last) {
                    const size_t off = (size_t)zb[k] * plane;
                    const size_t len = (size_t)(zb[k + 1] - zb[k]) * plane;
                    if (!check(cudaEventRecord(h.ev_out[k], s)) ||
                        !check(cudaStreamWaitEvent(h.s_out, h.ev_out[k], 0)) ||
                        !check(cudaMemcpyAsync(hout + off, dout + off, len,
                                               cudaMemcpyDeviceToHost, h.s_out)))
                        return STENCIL_ERR_CUDA;
                }
            }
        }
        src = dst;
    }
    if (!check(cudaEventRecord(h.ev_done, h.s_out)) || !check(cudaStreamWaitEvent(s, h.ev_done, 0)))
        return STENCIL_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(s));
}

extern "C" {

int stencil_abi_version(void) { return STENCIL_ABI_VERSION; }

uint64_t stencil_launch_count(void) { return g_launches.load(); }

int stencil_size_class(int64_t cells) { return size_class_of(cells); }

int stencil_geometry_class(int ndim, const int64_t *dims) {
    if ((ndim != 2 && ndim != 3) || !dims) return STENCIL_ERR_BADARG;
    int64_t d[3] = {1, 1, 1};
    for (int i = 0; i < ndim; ++i) d[3 - ndim + i] = dims[i];
    return geometry_class_of(ndim, d);
}

const char *stencil_strerror(int code) {
    switch (code) {
    case STENCIL_OK: return "ok";
    case STENCIL_ERR_BADARG: return "invalid argument";
    case STENCIL_ERR_UNSUPPORTED: return "unsupported stencil configuration";
    case STENCIL_ERR_OOM: return "out of memory";
    case STENCIL_ERR_CUDA: return "CUDA runtime error";
    case STENCIL_ERR_TIMEOUT: return "device-side wait timed out";
    case STENCIL_ERR_BOUNDS: return "device-side index check failed";
    default: return "unknown status code";
    }
}

int stencil_plan(stencil_handle *out, int ndim, const int64_t *dims, int shape, int radius,
                 int kind, const double *coeffs, int64_t ncoeffs, const int32_t *custom_offsets,
                 int dtype, int boundary) {
    // a dispatch map named by STENCIL_DISPATCH_MAP is read once, before the first plan
    static std::once_flag env_map_once;
    std::call_once(env_map_once, [] {
        const char *path = std::getenv("STENCIL_DISPATCH_MAP");
        if (path && *path) stencil_load_dispatch_map(path);
    });
    if (!out) return STENCIL_ERR_BADARG;
    *out = nullptr;
    if ((ndim != 2 && ndim != 3) || !dims) return STENCIL_ERR_BADARG;
    if (shape < STENCIL_STAR || shape > STENCIL_CUSTOM) return STENCIL_ERR_BADARG;
    if (radius < 1 || radius > 4) return STENCIL_ERR_BADARG;
    if (dtype < STENCIL_F32 || dtype > STENCIL_BF16) return STENCIL_ERR_BADARG;
    if (boundary != STENCIL_DIRICHLET0 && boundary != STENCIL_PERIODIC) return STENCIL_ERR_BADARG;
    if (kind < STENCIL_CONST || kind > STENCIL_DIVKGRAD) return STENCIL_ERR_BADARG;
    if ((shape == STENCIL_CUSTOM) != (custom_offsets != nullptr)) return STENCIL_ERR_BADARG;
    int64_t d[3] = {1, 1, 1};
    for (int i = 0; i < ndim; ++i) {
        if (dims[i] < 1) return STENCIL_ERR_BADARG;
        d[3 - ndim + i] = dims[i];
    }
    // kernels index one plane with 32-bit integers
    if (d[1] * d[2] > ((int64_t)1 << 30) || d[0] > ((int64_t)1 << 30)) return STENCIL_ERR_UNSUPPORTED;
    // the offsets the caller sees (canonical order, or a custom set in the caller's order) and
    // the compiled offset set the kernels run (the same, or the smallest compiled set that
    // contains the custom one, its other offsets weighted 0)
    std::vector<int32_t> offs;
    int kshape = shape, kradius = radius;
    if (shape == STENCIL_CUSTOM) {
        if (kind != STENCIL_CONST) return STENCIL_ERR_UNSUPPORTED;
        if (ncoeffs < 1 || ncoeffs > 729) return STENCIL_ERR_BADARG;
        offs.assign(custom_offsets, custom_offsets + ncoeffs * ndim);
        int rinf = 0, rl1 = 0;
        bool axial = true;  // at most one nonzero component per offset
        for (int64_t i = 0; i < ncoeffs; ++i) {
            int nz = 0, l1 = 0;
            for (int a = 0; a < ndim; ++a) {
                const int c = offs[i * ndim + a];
                if (c < -radius || c > radius) return STENCIL_ERR_BADARG;
                nz += c != 0;
                l1 += std::abs(c);
                rinf = std::max(rinf, std::abs(c));
            }
            rl1 = std::max(rl1, l1);
            axial = axial && nz <= 1;
            for (int64_t j = 0; j < i; ++j)  // duplicates are an error
                if (std::equal(offs.begin() + j * ndim, offs.begin() + (j + 1) * ndim,
                               offs.begin() + i * ndim))
                    return STENCIL_ERR_BADARG;
        }
        rinf = std::max(rinf, 1);
        if (axial) {
            kshape = STENCIL_STAR;
            kradius = rinf;
        } else {
            kshape = STENCIL_BOX;
            kradius = rinf;
            if (rl1 <= 4 && make_offsets(ndim, STENCIL_DIAMOND, rl1).size() <
                                make_offsets(ndim, STENCIL_BOX, rinf).size()) {
                kshape = STENCIL_DIAMOND;
                kradius = rl1;
            }
        }
    } else {
        offs = make_offsets(ndim, shape, radius);
    }
    const int64_t npts = (int64_t)offs.size() / ndim;
    if (kind == STENCIL_CONST) {
        if (!coeffs || ncoeffs != npts) return STENCIL_ERR_BADARG;
        for (int64_t i = 0; i < npts; ++i)
            if (!std::isfinite(coeffs[i])) return STENCIL_ERR_BADARG;
    } else {
        if (coeffs || ncoeffs != 0) return STENCIL_ERR_BADARG;
        if (kind == STENCIL_DIVKGRAD && (shape != STENCIL_STAR || radius != 1))
            return STENCIL_ERR_BADARG;
    }
    stencil_plan_s *p = new (std::nothrow) stencil_plan_s();
    if (!p) return STENCIL_ERR_OOM;
    p->status_slot = status_acquire();  // host only: the word's address is looked up at launch
    if (p->status_slot < 0) {
        delete p;
        return STENCIL_ERR_OOM;
    }
    p->ndim = ndim;
    p->dims[0] = d[0];
    p->dims[1] = d[1];
    p->dims[2] = d[2];
    p->shape = kshape;
    p->radius = kradius;
    p->custom = shape == STENCIL_CUSTOM;
    p->kind = kind;
    p->dtype = dtype;
    p->boundary = boundary;
    p->npts = npts;
    p->offsets = offs;
    if (kind == STENCIL_CONST) {
        p->coeffs.assign(coeffs, coeffs + npts);
        // kernel coefficients over the compiled set, in its canonical order: the coefficient
        // of each offset, and (adjoint) the coefficient of its negation; 0 where the plan's
        // set has no such offset
        const std::vector<int32_t> koffs = make_offsets(ndim, kshape, kradius);
        const int64_t kn = (int64_t)koffs.size() / ndim;
        p->cf.assign(kn, 0.0f);
        p->cf_flip.assign(kn, 0.0f);
        for (int64_t i = 0; i < kn; ++i) {
            for (int64_t j = 0; j < npts; ++j) {
                bool same = true, neg = true;
                for (int a = 0; a < ndim; ++a) {
                    if (offs[j * ndim + a] != koffs[i * ndim + a]) same = false;
                    if (offs[j * ndim + a] != -koffs[i * ndim + a]) neg = false;
                }
                if (same) p->cf[i] = (float)coeffs[j];
                if (neg) p->cf_flip[i] = (float)coeffs[j];
            }
        }
    }
    stencil_variant v;
    if (!lookup_map(*p, &v) || validate_variant(*p, v) != STENCIL_OK) v = default_variant(*p);
    p->variant = v;
    *out = p;
    return STENCIL_OK;
}

int stencil_plan_kernel_set(stencil_handle h, int *shape, int *radius) {
    if (!h) return STENCIL_ERR_BADARG;
    if (shape) *shape = h->shape;
    if (radius) *radius = h->radius;
    return STENCIL_OK;
}

int stencil_offsets(stencil_handle h, int32_t *offsets_out, int64_t capacity, int64_t *n) {
    if (!h || !n || capacity < 0 || (capacity > 0 && !offsets_out)) return STENCIL_ERR_BADARG;
    *n = h->npts;
    const int64_t m = std::min(capacity, h->npts);
    if (m > 0) std::memcpy(offsets_out, h->offsets.data(), sizeof(int32_t) * m * h->ndim);
    return STENCIL_OK;
}

int stencil_destroy(stencil_handle h) {
    if (!h) return STENCIL_OK;
    if (h->scratch || h->stage_in || h->stage_out || h->launched || h->s_in)
        cudaDeviceSynchronize();
    status_release(h->status_slot, h->launched);
    if (h->scratch) cudaFree(h->scratch);
    if (h->stage_in) cudaFree(h->stage_in);
    if (h->stage_out) cudaFree(h->stage_out);
    for (int i = 0; i < stencil_plan_s::kMaxSlabs; ++i) {
        if (h->ev_in[i]) cudaEventDestroy(h->ev_in[i]);
        if (h->ev_out[i]) cudaEventDestroy(h->ev_out[i]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->ev_done) cudaEventDestroy(h->ev_done);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    delete h;
    return STENCIL_OK;
}

int stencil_apply(stencil_handle h, const void *in, void *out, int steps, void *stream) {
    int rc = check_apply_args(h, in, out, steps);
    if (rc) return rc;
    if (h->kind != STENCIL_CONST) return STENCIL_ERR_BADARG;
    return run_steps(*h, h->cf.data(), in, out, steps, (cudaStream_t)stream);
}

int stencil_apply_adjoint(stencil_handle h, const void *in, void *out, int steps, void *stream) {
    int rc = check_apply_args(h, in, out, steps);
    if (rc) return rc;
    if (h->kind != STENCIL_CONST) return STENCIL_ERR_BADARG;
    return run_steps(*h, h->cf_flip.data(), in, out, steps, (cudaStream_t)stream);
}

int stencil_apply_host(stencil_handle h, const void *in_host, void *out_host, int steps,
                       void *stream) {
    if (!h || !in_host || !out_host || steps < 1) return STENCIL_ERR_BADARG;
    if (h->kind != STENCIL_CONST) return STENCIL_ERR_BADARG;
    const size_t bytes = (size_t)h->dims[0] * h->dims[1] * h->dims[2] * dtype_size(h->dtype);
    if (!h->stage_in || h->stage_bytes < bytes) {
        if (h->stage_in) cudaFree(h->stage_in);
        if (h->stage_out) cudaFree(h->stage_out);
        h->stage_in = h->stage_out = nullptr;
        h->stage_bytes = 0;
        if (cudaMalloc(&h->stage_in, bytes) != cudaSuccess ||
            cudaMalloc(&h->stage_out, bytes) != cudaSuccess) {
            cudaGetLastError();
            return STENCIL_ERR_OOM;
        }
        h->stage_bytes = bytes;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (h->ndim == 3 && h->variant.family == STENCIL_FAMILY_STREAM &&
        h->dims[0] >= 2 * std::max(16, 2 * h->radius))
        return apply_host_pipelined(*h, in_host, out_host, steps, s);
    if (cudaMemcpyAsync(h->stage_in, in_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return STENCIL_ERR_CUDA;
    int rc = run_steps(*h, h->cf.data(), h->stage_in, h->stage_out, steps, s);
    if (rc) return rc;
    if (cudaMemcpyAsync(out_host, h->stage_out, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return STENCIL_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(s));
}

int stencil_sync_status(stencil_handle h, void *stream) {
    if (!h) return STENCIL_ERR_BADARG;
    return status_take(h->status_slot, (cudaStream_t)stream);
}

int stencil_set_wait_limit(stencil_handle h, double seconds, int phantom_arrivals) {
    if (!h || !(seconds > 0.0) || seconds > 3600.0 || phantom_arrivals < 0 ||
        phantom_arrivals > 1000)
        return STENCIL_ERR_BADARG;
    h->wait.ns = (unsigned long long)(seconds * 1e9);
    if (h->wait.ns == 0) h->wait.ns = 1;
    h->wait.phantom = phantom_arrivals;
    return STENCIL_OK;
}

int stencil_plan_get_variant(stencil_handle h, stencil_variant *v) {
    if (!h || !v) return STENCIL_ERR_BADARG;
    *v = h->variant;
    return STENCIL_OK;
}

int stencil_plan_set_variant(stencil_handle h, const stencil_variant *v) {
    if (!h || !v) return STENCIL_ERR_BADARG;
    int rc = validate_variant(*h, *v);
    if (rc) return rc;
    h->variant = *v;
    return STENCIL_OK;
}

int stencil_load_dispatch_map(const char *path) {
    std::vector<MapEntry> entries;
    BatchShape batch[3];
    if (path) {
        FILE *f = std::fopen(path, "r");
        if (!f) return STENCIL_ERR_BADARG;
        char line[512];
        while (std::fgets(line, sizeof(line), f)) {
            char *hash = std::strchr(line, '#');
            if (hash) *hash = 0;
            // "batch dtype : tile_y tile_x fuse" -- the batched launch's shape per storage type
            int bdt = -1;
            BatchShape bs;
            if (std::sscanf(line, " batch %d : %d %d %d", &bdt, &bs.tile_y, &bs.tile_x,
                            &bs.fuse) == 4) {
                if (bdt < 0 || bdt > 2 || bs.tile_y < 1 || bs.tile_x < 1 || bs.fuse < 1) {
                    std::fclose(f);
                    return STENCIL_ERR_BADARG;
                }
                batch[bdt] = bs;
                continue;
            }
            MapEntry e;
            std::memset(&e, 0, sizeof(e));
            e.key[7] = -1;  // no geometry field: any geometry
            char *colon = std::strchr(line, ':');
            int nk = 0, nv = 0;
            if (colon) {
                *colon = 0;
                nk = std::sscanf(line, "%d %d %d %d %d %d %d %d", &e.key[0], &e.key[1],
                                 &e.key[2], &e.key[3], &e.key[4], &e.key[5], &e.key[6],
                                 &e.key[7]);
                nv = std::sscanf(colon + 1, "%d %d %d %d %d %d %d %d %d", &e.v.family,
                                 &e.v.block_x, &e.v.block_y, &e.v.vec_y, &e.v.z_chunk,
                                 &e.v.fuse, &e.v.tile_x, &e.v.tile_y, &e.v.stages);
            }
            // 7 or 8 key fields (the geometry is optional), 8 or 9 values (the ring depth is
            // optional: 0 = automatic)
            if ((nk == 7 || nk == 8) && (nv == 8 || nv == 9)) {
                entries.push_back(e);
            } else {
                if (colon) *colon = ':';
                bool blank = true;
                for (char *c = line; *c; ++c)
                    if (!std::isspace((unsigned char)*c)) blank = false;
                if (!blank) {
                    std::fclose(f);
                    return STENCIL_ERR_BADARG;
                }
            }
        }
        std::fclose(f);
    }
    std::lock_guard<std::mutex> lk(g_map_mu);
    g_map.swap(entries);
    for (int i = 0; i < 3; ++i) g_batch_map[i] = batch[i];
    return STENCIL_OK;
}

}  // extern "C"

namespace gst {

// Variable-coefficient sweeps: `steps` launches ping-ponging through out and the scratch grid.
static int run_var_steps(stencil_plan_s &p, const void *in, const void *const *arrays,
                         void *out, int steps, bool adjoint, cudaStream_t s) {
    if (steps > 1) {
        int rc = ensure_scratch(p);
        if (rc) return rc;
    }
    VarLaunch L;
    L.ndim = p.ndim;
    L.nz = p.dims[0];
    L.ny = p.dims[1];
    L.nx = p.dims[2];
    L.shape = p.shape;
    L.radius = p.radius;
    L.dtype = p.dtype;
    L.periodic = p.boundary == STENCIL_PERIODIC;
    L.arrays = arrays;
    L.narrays = p.kind == STENCIL_DIVKGRAD ? 1 : (int)p.npts;
    L.block_y = p.variant.block_y;
    L.z_chunk = p.variant.z_chunk;
    L.vec_y = p.variant.vec_y;
    L.err = status_word(p.status_slot);
    L.wait = p.wait;
    L.stream = s;
    p.launched = true;
    const void *src = in;
    for (int g = 0; g < steps; ++g) {
        void *dst = ((steps - 1 - g) % 2 == 0) ? out : p.scratch;
        L.in = src;
        L.out = dst;
        int rc;
        if (p.kind == STENCIL_DIVKGRAD) {
            // the operator is symmetric: its adjoint is itself
            rc = p.dtype == STENCIL_F32   ? launch_divkgrad_f32(L)
                 : p.dtype == STENCIL_F16 ? launch_divkgrad_f16(L)
                                          : launch_divkgrad_bf16(L);
        } else if (!adjoint) {
            rc = p.dtype == STENCIL_F32   ? launch_var_f32_fwd(L)
                 : p.dtype == STENCIL_F16 ? launch_var_f16_fwd(L)
                                          : launch_var_bf16_fwd(L);
        } else {
            rc = p.dtype == STENCIL_F32   ? launch_var_f32_adj(L)
                 : p.dtype == STENCIL_F16 ? launch_var_f16_adj(L)
                                          : launch_var_bf16_adj(L);
        }
        if (rc) return map_launch_rc(rc);
        src = dst;
    }
    return STENCIL_OK;
}

static int apply_var_common(stencil_handle h, const void *in, const void *const *arrays,
                            void *out, int steps, void *stream, bool adjoint) {
    int rc = check_apply_args(h, in, out, steps);
    if (rc) return rc;
    if (h->kind != STENCIL_VAR && h->kind != STENCIL_DIVKGRAD) return STENCIL_ERR_BADARG;
    if (!arrays) return STENCIL_ERR_BADARG;
    const int n = h->kind == STENCIL_DIVKGRAD ? 1 : (int)h->npts;
    if (n > kMaxVarArrays) return STENCIL_ERR_UNSUPPORTED;
    const size_t bytes = (size_t)h->dims[0] * h->dims[1] * h->dims[2] * dtype_size(h->dtype);
    for (int i = 0; i < n; ++i) {
        if (!arrays[i]) return STENCIL_ERR_BADARG;
        if (overlaps(arrays[i], out, bytes)) return STENCIL_ERR_BADARG;
    }
    return run_var_steps(*h, in, arrays, out, steps, adjoint, (cudaStream_t)stream);
}

int launch_stream(const StreamLaunch &L) {
#define GST_CASE(DT, ND)                                                  \
    if (L.ndim == ND) {                                                   \
        if (L.shape == STENCIL_STAR) return launch_stream_##DT##_##ND##d_star(L);       \
        if (L.shape == STENCIL_BOX) return launch_stream_##DT##_##ND##d_box(L);         \
        if (L.shape == STENCIL_DIAMOND) return launch_stream_##DT##_##ND##d_diamond(L); \
    }
    switch (L.dtype) {
    case STENCIL_F32:
        GST_CASE(f32, 2) GST_CASE(f32, 3) break;
    case STENCIL_F16:
        GST_CASE(f16, 2) GST_CASE(f16, 3) break;
    case STENCIL_BF16:
        GST_CASE(bf16, 2) GST_CASE(bf16, 3) break;
    default: break;
    }
#undef GST_CASE
    return -2;
}

}  // namespace gst

extern "C" {

int stencil_apply_var(stencil_handle h, const void *in, const void *const *coeff_arrays,
                      void *out, int steps, void *stream) {
    return gst::apply_var_common(h, in, coeff_arrays, out, steps, stream, false);
}

int stencil_apply_adjoint_var(stencil_handle h, const void *in, const void *const *coeff_arrays,
                              void *out, int steps, void *stream) {
    return gst::apply_var_common(h, in, coeff_arrays, out, steps, stream, true);
}

}  // extern "C"

namespace gst {

// One launch of `k` steps with an explicit destination (used by the allocation-free entry
// point, which supplies its own ping-pong buffer).
int launch_group_with(stencil_plan_s &p, const float *cf, const void *src, void *dst, int k,
                      cudaStream_t s) {
    return launch_group(p, cf, src, dst, k, s);
}

int plan_steps_per_launch(const stencil_plan_s &p) { return steps_per_launch(p); }

}  // namespace gst

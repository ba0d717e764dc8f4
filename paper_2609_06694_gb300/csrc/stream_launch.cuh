// Host-side launchers of the streaming sweep kernel, instantiated per storage type.
#pragma once

#include <cstring>

#include <cudaTypedefs.h>

#include "internal.h"
#include "stream.cuh"

namespace gst {

// cuTensorMapEncodeTiled from the driver (looked up once; null if unavailable).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

template <typename T> constexpr CUtensorMapDataType tensor_dtype() {
    if constexpr (sizeof(T) == 4) return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    else if constexpr (Storage<T>::kDType == kF16) return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    else return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}

// Patch chunks of a tile (chunks the tensor copy zero-fills but a periodic grid wraps).
inline int64_t tile_patches(int64_t nx, int64_t ny, int x0, int y0, int R, int A, int pitch,
                            int rows) {
    const int64_t cpr = pitch / A;
    const int64_t lo_row = std::max<int64_t>(0, R - y0);
    const int64_t hi_row = std::min<int64_t>(rows, std::max<int64_t>(0, ny - (y0 - R)));
    const int64_t lo_chk = std::max<int64_t>(0, (A - x0 + A - 1) / A);
    const int64_t hi_chk = std::min<int64_t>(cpr, std::max<int64_t>(0, (nx - (x0 - A) + A - 1) / A));
    const int64_t row_oob = lo_row + (rows - hi_row);
    return row_oob * cpr + (hi_row - lo_row) * (lo_chk + (cpr - hi_chk));
}

// Queue mode: 3D stars split off their in-plane cross; other small stencils unroll the z loop
// by 2R+1 while the unrolled body stays small; larger ones rotate their partial-sum queue.
constexpr int stream_queue_mode(int ndim, int shape, int r, int vx, int vy) {
    if (ndim == 3 && shape == kStar) return kQueueStarSplit;
    if (ndim == 2 || shape_count(ndim, shape, r) * vx * vy * (2 * r + 1) <= 2000)
        return kQueueUnrolled;
    return kQueueRotate;
}

// CTAs of a kernel that can be resident on the whole GPU at once (cached per kernel and
// launch shape).
inline int resident_slots(const void *kern, int threads, size_t smem) {
    struct Entry {
        const void *k;
        int t;
        size_t s;
        int slots;
    };
    static Entry cache[64];
    static int ncache = 0;
    for (int i = 0; i < ncache; ++i)
        if (cache[i].k == kern && cache[i].t == threads && cache[i].s == smem) return cache[i].slots;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int slots = per * sms;
    if (ncache < 64) cache[ncache++] = {kern, threads, smem, slots};
    return slots;
}

template <typename T, int NDIM, int SHAPE, int R, int VY>
int launch_stream_t(const StreamLaunch &L) {
    constexpr int VX = 16 / (int)sizeof(T);
    constexpr int NSTAGE = NDIM == 3 ? 4 : 2;  // 2D grids load a single plane
    constexpr int NPTS = OffsetTable<NDIM, SHAPE, R>::count;
    constexpr int QM = stream_queue_mode(NDIM, SHAPE, R, VX, VY);
    using K = StreamKernel<T, NDIM, SHAPE, R, VY, NSTAGE, QM>;
    auto kern = stream_sweep_kernel<T, NDIM, SHAPE, R, VY, NSTAGE, QM>;

    const int by = L.block_y;
    if (L.block_x != K::BX || by < 1 || K::BX * by > K::MAX_THREADS || (K::BX * by) % 32 != 0)
        return -1;
    const int TX = K::TX, TY = by * VY;
    const int64_t nx = L.nx, ny = L.ny, nz = NDIM == 3 ? L.nz : 1;
    if (nx * ny > (int64_t)INT32_MAX - 4 * TX) return -2;

    StreamParams<T> p;
    p.in = static_cast<const T *>(L.in);
    p.out = static_cast<T *>(L.out);
    p.nx = (int)nx;
    p.ny = (int)ny;
    p.nz = (int)nz;
    p.periodic = L.periodic;
    p.tiles_x = (int)((nx + TX - 1) / TX);
    p.tiles_y = (int)((ny + TY - 1) / TY);
    const bool ptr_ok = ((uintptr_t)L.in % 16 == 0) && ((uintptr_t)L.out % 16 == 0);
    p.aligned = (ptr_ok && (nx * (int64_t)sizeof(T)) % 16 == 0) ? 1 : 0;
    p.err = L.err;

    // Tensor-map (TMA) loads when rows are 16-byte aligned, the box fits the TMA limits and,
    // for a periodic grid, the worst edge tile's wrapped chunks fit KP per thread.
    p.use_tma = 0;
    std::memset(&p.tmap, 0, sizeof(p.tmap));
    const int rows = TY + 2 * R;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (p.aligned && enc && rows <= 256 && K::PITCH <= 256 && L.use_tma != 0) {
        bool fits = true;
        if (L.periodic) {
            const int xs[2] = {0, (p.tiles_x - 1) * TX};
            const int ys[2] = {0, (p.tiles_y - 1) * TY};
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    if (tile_patches(nx, ny, xs[a], ys[b], R, K::A, K::PITCH, rows) >
                        (int64_t)K::KP * K::BX * by)
                        fits = false;
        }
        if (fits) {
            const cuuint64_t gdim[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
            const cuuint64_t gstride[2] = {(cuuint64_t)(nx * sizeof(T)),
                                           (cuuint64_t)(nx * ny * sizeof(T))};
            const cuuint32_t box[3] = {(cuuint32_t)K::PITCH, (cuuint32_t)rows, 1u};
            const cuuint32_t estr[3] = {1u, 1u, 1u};
            if (enc(&p.tmap, tensor_dtype<T>(), 3, const_cast<void *>(L.in), gdim, gstride, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
                p.use_tma = 1;
        }
    }

    ConstCoeffs<NPTS> cf;
    for (int i = 0; i < NPTS; ++i) cf.c[i] = L.coeffs[i];

    const size_t smem = K::smem_bytes(by);
    static size_t smem_set = 0;  // per instantiation
    if (smem > 48 * 1024 && smem > smem_set) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -4;
        smem_set = smem;
    }
    // Work split: z_chunk > 0 gives every CTA z_chunk planes; z_chunk == 0 sizes the grid to
    // the CTAs that fit on the GPU at once (a multiple of the SM count) and gives each an equal
    // share of the (tile, z) planes.
    const int64_t total = (int64_t)p.tiles_x * p.tiles_y * nz;
    int64_t work;
    if (L.z_chunk > 0) {
        work = L.z_chunk;
    } else {
        const int slots = resident_slots(reinterpret_cast<const void *>(kern), K::BX * by, smem);
        if (slots < 1) return -2;
        work = (total + slots - 1) / slots;
    }
    if (work > INT32_MAX) work = INT32_MAX;
    p.work = (int)work;
    const int64_t nblocks = (total + work - 1) / work;
    if (nblocks > INT32_MAX) return -2;
    kern<<<(unsigned)nblocks, dim3(K::BX, by), smem, L.stream>>>(p, cf);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <typename T, int NDIM, int SHAPE, int R> int launch_stream_vy(const StreamLaunch &L) {
    if (L.vec_y == 1) return launch_stream_t<T, NDIM, SHAPE, R, 1>(L);
    if constexpr (stream_vy_compiled(NDIM, SHAPE, R, 2)) {
        if (L.vec_y == 2) return launch_stream_t<T, NDIM, SHAPE, R, 2>(L);
    }
    if constexpr (stream_vy_compiled(NDIM, SHAPE, R, 4)) {
        if (L.vec_y == 4) return launch_stream_t<T, NDIM, SHAPE, R, 4>(L);
    }
    return -2;
}

template <typename T, int NDIM, int SHAPE> int launch_stream_r(const StreamLaunch &L) {
    switch (L.radius) {
    case 1: return launch_stream_vy<T, NDIM, SHAPE, 1>(L);
    case 2: return launch_stream_vy<T, NDIM, SHAPE, 2>(L);
    case 3: return launch_stream_vy<T, NDIM, SHAPE, 3>(L);
    case 4: return launch_stream_vy<T, NDIM, SHAPE, 4>(L);
    default: return -2;
    }
}

template <typename T, int NDIM> int launch_stream_shape(const StreamLaunch &L) {
    switch (L.shape) {
    case kStar: return launch_stream_r<T, NDIM, kStar>(L);
    case kBox: return launch_stream_r<T, NDIM, kBox>(L);
    case kDiamond: return launch_stream_r<T, NDIM, kDiamond>(L);
    default: return -2;
    }
}

}  // namespace gst

// Host-side helpers of the plane-ring kernels (ring.cuh): tensor maps, residency and the
// ring depth.
#pragma once

#include <algorithm>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "ring.cuh"

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

// The column-aligned split of z_chunk == -1 (RingWork with work = -c): c chunks per tile column,
// as many as the resident CTAs allow (at least one, at most nz); returns -c and the grid.
inline int ring_column_split(int64_t tiles, int64_t nz, int slots, int64_t *nblocks) {
    const int64_t c = std::max<int64_t>(1, std::min<int64_t>(nz, slots / std::max<int64_t>(1, tiles)));
    *nblocks = tiles * c;
    return -(int)c;
}

// CTAs of a kernel that can be resident on the whole current device at once (cached per
// device, kernel and launch shape, under a mutex).
inline int resident_slots(const void *kern, int threads, size_t smem) {
    struct Entry {
        int dev;
        const void *k;
        int t;
        size_t s;
        int slots;
    };
    static Entry cache[128];
    static int ncache = 0;
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < ncache; ++i)
        if (cache[i].dev == dev && cache[i].k == kern && cache[i].t == threads &&
            cache[i].s == smem)
            return cache[i].slots;
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int slots = per * sms;
    if (ncache < 128) cache[ncache++] = {dev, kern, threads, smem, slots};
    return slots;
}

// CTAs of a kernel that fit on one SM (registers, threads and shared memory), cached.
inline int ctas_per_sm(const void *kern, int threads, size_t smem) {
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 0;
    }
    return resident_slots(kern, threads, smem) / sms;
}

// Ring depth: the requested value, or (0) the deepest ring that keeps the CTAs the registers
// allow resident on an SM -- more planes in flight hide more of the memory latency.  `slot`
// is the bytes of one slot (all fields).
inline int ring_stages(int requested, int ndim, const void *kern, int threads, size_t slot) {
    if (ndim == 2) return 2;  // one plane per tile
    if (requested >= 2) return std::min(requested, kMaxStages);
    int dev = 0, per_sm = 0, optin = 0, reserved = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess) {
        cudaGetLastError();
        return 4;
    }
    // per slot: the slot and three mbarriers; per CTA: the abort flag and the patch list
    // (RingLayout::bytes)
    const size_t per_slot = slot + 24, fixed = 16 + 8 * kMaxPatches;
    const int ctas = std::max(1, ctas_per_sm(kern, threads, 2 * per_slot + fixed));
    const size_t budget = std::min<size_t>((size_t)optin, (size_t)per_sm / ctas - reserved);
    const int ns = (int)((budget - fixed) / per_slot);
    return std::max(2, std::min(ns, kMaxStages));
}

// A 3D tensor map of one field (nz x ny x nx, x fastest) with the box (pitch, rows, 1): the
// plane tile a ring slot holds.  False when the driver entry point is missing or the
// encoding is refused (the caller then loads without tensor maps).
template <typename T>
inline bool encode_plane_map(CUtensorMap *map, const void *base, int64_t nx, int64_t ny,
                             int64_t nz, int pitch, int rows) {
    std::memset(map, 0, sizeof(*map));
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || rows > 256 || pitch > 256) return false;
    const cuuint64_t gdim[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t gstride[2] = {(cuuint64_t)(nx * sizeof(T)), (cuuint64_t)(nx * ny * sizeof(T))};
    const cuuint32_t box[3] = {(cuuint32_t)pitch, (cuuint32_t)rows, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(map, tensor_dtype<T>(), 3, const_cast<void *>(base), gdim, gstride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

}  // namespace gst

// Host-side launchers of the variable-coefficient and div(k grad u) kernels.
#pragma once

#include <algorithm>

#include "internal.h"
#include "ring_launch.cuh"
#include "var.cuh"

namespace gst {

// Offset sets with at most kMaxVarPts points have VAR kernels.
constexpr bool var_compiled(int ndim, int shape, int r) {
    return r >= 1 && r <= 4 && shape_count(ndim, shape, r) <= kMaxVarPts;
}

template <typename T> static int fill_var_params(const VarLaunch &L, VarParams<T> &p, int by) {
    constexpr int VX = 16 / (int)sizeof(T), TX = 128;
    p.in = static_cast<const T *>(L.in);
    p.out = static_cast<T *>(L.out);
    bool ptr_ok = ((uintptr_t)L.in % 16 == 0) && ((uintptr_t)L.out % 16 == 0);
    for (int i = 0; i < kMaxVarPts; ++i) p.w[i] = nullptr;
    for (int i = 0; i < L.narrays; ++i) {
        p.w[i] = static_cast<const T *>(L.arrays[i]);
        if ((uintptr_t)L.arrays[i] % 16) ptr_ok = false;
    }
    p.nx = (int)L.nx;
    p.ny = (int)L.ny;
    p.nz = L.ndim == 3 ? (int)L.nz : 1;
    p.periodic = L.periodic;
    p.aligned = (ptr_ok && (L.nx * (int64_t)sizeof(T)) % 16 == 0) ? 1 : 0;
    p.tiles_x = (int)((L.nx + TX - 1) / TX);
    p.tiles_y = (int)((L.ny + by - 1) / by);
    p.zchunk = (L.ndim == 3 && L.z_chunk > 0) ? L.z_chunk : p.nz;
    (void)VX;
    return 0;
}

template <typename T, int NDIM, int SHAPE, int R, bool ADJ>
int launch_var_t(const VarLaunch &L) {
    constexpr int VX = 16 / (int)sizeof(T), BX = 128 / VX, PITCH = 128 + 2 * VX;
    constexpr int RZ = NDIM == 3 ? R : 0;
    constexpr int NSLOT = 2 * RZ + 2;
    const int by = L.block_y > 0 ? L.block_y : 8;
    if (BX * by > 256 || (BX * by) % 32) return -1;
    VarParams<T> p;
    fill_var_params<T>(L, p, by);
    const int64_t zchunks = NDIM == 3 ? (p.nz + p.zchunk - 1) / p.zchunk : 1;
    const int64_t nblocks = (int64_t)p.tiles_x * p.tiles_y * zchunks;
    if (nblocks > INT32_MAX) return -2;
    const size_t smem = (size_t)NSLOT * PITCH * (by + 2 * R) * sizeof(T);
    auto kern = var_sweep_kernel<T, NDIM, SHAPE, R, ADJ>;
    if (!smem_opt_in(reinterpret_cast<const void *>(kern), smem, false)) return -4;
    kern<<<(unsigned)nblocks, dim3(BX, by), smem, L.stream>>>(p);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <typename T, int NDIM, bool ADJ> int launch_var_shape(const VarLaunch &L) {
#define GST_VAR(S, RR)                                                      \
    if (L.shape == S && L.radius == RR) {                                   \
        if constexpr (var_compiled(NDIM, S, RR))                            \
            return launch_var_t<T, NDIM, S, RR, ADJ>(L);                    \
        else                                                                \
            return -2;                                                      \
    }
    GST_VAR(kStar, 1) GST_VAR(kStar, 2) GST_VAR(kStar, 3) GST_VAR(kStar, 4)
    GST_VAR(kBox, 1) GST_VAR(kBox, 2) GST_VAR(kBox, 3) GST_VAR(kBox, 4)
    GST_VAR(kDiamond, 1) GST_VAR(kDiamond, 2) GST_VAR(kDiamond, 3) GST_VAR(kDiamond, 4)
#undef GST_VAR
    return -2;
}

template <typename T, bool ADJ> int launch_var_dt(const VarLaunch &L) {
    if (L.ndim == 2) return launch_var_shape<T, 2, ADJ>(L);
    if (L.ndim == 3) return launch_var_shape<T, 3, ADJ>(L);
    return -1;
}

template <typename T, int NDIM, int VY> int launch_divkgrad_nd(const VarLaunch &L) {
    using K = DivkKernel<T, NDIM, VY>;
    auto kern = divkgrad_kernel<T, NDIM, VY>;
    int by = L.block_y > 0 ? L.block_y : 128 / K::BX;
    by = std::min(by, K::MAX_THREADS / K::BX);
    if ((K::BX * by) % 32) return -1;
    const int64_t nx = L.nx, ny = L.ny, nz = NDIM == 3 ? L.nz : 1;
    if (nx * ny > (int64_t)INT32_MAX - 4 * K::TX) return -2;
    DivkParams<T> p;
    p.field[0] = static_cast<const T *>(L.in);
    p.field[1] = static_cast<const T *>(L.arrays[0]);
    p.out = static_cast<T *>(L.out);
    p.nx = (int)nx;
    p.ny = (int)ny;
    p.nz = (int)nz;
    p.periodic = L.periodic;
    const bool ptr_ok = (uintptr_t)L.in % 16 == 0 && (uintptr_t)L.arrays[0] % 16 == 0 &&
                        (uintptr_t)L.out % 16 == 0;
    p.aligned = (ptr_ok && (nx * (int64_t)sizeof(T)) % 16 == 0) ? 1 : 0;
    p.tiles_x = (int)((nx + K::TX - 1) / K::TX);
    p.tiles_y = (int)((ny + by * VY - 1) / (by * VY));
    p.err = L.err;
    p.wait_ns = L.wait.ns;
    p.phantom = L.wait.phantom;
    const int rows = by * VY + 2;
    p.use_tma = (p.aligned &&
                 encode_plane_map<T>(&p.tmap[0], L.in, nx, ny, nz, K::PITCH, rows) &&
                 encode_plane_map<T>(&p.tmap[1], L.arrays[0], nx, ny, nz, K::PITCH, rows))
                    ? 1
                    : 0;
    const int threads = K::BX * by + 32;
    // consumers hold the 2RZ+1 planes of their window: the ring needs at least one more
    p.nstage = std::max(2 * K::RZ + 2, ring_stages(0, NDIM, reinterpret_cast<const void *>(kern),
                                                   threads, 2 * K::field_bytes(by)));
    const size_t smem = K::smem_bytes(by, p.nstage);
    if (!smem_opt_in(reinterpret_cast<const void *>(kern), smem, true)) return -4;
    // z chunks of z_chunk planes per CTA; z_chunk == 0 sizes the grid to the CTAs that fit on
    // the GPU at once and gives each an equal share of the (tile, z) planes (one wave, no tail)
    const int64_t total = (int64_t)p.tiles_x * p.tiles_y * nz;
    int64_t work = nz;
    if (NDIM == 3 && L.z_chunk > 0) {
        work = L.z_chunk;
    } else if (NDIM == 3) {
        const int slots = resident_slots(reinterpret_cast<const void *>(kern), threads, smem);
        if (slots < 1) return -2;
        work = (total + slots - 1) / slots;
    }
    p.work = (int)std::min<int64_t>(work, INT32_MAX);
    int64_t nblocks = (total + p.work - 1) / p.work;
    // z_chunk == -1: the same number of aligned chunks in every tile column (RingWork)
    if (NDIM == 3 && L.z_chunk < 0) {
        const int slots = resident_slots(reinterpret_cast<const void *>(kern), threads, smem);
        if (slots < 1) return -2;
        p.work = ring_column_split((int64_t)p.tiles_x * p.tiles_y, nz, slots, &nblocks);
    }
    if (nblocks > INT32_MAX) return -2;
    kern<<<(unsigned)nblocks, dim3(K::BX, by + 32 / K::BX), smem, L.stream>>>(p);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <typename T> int launch_divkgrad_t(const VarLaunch &L) {
    if (L.vec_y == 2)
        return L.ndim == 3 ? launch_divkgrad_nd<T, 3, 2>(L) : launch_divkgrad_nd<T, 2, 2>(L);
    if (L.vec_y != 1) return -1;
    return L.ndim == 3 ? launch_divkgrad_nd<T, 3, 1>(L) : launch_divkgrad_nd<T, 2, 1>(L);
}

}  // namespace gst

// Host-side launchers of the streaming sweep kernel, instantiated per storage type.
#pragma once

#include <cstring>
#include <type_traits>

#include "internal.h"
#include "ring_launch.cuh"
#include "stream.cuh"

namespace gst {

// Queue mode: the z loop is unrolled by 2R+1 while the unrolled body stays small; larger
// stencils rotate their partial-sum queue.
constexpr int stream_queue_mode(int ndim, int shape, int r, int vx, int vy) {
    if (ndim == 2 || shape_count(ndim, shape, r) * vx * vy * (2 * r + 1) <= 2000)
        return kQueueUnrolled;
    return kQueueRotate;
}

// The launch proper: ring depth, shared memory, work split, grid.
template <typename T, int NDIM, int SHAPE, int R, int VY, int QM, class EPI, bool SIDE>
int launch_stream_go(const StreamLaunch &L, StreamParams<T> &p,
                     const ConstCoeffs<OffsetTable<NDIM, SHAPE, R>::count> &cf,
                     const typename EPI::Params &ep) {
    using K = StreamKernel<T, NDIM, SHAPE, R, VY, QM>;
    auto kern = stream_sweep_kernel<T, NDIM, SHAPE, R, VY, QM, EPI, SIDE>;
    const int by = L.block_y;
    const int threads = K::BX * by + 32;  // consumers + the producer warp
    p.nstage = ring_stages(L.stages, NDIM, reinterpret_cast<const void *>(kern), threads,
                           K::slot_bytes(by, SIDE));
    const size_t smem = K::smem_bytes(by, SIDE, p.nstage);
    if (!smem_opt_in(reinterpret_cast<const void *>(kern), smem, true)) return -4;
    // Work split: z_chunk > 0 gives every CTA z_chunk planes; z_chunk == 0 sizes the grid to
    // the CTAs that fit on the GPU at once (a multiple of the SM count) and gives each an equal
    // share of the (tile, z) planes.
    const int64_t total = (int64_t)p.tiles_x * p.tiles_y * p.z_cnt;
    int64_t work, nblocks;
    if (L.z_chunk > 0) {
        work = L.z_chunk;
    } else {
        const int slots = resident_slots(reinterpret_cast<const void *>(kern), threads, smem);
        if (slots < 1) return -2;
        work = (total + slots - 1) / slots;
    }
    if (work > INT32_MAX) work = INT32_MAX;
    p.work = (int)work;
    nblocks = (total + work - 1) / work;
    // z_chunk == -1: the same number of aligned chunks in every tile column (RingWork)
    if (L.z_chunk < 0) {
        const int slots = resident_slots(reinterpret_cast<const void *>(kern), threads, smem);
        if (slots < 1) return -2;
        p.work = ring_column_split((int64_t)p.tiles_x * p.tiles_y, p.z_cnt, slots, &nblocks);
    }
    if (nblocks > INT32_MAX) return -2;
    kern<<<(unsigned)nblocks, dim3(K::BX, by + 32 / K::BX), smem, L.stream>>>(p, cf, ep);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

// One launch of the streaming kernel; EPI decides what happens to finished outputs (the plain
// store, or a fused update with its own parameter block `ep`).
template <typename T, int NDIM, int SHAPE, int R, int VY, class EPI = PlainStoreEpi>
int launch_stream_t(const StreamLaunch &L,
                    const typename EPI::Params &ep = typename EPI::Params{}) {
    constexpr int VX = 16 / (int)sizeof(T);
    constexpr int NPTS = OffsetTable<NDIM, SHAPE, R>::count;
    constexpr int QM = stream_queue_mode(NDIM, SHAPE, R, VX, VY);
    using K = StreamKernel<T, NDIM, SHAPE, R, VY, QM>;

    const int by = L.block_y;
    if (L.block_x != K::BX || by < 1 || K::BX * by > K::MAX_THREADS || (K::BX * by) % 32 != 0)
        return -1;
    const int TX = K::TX, TY = by * VY;
    const int64_t nx = L.nx, ny = L.ny, nz = NDIM == 3 ? L.nz : 1;
    if (nx * ny > (int64_t)INT32_MAX - 4 * TX) return -2;

    StreamParams<T> p{};
    p.in = static_cast<const T *>(L.in);
    p.out = static_cast<T *>(L.out);
    p.nx = (int)nx;
    p.ny = (int)ny;
    p.nz = (int)nz;
    p.periodic = L.periodic;
    p.tiles_x = (int)((nx + TX - 1) / TX);
    p.tiles_y = (int)((ny + TY - 1) / TY);
    p.z_lo = NDIM == 3 ? (int)std::max<int64_t>(0, L.z_lo) : 0;
    const int64_t z_hi = NDIM == 3 ? (L.z_hi < 0 ? nz : std::min<int64_t>(L.z_hi, nz)) : 1;
    if (z_hi <= p.z_lo) return 0;  // nothing to sweep
    p.z_cnt = (int)(z_hi - p.z_lo);
    const bool ptr_ok = ((uintptr_t)L.in % 16 == 0) && ((uintptr_t)L.out % 16 == 0);
    p.aligned = (ptr_ok && (nx * (int64_t)sizeof(T)) % 16 == 0) ? 1 : 0;
    p.err = L.err;
    p.wait_ns = L.wait.ns;
    p.phantom = L.wait.phantom;

    // Tensor-map (TMA) loads when rows are 16-byte aligned and the box fits the TMA limits
    // (the chunks a periodic grid wraps into an edge tile are filled inside the kernel).
    const int rows = TY + 2 * R;
    p.use_tma = (p.aligned && L.use_tma != 0 &&
                 encode_plane_map<T>(&p.tmap, L.in, nx, ny, nz, K::PITCH, rows))
                    ? 1
                    : 0;
    // periodic grids: the wrapped x halo chunks of edge tiles by a second map (one chunk wide)
    p.use_side = (p.use_tma && L.periodic &&
                  encode_plane_map<T>(&p.side_tmap, L.in, nx, ny, nz, 2 * K::A, rows))
                     ? 1
                     : 0;

    // periodic tile rows at the y ends: their wrapped rows by split tensor copies (ring.cuh,
    // mode 6) where each split lands on a 128-byte boundary of the slot (and of the side
    // arrays, 32-byte rows), the top row of tiles needs no bottom wrap (ny >= TY + 2R) and
    // only the last row of tiles wraps at the bottom (its hb output rows >= R).  Compiled
    // for radius 4 only (the one radius whose top split lands on 128 bytes: R rows of 16-byte
    // chunks); the smaller kernels keep the producer's registers.
    p.ysplit = 0;
    if (R == 4 && p.use_tma && L.periodic && p.tiles_y >= 2 && ny >= TY + 2 * R) {
        const int64_t hb = ny - (int64_t)(p.tiles_y - 1) * TY;
        const int64_t row_bytes = (int64_t)K::PITCH * (int64_t)sizeof(T);
        auto fits = [&](int64_t split) {
            return (split * row_bytes) % 128 == 0 &&
                   (!p.use_side || (split * kSideRowBytes) % 128 == 0);
        };
        auto maps = [&](int k, int box_rows) {
            return encode_plane_map<T>(&p.ymap[k], L.in, nx, ny, nz, K::PITCH, box_rows) &&
                   (!p.use_side || encode_plane_map<T>(&p.ymap[k + 3], L.in, nx, ny, nz,
                                                       2 * K::A, box_rows));
        };
        if (hb >= R && maps(2, R)) {
            if (fits(R) && maps(0, TY + R)) p.ysplit |= 1;
            if (fits(hb + R) && maps(1, (int)hb + R)) p.ysplit |= 2;
        }
    }

    ConstCoeffs<NPTS> cf;
    for (int i = 0; i < NPTS; ++i) cf.c[i] = L.coeffs[i];

    // the side-array kernel (with the y-split copies) only where side chunks may be taken
    // (plain periodic sweeps)
    if constexpr (std::is_same<EPI, PlainStoreEpi>::value) {
        if (p.use_side) return launch_stream_go<T, NDIM, SHAPE, R, VY, QM, EPI, true>(L, p, cf, ep);
    }
    p.use_side = 0;
    p.ysplit = 0;
    return launch_stream_go<T, NDIM, SHAPE, R, VY, QM, EPI, false>(L, p, cf, ep);
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

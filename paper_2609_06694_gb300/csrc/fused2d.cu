// Launchers of the fused multi-step 2D kernel (all storage types, shapes and radii).
#include "fused2d.cuh"
#include "internal.h"

namespace gst {

size_t fused2d_smem_bytes(int tile_x, int tile_y, int radius, int steps) {
    const size_t h = (size_t)radius * steps;
    return (steps > 1 ? 2 : 1) * (tile_x + 2 * h) * (tile_y + 2 * h) * sizeof(float);
}

template <typename T, int SHAPE, int R> static int launch_fused2d_t(const Fused2DLaunch &L) {
    constexpr int NPTS = OffsetTable<2, SHAPE, R>::count;
    auto kern = fused2d_kernel<T, SHAPE, R>;
    if (L.steps < 1 || L.tile_x < 1 || L.tile_y < 1) return -1;
    if (L.block_threads < 32 || L.block_threads > 256 || L.block_threads % 32) return -1;
    const size_t smem = fused2d_smem_bytes(L.tile_x, L.tile_y, R, L.steps);
    if (smem > 227 * 1024) return -2;
    if (!smem_opt_in(reinterpret_cast<const void *>(kern), smem, false)) return -4;
    ConstCoeffs<NPTS> cf;
    for (int i = 0; i < NPTS; ++i) cf.c[i] = L.coeffs[i];
    const int64_t tiles_x = (L.nx + L.tile_x - 1) / L.tile_x;
    const int64_t tiles_y = (L.ny + L.tile_y - 1) / L.tile_y;
    if (tiles_x * tiles_y > INT32_MAX || L.nx * L.ny > INT32_MAX) return -2;
    kern<<<(unsigned)(tiles_x * tiles_y), L.block_threads, smem, L.stream>>>(
        static_cast<const T *>(L.in), static_cast<T *>(L.out), (int)L.ny, (int)L.nx, L.periodic,
        L.steps, L.tile_y, L.tile_x, (int)tiles_x, cf);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <typename T, int SHAPE> static int launch_fused2d_r(const Fused2DLaunch &L) {
    switch (L.radius) {
    case 1: return launch_fused2d_t<T, SHAPE, 1>(L);
    case 2: return launch_fused2d_t<T, SHAPE, 2>(L);
    case 3: return launch_fused2d_t<T, SHAPE, 3>(L);
    case 4: return launch_fused2d_t<T, SHAPE, 4>(L);
    default: return -2;
    }
}

template <typename T> static int launch_fused2d_s(const Fused2DLaunch &L) {
    switch (L.shape) {
    case kStar: return launch_fused2d_r<T, kStar>(L);
    case kBox: return launch_fused2d_r<T, kBox>(L);
    case kDiamond: return launch_fused2d_r<T, kDiamond>(L);
    default: return -2;
    }
}

int launch_fused2d(const Fused2DLaunch &L) {
    switch (L.dtype) {
    case kF32: return launch_fused2d_s<float>(L);
    case kF16: return launch_fused2d_s<__half>(L);
    case kBF16: return launch_fused2d_s<__nv_bfloat16>(L);
    default: return -2;
    }
}

}  // namespace gst

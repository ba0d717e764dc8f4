// Launchers of the two-step fused 3D kernel (fused3d.cuh): every storage type; star and
// diamond offset sets of radius 1 and 2, the 27-point box.
#include <algorithm>
#include <cstring>

#include "fused3d.cuh"
#include "internal.h"
#include "ring_launch.cuh"

namespace gst {

template <typename T, int SHAPE, int R> static int launch_fused3d_t(const StreamLaunch &L) {
    using K = Fused3DKernel<T, SHAPE, R>;
    auto kern = fused3d_kernel<T, SHAPE, R>;
    const int by = L.block_y;
    if (L.block_x != K::BX || L.vec_y != K::VY2 || by < 2 * R || K::BX * by > K::MAX_THREADS ||
        (K::BX * by) % 32 != 0)
        return -1;
    const int64_t nx = L.nx, ny = L.ny, nz = L.nz;
    if (nx * ny > (int64_t)INT32_MAX - 4 * K::TX) return -2;
    const int TY = by * K::VY2;
    Fused3DParams<T> p{};
    p.in = static_cast<const T *>(L.in);
    p.out = static_cast<T *>(L.out);
    p.nx = (int)nx;
    p.ny = (int)ny;
    p.nz = (int)nz;
    p.periodic = L.periodic;
    const bool ptr_ok = ((uintptr_t)L.in % 16 == 0) && ((uintptr_t)L.out % 16 == 0);
    // the kernel writes its intermediate plane as 16-byte vectors and stores whole vectors
    // where a row is complete: rows of a multiple of 16 bytes only
    p.aligned = (ptr_ok && (nx * (int64_t)sizeof(T)) % 16 == 0) ? 1 : 0;
    p.tiles_x = (int)((nx + K::TX - 1) / K::TX);
    p.tiles_y = (int)((ny + TY - 1) / TY);
    p.err = L.err;
    p.wait_ns = L.wait.ns;
    p.phantom = L.wait.phantom;
    p.use_tma = (p.aligned && L.use_tma != 0 &&
                 encode_plane_map<T>(&p.tmap, L.in, nx, ny, nz, K::PITCH, TY + 4 * R))
                    ? 1
                    : 0;
    const int threads = K::BX * by + 32;
    // ring depth: as requested, else 4; fewer when the shared memory of one CTA runs out
    int ns = L.stages >= 2 ? std::min(L.stages, kMaxStages) : 4;
    while (ns > 2 && K::smem_bytes(by, ns) > 227 * 1024) --ns;
    const size_t smem = K::smem_bytes(by, ns);
    if (smem > 227 * 1024) return -2;
    p.nstage = ns;
    if (!smem_opt_in(reinterpret_cast<const void *>(kern), smem, true)) return -4;
    const int64_t total = (int64_t)p.tiles_x * p.tiles_y * nz;
    int64_t work;
    if (L.z_chunk > 0) {
        work = L.z_chunk;
    } else {
        const int slots = resident_slots(reinterpret_cast<const void *>(kern), threads, smem);
        if (slots < 1) return -2;
        work = (total + slots - 1) / slots;
    }
    p.work = (int)std::min<int64_t>(work, INT32_MAX);
    const int64_t nblocks = (total + p.work - 1) / p.work;
    if (nblocks > INT32_MAX) return -2;
    ConstCoeffs<K::NPTS> cf;
    for (int i = 0; i < K::NPTS; ++i) cf.c[i] = L.coeffs[i];
    kern<<<(unsigned)nblocks, dim3(K::BX, by + 32 / K::BX), smem, L.stream>>>(p, cf);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <typename T> static int launch_fused3d_dt(const StreamLaunch &L) {
    if (L.shape == kStar && L.radius == 1) return launch_fused3d_t<T, kStar, 1>(L);
    if (L.shape == kStar && L.radius == 2) return launch_fused3d_t<T, kStar, 2>(L);
    if (L.shape == kDiamond && L.radius == 1) return launch_fused3d_t<T, kStar, 1>(L);
    if (L.shape == kDiamond && L.radius == 2) return launch_fused3d_t<T, kDiamond, 2>(L);
    if (L.shape == kBox && L.radius == 1) return launch_fused3d_t<T, kBox, 1>(L);
    return -2;
}

int launch_fused3d(const StreamLaunch &L) {
    if (L.ndim != 3) return -2;
    switch (L.dtype) {
    case kF32: return launch_fused3d_dt<float>(L);
    case kF16: return launch_fused3d_dt<__half>(L);
    case kBF16: return launch_fused3d_dt<__nv_bfloat16>(L);
    default: return -2;
    }
}

}  // namespace gst

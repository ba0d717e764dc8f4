// Host launcher of the tensor-core (Toeplitz) radius-2 box sweep (toeplitz.cuh).
#include <algorithm>

#include "internal.h"
#include "ring_launch.cuh"
#include "toeplitz.cuh"

namespace gst {

namespace {

template <typename T, int NB, int DZN, int MW>
int launch_tz(const StreamLaunch &L) {
    const int ndim = L.ndim;
    const int64_t nz = ndim == 3 ? L.nz : 1;
    CUtensorMap map;
    if (!encode_plane_map<T>(&map, L.in, L.nx, L.ny, nz, 8, tz::kRows)) return -2;
    ToeplitzParams P;
    P.out = L.out;
    P.nz = (int)nz;
    P.ny = (int)L.ny;
    P.nx = (int)L.nx;
    P.tiles_x = (int)((L.nx + 16 * NB - 1) / (16 * NB));
    P.tiles_y = (int)((L.ny + 127) / 128);
    P.z_lo = ndim == 3 ? (int)L.z_lo : 0;
    P.z_hi = ndim == 3 ? (int)(L.z_hi < 0 ? nz : L.z_hi) : 1;
    P.err = L.err;
    P.wait_ns = L.wait.ns;
    P.phantom = L.wait.phantom;
    const void *kern = (const void *)toeplitz_box_kernel<T, NB, DZN, MW>;
    constexpr int threads = tz::threads(MW);
    // ring depth: at least 5 (the input planes of one output plane in 3D), as deep as two CTAs
    // per SM allow, else as deep as one allows
    int ns = L.stages;
    if (ns == 0) {
        int dev = 0, per_sm = 0, optin = 0, reserved = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        const int fixed = tz::smem_bytes(NB, DZN, 0);
        const int two = (per_sm / 2 - reserved - fixed - 16) / (tz::slot_bytes(NB) + 16);
        const int one = (std::min(optin, per_sm - reserved) - fixed - 16) /
                        (tz::slot_bytes(NB) + 16);
        ns = DZN == 1 ? 2 : (two >= 6 ? std::min(two, 12) : std::min(one, 12));
    }
    if (ns < (DZN == 1 ? 2 : 5) || ns > 12) return -1;
    P.stages = ns;
    // no more CTAs per SM than the tensor memory holds (512 columns), so that no CTA waits in
    // its allocation: the shared-memory request is raised to keep the others off the SM
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int max_ctas = 512 / tz::tmem_cols(NB);
    const int smem = std::max(tz::smem_bytes(NB, DZN, ns), per_sm / (max_ctas + 1) + 1024);
    if (!smem_opt_in(kern, (size_t)smem, false)) return -2;
    const int nzr = P.z_hi - P.z_lo;
    if (nzr <= 0) return 0;
    const int items_xy = P.tiles_x * P.tiles_y;
    int zc = L.z_chunk;
    if (ndim == 2) {
        zc = 1;
    } else if (zc <= 0) {
        // one wave: as many z chunks per column of tiles as the resident CTAs allow
        const int slots = resident_slots(kern, threads, smem);
        const int chunks = std::max(1, std::min(nzr, slots / std::max(1, items_xy)));
        zc = (nzr + chunks - 1) / chunks;
    }
    P.z_chunk = zc;
    const int64_t grid = (int64_t)items_xy * ((nzr + zc - 1) / zc);
    if (grid > 0x7fffffff) return -1;
    ToeplitzCoeffs<DZN * 25> cf;
    for (int i = 0; i < DZN * 25; ++i) cf.c[i] = L.coeffs[i];
    toeplitz_box_kernel<T, NB, DZN, MW><<<(unsigned)grid, threads, smem, L.stream>>>(map, P, cf);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <typename T, int DZN>
int launch_nb(const StreamLaunch &L, int nb, int mw) {
    switch (nb * 8 + mw) {
    case 1 * 8 + 1: return launch_tz<T, 1, DZN, 1>(L);
    case 1 * 8 + 2: return launch_tz<T, 1, DZN, 2>(L);
    case 2 * 8 + 1: return launch_tz<T, 2, DZN, 1>(L);
    case 2 * 8 + 2: return launch_tz<T, 2, DZN, 2>(L);
    case 4 * 8 + 1: return launch_tz<T, 4, DZN, 1>(L);
    case 4 * 8 + 2: return launch_tz<T, 4, DZN, 2>(L);
    case 4 * 8 + 4: return launch_tz<T, 4, DZN, 4>(L);
    default: return -1;
    }
}

}  // namespace

int launch_toeplitz(const StreamLaunch &L, int nb, int mw) {
    if (!toeplitz_compiled(L.ndim, L.shape, L.radius, L.dtype) || L.periodic || L.nx % 8 != 0)
        return -2;
    if (L.dtype == 2)
        return L.ndim == 3 ? launch_nb<__nv_bfloat16, 5>(L, nb, mw)
                           : launch_nb<__nv_bfloat16, 1>(L, nb, mw);
    return L.ndim == 3 ? launch_nb<__half, 5>(L, nb, mw) : launch_nb<__half, 1>(L, nb, mw);
}

}  // namespace gst

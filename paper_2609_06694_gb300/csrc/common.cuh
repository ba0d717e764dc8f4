// Device-side building blocks shared by the stencil kernels: storage-type traits,
// compile-time offset sets (ForgeStencil Sec. 2.1), cp.async wrappers, bounded waits and the
// device error word.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gst {

// ---------------------------------------------------------------------------------------
// Shapes and status codes (same numeric values as include/stencil.h)
// ---------------------------------------------------------------------------------------
enum Shape : int { kStar = 0, kBox = 1, kDiamond = 2 };
enum DType : int { kF32 = 0, kF16 = 1, kBF16 = 2 };
enum Boundary : int { kDirichlet0 = 0, kPeriodic = 1 };

constexpr int kErrTimeout = -5;
constexpr int kErrBounds = -6;

// ---------------------------------------------------------------------------------------
// Storage types.  Values are held as T in memory and as float in registers; the conversion
// to T rounds to nearest even.
// ---------------------------------------------------------------------------------------
template <typename T> struct Storage;
template <> struct Storage<float> {
    static constexpr int kDType = kF32;
    __device__ __forceinline__ static float to_float(float v) { return v; }
    __device__ __forceinline__ static float from_float(float v) { return v; }
};
template <> struct Storage<__half> {
    static constexpr int kDType = kF16;
    __device__ __forceinline__ static float to_float(__half v) { return __half2float(v); }
    __device__ __forceinline__ static __half from_float(float v) { return __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
    static constexpr int kDType = kBF16;
    __device__ __forceinline__ static float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ __forceinline__ static __nv_bfloat16 from_float(float v) { return __float2bfloat16_rn(v); }
};

// Round an f32 value to the storage grid of T and back (identity for float).
template <typename T> __device__ __forceinline__ float round_to_storage(float v) {
    return Storage<T>::to_float(Storage<T>::from_float(v));
}

// ---------------------------------------------------------------------------------------
// Offset sets in canonical order (lexicographic in (dz, dy, dx), each from -r to r).
// For a 2D stencil dz is always 0.
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr int iabs_c(int v) { return v < 0 ? -v : v; }

__host__ __device__ constexpr bool in_shape(int ndim, int shape, int r, int dz, int dy, int dx) {
    if (ndim == 2 && dz != 0) return false;
    if (iabs_c(dz) > r || iabs_c(dy) > r || iabs_c(dx) > r) return false;
    if (shape == kStar) return ((dz != 0) + (dy != 0) + (dx != 0)) <= 1;
    if (shape == kBox) return true;
    return iabs_c(dz) + iabs_c(dy) + iabs_c(dx) <= r;  // diamond
}

__host__ __device__ constexpr int shape_count(int ndim, int shape, int r) {
    int n = 0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (in_shape(ndim, shape, r, dz, dy, dx)) ++n;
    return n;
}

// Canonical index of an offset, or -1 if it is not in the set.
__host__ __device__ constexpr int shape_index(int ndim, int shape, int r, int dz, int dy, int dx) {
    if (!in_shape(ndim, shape, r, dz, dy, dx)) return -1;
    int n = 0;
    for (int a = -r; a <= r; ++a)
        for (int b = -r; b <= r; ++b)
            for (int c = -r; c <= r; ++c) {
                if (a == dz && b == dy && c == dx) return n;
                if (in_shape(ndim, shape, r, a, b, c)) ++n;
            }
    return -1;
}

// Largest |dx| among offsets with the given (dz, dy); -1 if there is none.
__host__ __device__ constexpr int max_dx(int ndim, int shape, int r, int dz, int dy) {
    int m = -1;
    for (int dx = -r; dx <= r; ++dx)
        if (in_shape(ndim, shape, r, dz, dy, dx) && iabs_c(dx) > m) m = iabs_c(dx);
    return m;
}

// Largest |dx| among offsets with the given dy over every dz; -1 if none.
__host__ __device__ constexpr int max_dx_any_dz(int ndim, int shape, int r, int dy) {
    int m = -1;
    for (int dz = -r; dz <= r; ++dz) {
        int v = max_dx(ndim, shape, r, dz, dy);
        if (v > m) m = v;
    }
    return m;
}

// Per-stencil lookup table, computed once per (ndim, shape, radius) at compile time:
// canonical index of every offset (-1 outside the set) and the largest |dx| per (dz, dy).
template <int NDIM, int SHAPE, int R> struct OffsetTable {
    static constexpr int D = 2 * R + 1;
    struct Tab {
        int idx[D][D][D];
        int mdx[D][D];     // max |dx| at (dz, dy), -1 if none
        int mdx_any[D];    // max |dx| at dy over every dz, -1 if none
        int count;
    };
    static constexpr Tab make() {
        Tab t{};
        int n = 0;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) {
                t.mdx[a][b] = -1;
                for (int c = 0; c < D; ++c) {
                    if (in_shape(NDIM, SHAPE, R, a - R, b - R, c - R)) {
                        t.idx[a][b][c] = n++;
                        if (iabs_c(c - R) > t.mdx[a][b]) t.mdx[a][b] = iabs_c(c - R);
                    } else {
                        t.idx[a][b][c] = -1;
                    }
                }
            }
        for (int b = 0; b < D; ++b) {
            t.mdx_any[b] = -1;
            for (int a = 0; a < D; ++a)
                if (t.mdx[a][b] > t.mdx_any[b]) t.mdx_any[b] = t.mdx[a][b];
        }
        t.count = n;
        return t;
    }
    static constexpr Tab tab = make();
    __host__ __device__ static constexpr int index(int dz, int dy, int dx) {
        return tab.idx[dz + R][dy + R][dx + R];
    }
    __host__ __device__ static constexpr int max_dx_any(int dy) { return tab.mdx_any[dy + R]; }
    static constexpr int count = tab.count;
};

// ---------------------------------------------------------------------------------------
// cp.async (16-byte, L2-only) with zero fill, and group waits.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src, int src_bytes) {
    uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem_src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------------------
// mbarrier + bulk asynchronous copies (global -> shared, completion counted in bytes).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking test for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete; false after `limit_ns` without it.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned int i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
    }
}
// As mbar_wait_bounded, but also gives up (false) once *abort_flag is nonzero: another warp of
// the CTA has stopped, so the arrival may never come.
__device__ __forceinline__ bool mbar_wait_abortable(uint32_t bar, uint32_t parity,
                                                    unsigned long long limit_ns,
                                                    const volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned int i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0 && (*abort_flag != 0 || globaltimer_ns() - t0 > limit_ns)) return false;
    }
}
// Order earlier generic-proxy accesses of shared memory before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) into shared memory,
// completing `bytes` transactions on the mbarrier.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                              uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// 16-byte cp.async to a shared-memory address, zero-filling when src_bytes == 0.
__device__ __forceinline__ void cp_async16_u32(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
// Arrive on the mbarrier once all earlier cp.async of this thread have landed (the arrival is
// one of the barrier's expected arrivals).
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// 3D tiled tensor copy global -> shared (TMA); out-of-range elements are filled with zeros.
// x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// ---------------------------------------------------------------------------------------
// Device error word: the first nonzero code wins.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void latch_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

__host__ __device__ constexpr int imod_c(int a, int n) {
    int m = a % n;
    return m < 0 ? m + n : m;
}

__device__ __forceinline__ int wrap_or_flag(int i, int n, bool periodic, bool &ok) {
    if (i >= 0 && i < n) return i;
    if (periodic) {
        int m = i % n;
        return m < 0 ? m + n : m;
    }
    ok = false;
    return 0;
}

}  // namespace gst

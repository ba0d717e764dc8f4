// Several time steps of a 2D stencil in one launch (temporal blocking, ForgeStencil Sec. 4.3:
// intermediate time levels stay on chip).
//
// A CTA owns an output tile and loads it with a halo of H = R * steps cells into shared
// memory (FP32).  Step s recomputes the tile grown by R * (steps - s) cells, so after `steps`
// steps exactly the tile is valid; the cells of the halo that lie outside a Dirichlet grid are
// held at zero and every intermediate value is rounded to the storage type, so the fused
// result equals `steps` single sweeps bit for bit in exact arithmetic order.
//
// The tile engine is a device function so that the persistent batched kernel can run it on
// tiles of many grids.
#pragma once

#include "common.cuh"
#include "stream.cuh"

namespace gst {

struct Fused2DTile {
    int ny, nx;       // grid extents
    int periodic;
    int y0, x0;       // output tile origin
    int th, tw;       // output tile extents (clipped by the caller to the grid, >= 1)
    int steps;        // steps fused (>= 1)
};

// A load that bypasses L1 (cache at L2 only): needed when other SMs wrote the buffer earlier
// in the same launch and this SM may still hold stale lines of it.
template <typename T> __device__ __forceinline__ T load_l2(const T *p) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 2, "4- or 2-byte values");
    if constexpr (sizeof(T) == 4) {
        unsigned int v = __ldcg(reinterpret_cast<const unsigned int *>(p));
        T r;
        memcpy(&r, &v, 4);
        return r;
    } else {
        unsigned short v = __ldcg(reinterpret_cast<const unsigned short *>(p));
        T r;
        memcpy(&r, &v, 2);
        return r;
    }
}

// Runs `t.steps` sweeps on one tile.  `buf` holds 2 * (th + 2H) * (tw + 2H) floats.
// `coef(idx)` returns the coefficient of canonical offset idx.  All threads of the block must
// call this; it ends with a __syncthreads().  COHERENT loads the input through L2 only.
template <typename T, int SHAPE, int R, bool COHERENT = false, typename Coef>
__device__ __forceinline__ void fused2d_tile(const T *__restrict__ in, T *__restrict__ out,
                                             const Fused2DTile &t, float *buf, const Coef &coef) {
    const int H = R * t.steps;
    const int W = t.tw + 2 * H;
    const int Hh = t.th + 2 * H;
    const int n = W * Hh;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const bool periodic = t.periodic != 0;
    float *src = buf, *dst = buf + n;

    // load the tile with its halo (zero outside a Dirichlet grid)
    for (int e = tid; e < n; e += nthr) {
        int row = e / W, col = e - row * W;
        bool ok = true;
        int gy = wrap_or_flag(t.y0 - H + row, t.ny, periodic, ok);
        int gx = wrap_or_flag(t.x0 - H + col, t.nx, periodic, ok);
        const T *a = in + (size_t)gy * t.nx + gx;
        src[e] = ok ? Storage<T>::to_float(COHERENT ? load_l2(a) : *a) : 0.0f;
    }
    __syncthreads();

    for (int s = 1; s <= t.steps; ++s) {
        const int g = R * s;  // rows/cols of the region not recomputed at this step
        const int rw = W - 2 * g, rh = Hh - 2 * g;
        const int rn = rw * rh;
        const bool last = (s == t.steps);
        for (int e = tid; e < rn; e += nthr) {
            const int row = g + e / rw, col = g + e % rw;
            const float *c0 = src + row * W + col;
            float v = 0.0f;
            static_for<2 * R + 1>([&](auto dyi) {
                constexpr int dy = decltype(dyi)::value - R;
                static_for<2 * R + 1>([&](auto dxi) {
                    constexpr int dx = decltype(dxi)::value - R;
                    constexpr int idx = OffsetTable<2, SHAPE, R>::index(0, dy, dx);
                    if constexpr (idx >= 0) v = fmaf(coef(idx), c0[dy * W + dx], v);
                });
            });
            const int gy = t.y0 - H + row, gx = t.x0 - H + col;
            if (!periodic && (gy < 0 || gy >= t.ny || gx < 0 || gx >= t.nx)) v = 0.0f;
            if (last) {
                if (gy >= 0 && gy < t.ny && gx >= 0 && gx < t.nx && row >= H && row < H + t.th &&
                    col >= H && col < H + t.tw)
                    out[(size_t)gy * t.nx + gx] = Storage<T>::from_float(v);
            } else {
                dst[row * W + col] = round_to_storage<T>(v);
            }
        }
        __syncthreads();
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
}

template <typename T, int SHAPE, int R>
__global__ void __launch_bounds__(256)
    fused2d_kernel(const T *__restrict__ in, T *__restrict__ out, int ny, int nx, int periodic,
                   int steps, int tile_y, int tile_x, int tiles_x,
                   const __grid_constant__ ConstCoeffs<OffsetTable<2, SHAPE, R>::count> cf) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>(smem_raw);
    Fused2DTile t;
    t.ny = ny;
    t.nx = nx;
    t.periodic = periodic;
    t.steps = steps;
    const int tix = blockIdx.x % tiles_x, tiy = blockIdx.x / tiles_x;
    t.y0 = tiy * tile_y;
    t.x0 = tix * tile_x;
    t.th = min(tile_y, ny - t.y0);
    t.tw = min(tile_x, nx - t.x0);
    fused2d_tile<T, SHAPE, R>(in, out, t, buf, [&](int idx) { return cf.c[idx]; });
}

}  // namespace gst

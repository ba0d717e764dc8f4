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

// Runs `t.steps` sweeps on one tile.  `buf` holds (th + 2H) * (tw + 2H) floats, twice that
// when t.steps > 1.
// `coef(idx)` returns the coefficient of canonical offset idx.  All threads of the block must
// call this; it ends with a __syncthreads().  COHERENT loads the input through L2 only.
// VX: consecutive cells per lane and pass (1 suits narrow regions, 4 reuses each window row
// for four outputs).
template <typename T, int SHAPE, int R, bool COHERENT = false, int VX = 1, typename Coef>
__device__ __forceinline__ void fused2d_tile(const T *__restrict__ in, T *__restrict__ out,
                                             const Fused2DTile &t, float *buf, const Coef &coef) {
    using OT = OffsetTable<2, SHAPE, R>;
    const int H = R * t.steps;
    const int W = t.tw + 2 * H;
    const int Hh = t.th + 2 * H;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const bool periodic = t.periodic != 0;
    const int gx0 = t.x0 - H, gy0 = t.y0 - H;  // grid position of region cell (0, 0)
    const bool x_in = gx0 >= 0 && gx0 + W <= t.nx;  // every column of the region is in the grid
    float *src = buf, *dst = buf + W * Hh;  // dst is used only when steps > 1

    // Load the tile with its halo (zero outside a Dirichlet grid), one warp per row: every lane
    // issues its four loads of a 128-column block before it stores any of them.
    for (int r = warp; r < Hh; r += nwarps) {
        bool rok = true;
        const int gy = wrap_or_flag(gy0 + r, t.ny, periodic, rok);
        float *srow = src + r * W;
        const T *grow = in + (size_t)gy * t.nx;
        for (int cb = 0; cb < W; cb += 128) {
            float v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = cb + lane + 32 * k;
                v[k] = 0.0f;
                if (rok && c < W) {
                    if (x_in) {
                        const T *a = grow + gx0 + c;
                        v[k] = Storage<T>::to_float(COHERENT ? load_l2(a) : *a);
                    } else {
                        bool ok = true;
                        const int gx = wrap_or_flag(gx0 + c, t.nx, periodic, ok);
                        const T *a = grow + gx;
                        if (ok) v[k] = Storage<T>::to_float(COHERENT ? load_l2(a) : *a);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = cb + lane + 32 * k;
                if (c < W) srow[c] = v[k];
            }
        }
    }
    __syncthreads();

    for (int s = 1; s <= t.steps; ++s) {
        const int g = R * s;  // border of the region not recomputed at this step
        const int r1 = Hh - g, c1 = W - g;
        const bool last = (s == t.steps);
        for (int r = g + warp; r < r1; r += nwarps) {
            const int gy = gy0 + r;
            const bool row_out = !periodic && (gy < 0 || gy >= t.ny);
            for (int cb = g + lane * VX; cb < c1; cb += 32 * VX) {
                float v[VX];
#pragma unroll
                for (int i = 0; i < VX; ++i) v[i] = 0.0f;
                const bool full = cb + VX + R <= W;  // the whole window lies in this row
                static_for<2 * R + 1>([&](auto dyi) {
                    constexpr int dy = decltype(dyi)::value - R;
                    constexpr int m = OT::tab.mdx[R][dy + R];
                    if constexpr (m >= 0) {
                        const float *wrow = src + (r + dy) * W + cb;
                        float win[VX + 2 * R];
#pragma unroll
                        for (int i = -m; i < VX + m; ++i)
                            win[i + R] = (full || cb + i < W) ? wrow[i] : 0.0f;
                        static_for<2 * R + 1>([&](auto dxi) {
                            constexpr int dx = decltype(dxi)::value - R;
                            constexpr int idx = OT::index(0, dy, dx);
                            if constexpr (idx >= 0) {
                                const float c = coef(idx);
#pragma unroll
                                for (int i = 0; i < VX; ++i) v[i] = fmaf(c, win[i + dx + R], v[i]);
                            }
                        });
                    }
                });
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    const int col = cb + i;
                    if (col >= c1) break;
                    const int gx = gx0 + col;
                    if (last) {
                        // the last step's region is exactly the output tile (inside the grid)
                        out[(size_t)gy * t.nx + gx] = Storage<T>::from_float(v[i]);
                    } else {
                        const bool out_of_grid = row_out || (!periodic && !x_in &&
                                                             (gx < 0 || gx >= t.nx));
                        dst[r * W + col] = out_of_grid ? 0.0f : round_to_storage<T>(v[i]);
                    }
                }
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

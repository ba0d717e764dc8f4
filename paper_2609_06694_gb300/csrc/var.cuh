// Variable-coefficient sweeps (ForgeStencil Sec. 2.1: coefficients that vary in space are one
// more array per offset):
//   forward   out[p] = sum_o w_o[p]   * in[p + o]
//   adjoint   out[q] = sum_o w_o[q-o] * in[q - o]      (offset flipped, coefficient gathered
//                                                      at the shifted cell)
//   div(k grad u), unit spacing, conservative star-1 form with face k = mean of the two cells.
//
// Design: a CTA owns a 128-cell x TY tile and walks z, one output plane at a time with a
// single FP32 accumulator per cell.
//  * general VAR sweeps: the 2R+1 input planes an output plane needs (plus one in flight) sit
//    in a ring of shared-memory slots filled by all threads with 16-byte cp.async (zero fill
//    = Dirichlet ghosts, wrapped addresses = periodic); coefficient arrays are read straight
//    from global memory (each value is used once, so staging would not save traffic).
//  * div(k grad u): the warp-specialised plane ring of ring.cuh (a producer warp
//    tensor-copies the u and k tiles of each plane into one slot); consumer warps hold the
//    window z-1, z, z+1 and release plane z-1 once output z is computed.
#pragma once

#include "common.cuh"
#include "ring.cuh"
#include "stream.cuh"

namespace gst {

constexpr int kMaxVarPts = 27;  // coefficient arrays per VAR plan (3D box r1 has 27)

template <typename T> struct VarParams {
    const T *in;
    T *out;
    const T *w[kMaxVarPts];  // VAR: one array per offset (canonical order); DIVKGRAD: w[0] = k
    int nx, ny, nz;
    int periodic;
    int aligned;
    int tiles_x, tiles_y, zchunk;
};

// Copies one plane tile (rows y0-R .. y0+TY+R-1, 16-byte chunks x0-A .. x0+TX+A-1) into a
// shared-memory slot: cp.async when rows are 16-byte aligned, element loads otherwise.
template <typename T, int R, int A, int PITCH>
__device__ __forceinline__ void load_tile_plane(const T *__restrict__ field, T *slot_smem, int zi,
                                                int nx, int ny, int nz, bool periodic,
                                                bool aligned, int x0, int y0, int rows, int tid,
                                                int nthr, bool is3d) {
    bool zok = true;
    const int gz = is3d ? wrap_or_flag(zi, nz, periodic, zok) : 0;
    const T *plane = field + (size_t)gz * nx * ny;
    constexpr int CPR = PITCH / A;
    if (aligned) {
        const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(slot_smem));
        const int nchunks = CPR * rows;
        for (int c = tid; c < nchunks; c += nthr) {
            const int row = c / CPR, cc = c - row * CPR;
            bool ok = zok;
            const int gy = wrap_or_flag(y0 - R + row, ny, periodic, ok);
            const int gx = wrap_or_flag(x0 - A + cc * A, nx, periodic, ok);
            const T *src = ok ? plane + (size_t)gy * nx + gx : field;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sbase + c * 16),
                         "l"(src), "r"(ok ? 16 : 0)
                         : "memory");
        }
    } else {
        const int wcols = PITCH - 2 * A + 2 * R;
        const int n = wcols * rows;
        for (int e = tid; e < n; e += nthr) {
            const int row = e / wcols, col = e - row * wcols;
            bool ok = zok;
            const int gy = wrap_or_flag(y0 - R + row, ny, periodic, ok);
            const int gx = wrap_or_flag(x0 - R + col, nx, periodic, ok);
            slot_smem[row * PITCH + (A - R) + col] =
                ok ? plane[(size_t)gy * nx + gx] : Storage<T>::from_float(0.0f);
        }
    }
}

// The same copy with per-thread chunk addresses computed once per tile (the first KMAX chunks
// of every thread; any further chunks are addressed on the fly).  `load` works for any field
// of the grid's shape.
template <typename T, int R, int A, int PITCH> struct TileLoader {
    static constexpr int KMAX = 4;
    static constexpr int CPR = PITCH / A;
    uint32_t dst[KMAX];
    int src[KMAX];  // in-plane element offset, -1 = zero fill
    int nk, nchunks, x0, y0, nx, ny, nz, rows, tid, nthr;
    bool periodic, aligned, is3d;

    __device__ __forceinline__ void init(int x0_, int y0_, int rows_, int nx_, int ny_, int nz_,
                                         bool periodic_, bool aligned_, bool is3d_, int tid_,
                                         int nthr_) {
        x0 = x0_; y0 = y0_; rows = rows_; nx = nx_; ny = ny_; nz = nz_;
        periodic = periodic_; aligned = aligned_; is3d = is3d_; tid = tid_; nthr = nthr_;
        nchunks = CPR * rows;
        nk = 0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int c = tid + k * nthr;
            dst[k] = 0;
            src[k] = -1;
            if (c < nchunks) {
                const int row = c / CPR, cc = c - row * CPR;
                bool ok = true;
                const int gy = wrap_or_flag(y0 - R + row, ny, periodic, ok);
                const int gx = wrap_or_flag(x0 - A + cc * A, nx, periodic, ok);
                dst[k] = (uint32_t)(c * 16);
                src[k] = ok ? gy * nx + gx : -1;
                nk = k + 1;
            }
        }
    }
    __device__ __forceinline__ void load(const T *__restrict__ field, T *slot_smem, int zi) const {
        if (!aligned) {
            load_tile_plane<T, R, A, PITCH>(field, slot_smem, zi, nx, ny, nz, periodic, false, x0,
                                            y0, rows, tid, nthr, is3d);
            return;
        }
        bool zok = true;
        const int gz = is3d ? wrap_or_flag(zi, nz, periodic, zok) : 0;
        const T *plane = field + (size_t)gz * nx * ny;
        const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(slot_smem));
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < nk) {
                const bool ok = zok && src[k] >= 0;
                cp_async16_u32(sbase + dst[k], ok ? (const void *)(plane + src[k]) : field,
                               ok ? 16 : 0);
            }
        }
        for (int c = tid + KMAX * nthr; c < nchunks; c += nthr) {
            const int row = c / CPR, cc = c - row * CPR;
            bool ok = zok;
            const int gy = wrap_or_flag(y0 - R + row, ny, periodic, ok);
            const int gx = wrap_or_flag(x0 - A + cc * A, nx, periodic, ok);
            cp_async16_u32(sbase + (uint32_t)(c * 16),
                           ok ? (const void *)(plane + (size_t)gy * nx + gx) : field, ok ? 16 : 0);
        }
    }
};

// VX consecutive values of a global array as floats (vector load when allowed).
template <typename T, int VX>
__device__ __forceinline__ void load_cells(const T *__restrict__ src, bool vec, int nvalid,
                                           float (&v)[VX]) {
    if (vec) {
        uint4 raw = __ldg(reinterpret_cast<const uint4 *>(src));
        const T *e = reinterpret_cast<const T *>(&raw);
#pragma unroll
        for (int i = 0; i < VX; ++i) v[i] = Storage<T>::to_float(e[i]);
    } else {
#pragma unroll
        for (int i = 0; i < VX; ++i) v[i] = i < nvalid ? Storage<T>::to_float(src[i]) : 0.0f;
    }
}

template <typename T, int VX>
__device__ __forceinline__ void store_cells(T *dst, bool vec, int nvalid, const float (&v)[VX]) {
    if (vec) {
        T tmp[VX];
#pragma unroll
        for (int i = 0; i < VX; ++i) tmp[i] = Storage<T>::from_float(v[i]);
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(tmp);
    } else {
#pragma unroll
        for (int i = 0; i < VX; ++i)
            if (i < nvalid) dst[i] = Storage<T>::from_float(v[i]);
    }
}

// ---------------------------------------------------------------------------------------
// General variable-coefficient sweep (forward or adjoint)
// ---------------------------------------------------------------------------------------
template <typename T, int NDIM, int SHAPE, int R, bool ADJ>
__global__ void __launch_bounds__(256) var_sweep_kernel(const __grid_constant__ VarParams<T> p) {
    constexpr int VX = 16 / (int)sizeof(T), A = VX, TX = 128, BX = TX / VX;
    constexpr int PITCH = TX + 2 * A;
    constexpr int RZ = NDIM == 3 ? R : 0;
    constexpr int NSLOT = 2 * RZ + 2;  // planes zo-RZ .. zo+RZ plus one in flight
    using OT = OffsetTable<NDIM, SHAPE, R>;
    static_assert(OT::count <= kMaxVarPts, "too many coefficient arrays");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int by = blockDim.y, tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * BX + tx, nthr = BX * by;
    const int TY = by;  // one row per thread
    const int rows = TY + 2 * R;
    const int plane_elems = PITCH * rows;
    int b = blockIdx.x;
    const int tix = b % p.tiles_x;
    b /= p.tiles_x;
    const int tiy = b % p.tiles_y, tiz = b / p.tiles_y;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int x0 = tix * TX, y0 = tiy * TY;
    const int z_begin = NDIM == 3 ? tiz * p.zchunk : 0;
    const int z_end = NDIM == 3 ? min(nz, z_begin + p.zchunk) : 1;
    const bool periodic = p.periodic != 0, aligned = p.aligned != 0;
    const size_t pstride = (size_t)nx * ny;
    const int ox = x0 + tx * VX, oy = y0 + ty;
    const bool vec = aligned && ox + VX <= nx;
    const int nvalid = nx - ox;

    TileLoader<T, R, A, PITCH> loader;
    loader.init(x0, y0, rows, nx, ny, nz, periodic, aligned, NDIM == 3, tid, nthr);
    auto load = [&](int zi) {
        const int slot = ((zi - z_begin + RZ) % NSLOT + NSLOT) % NSLOT;
        loader.load(p.in, smem + slot * plane_elems, zi);
    };
    // prologue: planes z_begin-RZ .. z_begin+RZ
    for (int zi = z_begin - RZ; zi <= z_begin + RZ; ++zi) {
        load(zi);
        cp_async_commit();
    }
    const bool row_ok = oy < ny;
    // the coefficients output cell(s) of plane zo take for offset (dz, dy, dx): forward at the
    // output cell, adjoint at the shifted source cell q - o (wrapped; a source outside a
    // Dirichlet grid reads 0 from the tile anyway)
    auto fetch_w = [&](int zo, int idx, int dz, int dy, int dx, float (&w)[VX]) {
        if (!row_ok) {
#pragma unroll
            for (int i = 0; i < VX; ++i) w[i] = 0.0f;
        } else if constexpr (!ADJ) {
            load_cells<T, VX>(p.w[idx] + (size_t)zo * pstride + (size_t)oy * nx + ox, vec, nvalid,
                              w);
        } else {
            bool ok = true;
            const int gz = NDIM == 3 ? wrap_or_flag(zo - dz, nz, true, ok) : 0;
            const int gy = wrap_or_flag(oy - dy, ny, true, ok);
            const T *base = p.w[idx] + (size_t)gz * pstride + (size_t)gy * nx;
            if (dx == 0) {
                // no shift along x: the thread's cells of the source row, one vector
                load_cells<T, VX>(base + ox, vec, nvalid, w);
            } else {
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    bool okx = true;
                    const int gx = wrap_or_flag(ox + i - dx, nx, true, okx);
                    w[i] = Storage<T>::to_float(__ldg(base + gx));
                }
            }
        }
    };
    // The first NPRE offsets (at most 32 values per thread) fetch their coefficients of the
    // plane into registers before the wait for the input planes, so those global loads are in
    // flight during the wait and barrier; the rest load where they are used.  The adjoint's
    // gathers take part only when every offset fits (a partial set of gathered coefficients
    // cost more in registers than it saved: 2x slower for the bf16 box).
    constexpr int NPRE = OT::count * VX <= 32 ? OT::count : (ADJ ? 0 : 32 / VX);
    float wpre[NPRE > 0 ? NPRE : 1][VX];
    for (int zo = z_begin; zo < z_end; ++zo) {
        // plane zo+RZ+1 goes into the slot freed by plane zo-RZ-1
        if (zo + RZ + 1 < z_end + RZ) load(zo + RZ + 1);
        cp_async_commit();
        {
            static_for<2 * RZ + 1>([&](auto dzi_c) {
                static_for<2 * R + 1>([&](auto dyi_c) {
                    static_for<2 * R + 1>([&](auto dxi_c) {
                        constexpr int dz = decltype(dzi_c)::value - RZ;
                        constexpr int dy = decltype(dyi_c)::value - R;
                        constexpr int dx = decltype(dxi_c)::value - R;
                        constexpr int idx = OT::index(dz, dy, dx);
                        if constexpr (idx >= 0 && idx < NPRE)
                            fetch_w(zo, idx, dz, dy, dx, wpre[idx]);
                    });
                });
            });
        }
        cp_async_wait<1>();
        __syncthreads();
        float acc[VX];
#pragma unroll
        for (int i = 0; i < VX; ++i) acc[i] = 0.0f;
        static_for<2 * RZ + 1>([&](auto dzi_c) {
            constexpr int dz = decltype(dzi_c)::value - RZ;
            // forward reads plane zo+dz at rows/cols +d; the adjoint reads plane zo-dz at -d
            const int zsrc = ADJ ? zo - dz : zo + dz;
            const int slot = ((zsrc - z_begin + RZ) % NSLOT + NSLOT) % NSLOT;
            const T *sp = smem + slot * plane_elems;
            static_for<2 * R + 1>([&](auto dyi_c) {
                constexpr int dy = decltype(dyi_c)::value - R;
                constexpr int m = OT::tab.mdx[dz + R][dy + R];
                if constexpr (m >= 0) {
                    constexpr int ry = ADJ ? -dy : dy;
                    float win[VX + 2 * R];
                    load_span<T, -m, VX + m, -R>(sp + (ty + R + ry) * PITCH + A + tx * VX, win);
                    static_for<2 * R + 1>([&](auto dxi_c) {
                        constexpr int dx = decltype(dxi_c)::value - R;
                        constexpr int idx = OT::index(dz, dy, dx);
                        if constexpr (idx >= 0) {
                            constexpr int rx = ADJ ? -dx : dx;
                            if constexpr (idx < NPRE) {
#pragma unroll
                                for (int i = 0; i < VX; ++i)
                                    acc[i] = fmaf(wpre[idx][i], win[i + rx + R], acc[i]);
                            } else {
                                float w[VX];
                                fetch_w(zo, idx, dz, dy, dx, w);
#pragma unroll
                                for (int i = 0; i < VX; ++i)
                                    acc[i] = fmaf(w[i], win[i + rx + R], acc[i]);
                            }
                        }
                    });
                }
            });
        });
        if (row_ok && ox < nx)
            store_cells<T, VX>(p.out + (size_t)zo * pstride + (size_t)oy * nx + ox, vec, nvalid,
                               acc);
        __syncthreads();  // the slot of plane zo-RZ is refilled next iteration
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------------
// div(k grad u) on the plane ring (ring.cuh): the producer warp tensor-copies the u and k
// tiles of each plane into one slot (two fields); every consumer warp holds a window of the
// 2RZ+1 planes z-1, z, z+1, writes output plane z and releases plane z-1.
// ---------------------------------------------------------------------------------------
template <typename T> struct DivkParams {
    CUtensorMap tmap[2];  // u, k (valid when use_tma)
    const T *field[2];    // u, k
    T *out;
    int nx, ny, nz;
    int periodic, aligned, use_tma;
    int tiles_x, tiles_y, work, nstage;
    int *err;                    // device status word (may be null)
    unsigned long long wait_ns;  // bound on the ring's waits (0: default)
    int phantom;                 // fault injection only (see StreamParams)
};

// VY: output rows per consumer thread (1 or 2); two rows share one plane's wait, release and
// slot addressing, and the y face between them reads rows the thread loads anyway.
template <typename T, int NDIM, int VY = 1> struct DivkKernel {
    static constexpr int VX = 16 / (int)sizeof(T), A = VX, TX = 128, BX = TX / VX, R = 1;
    static constexpr int PITCH = TX + 2 * A;
    static constexpr int RZ = NDIM == 3 ? 1 : 0;
    static constexpr int MAX_THREADS = 224;  // consumers; the CTA adds the producer warp
    __host__ __device__ static constexpr uint32_t field_bytes(int by) {
        return RingLayout::field_size(PITCH, by * VY + 2 * R, (int)sizeof(T));
    }
    static size_t smem_bytes(int by, int nstage) {
        return RingLayout::bytes(2 * field_bytes(by), nstage);
    }
};

template <typename T, int NDIM, int VY>
__global__ void __launch_bounds__(DivkKernel<T, NDIM, VY>::MAX_THREADS + 32)
    divkgrad_kernel(const __grid_constant__ DivkParams<T> p) {
    using K = DivkKernel<T, NDIM, VY>;
    constexpr int VX = K::VX, A = K::A, TX = K::TX, BX = K::BX, R = 1, PITCH = K::PITCH;
    constexpr int RZ = K::RZ;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // blockDim = (BX, by + 32 / BX): by rows of consumer threads (VY output rows each), then
    // the producer warp
    const int by = (int)blockDim.y - 32 / BX;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * BX + tx, ncons = BX * by, lane = tid & 31;
    const int TY = by * VY, rows = TY + 2 * R;
    Ring g;
    g.setup(smem_raw, K::field_bytes(by), 2, p.nstage, p.wait_ns);
    if (tid == 0) g.init(ncons / 32, p.phantom);
    __syncthreads();  // the only CTA-wide barrier
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool periodic = p.periodic != 0, aligned = p.aligned != 0;
    RingWork wk;
    wk.setup(p.tiles_x, p.tiles_y, NDIM == 3 ? nz : 1, p.work, TX, TY, RZ);

    if (tid >= ncons) {
        RingSource<T, 2> src;
        src.tmap = p.tmap;
        src.field = p.field;
        src.nx = nx;
        src.ny = ny;
        src.nz = nz;
        src.periodic = periodic;
        src.aligned = aligned;
        src.use_tma = p.use_tma != 0;
        src.rows = rows;
        ring_produce<T, 2, NDIM, R, A, PITCH, TX>(g, src, wk, p.err, lane);
        return;
    }

    const size_t pstride = (size_t)nx * ny;
    const int off = (ty * VY + R) * PITCH + A + tx * VX;  // the thread's first cell in a field
    const uint32_t kofs = g.field_bytes / sizeof(T);  // k field, in elements after u
    RingPos wpos, rpos;  // next plane to wait for / to release
    bool failed = false;
    auto wait_plane = [&]() -> bool {
        if (!g.wait_full(wpos.slot, wpos.phase)) return false;
        wpos.advance(g.ns);
        return true;
    };
    auto release_plane = [&]() {
        g.release(rpos.slot, lane);
        rpos.advance(g.ns);
    };

    for (long long w = wk.w_first; w < wk.w_end && !failed;) {
        const RingPiece q = wk.piece_at(w);
        w += q.z_end - q.z_begin;
        const int ox = q.x0 + tx * VX, oy0 = q.y0 + ty * VY;
        const bool vec = aligned && ox + VX <= nx;
        const int nvalid = nx - ox;
        // prologue: planes z_begin - RZ .. z_begin + RZ - 1
        for (int k = 0; k < 2 * RZ && !failed; ++k) failed = !wait_plane();
        for (int zo = q.z_begin; zo < q.z_end && !failed; ++zo) {
            if (!wait_plane()) {  // plane zo + RZ
                failed = true;
                break;
            }
            // slots of planes zo - 1, zo, zo + 1 (wpos is one past zo + RZ)
            int s0 = wpos.slot - 1 - RZ;
            if (s0 < 0) s0 += g.ns;
            const T *su = reinterpret_cast<const T *>(g.slot_ptr(s0));
            float acc2[VY][VX];
#pragma unroll
            for (int v = 0; v < VY; ++v)
#pragma unroll
                for (int i = 0; i < VX; ++i) acc2[v][i] = 0.0f;
#pragma unroll
            for (int v = 0; v < VY; ++v) {
                const int oy = oy0 + v;
                float(&acc)[VX] = acc2[v];
                const bool active = oy < ny && ox < nx;
                if (active) {
                    const int i0 = off + v * PITCH;
                    float u0[VX + 2], k0[VX + 2];  // centre row with one cell each side
                    load_span<T, -1, VX + 1, -1>(su + i0, u0);
                    load_span<T, -1, VX + 1, -1>(su + kofs + i0, k0);
                    // Each face adds (k_c + k_n) (u_n - u_c); the sum is halved at the end (exact,
                    // so this equals the half-face form bit for bit).  A neighbour outside a
                    // Dirichlet grid has u = 0 and k = k_c (see the ghost-face term below).
                    // ALLIN: no face needs a select (the only form used: the ghost faces are
                    // completed afterwards).
                    auto compute = [&](auto allin_c) {
                        constexpr bool ALLIN = decltype(allin_c)::value;
                        auto face = [&](int i, float un, float kn, bool inside) {
                            const float kc = k0[i + 1];
                            const bool in = ALLIN || inside;
                            const float ssum = kc + (in ? kn : kc);
                            const float d = (in ? un : 0.0f) - u0[i + 1];
                            acc[i] = fmaf(ssum, d, acc[i]);
                        };
                        // axes in the oracle's order: z, y, x; within an axis the + face, then -
                        if constexpr (NDIM == 3) {
                            const int sp = s0 + 1 == g.ns ? 0 : s0 + 1;
                            const int sm = s0 == 0 ? g.ns - 1 : s0 - 1;
                            const T *up_ = reinterpret_cast<const T *>(g.slot_ptr(sp)) + i0;
                            const T *um_ = reinterpret_cast<const T *>(g.slot_ptr(sm)) + i0;
                            float up[VX], kp[VX], um[VX], km[VX];
                            load_span<T, 0, VX, 0>(up_, up);
                            load_span<T, 0, VX, 0>(up_ + kofs, kp);
                            load_span<T, 0, VX, 0>(um_, um);
                            load_span<T, 0, VX, 0>(um_ + kofs, km);
                            const bool inp = periodic || zo + 1 < nz, inm = periodic || zo - 1 >= 0;
#pragma unroll
                            for (int i = 0; i < VX; ++i) {
                                face(i, up[i], kp[i], inp);
                                face(i, um[i], km[i], inm);
                            }
                        }
                        {
                            float up[VX], kp[VX], um[VX], km[VX];
                            load_span<T, 0, VX, 0>(su + i0 + PITCH, up);
                            load_span<T, 0, VX, 0>(su + kofs + i0 + PITCH, kp);
                            load_span<T, 0, VX, 0>(su + i0 - PITCH, um);
                            load_span<T, 0, VX, 0>(su + kofs + i0 - PITCH, km);
                            const bool inp = periodic || oy + 1 < ny, inm = periodic || oy - 1 >= 0;
#pragma unroll
                            for (int i = 0; i < VX; ++i) {
                                face(i, up[i], kp[i], inp);
                                face(i, um[i], km[i], inm);
                            }
                        }
#pragma unroll
                        for (int i = 0; i < VX; ++i) {
                            const bool inp = periodic || ox + i + 1 < nx;
                            const bool inm = periodic || ox + i - 1 >= 0;
                            face(i, u0[i + 2], k0[i + 2], inp);
                            face(i, u0[i], k0[i], inm);
                        }
                    };
                    // Every face is taken as if both cells were inside the grid: the ring
                    // zero-fills whatever lies outside a Dirichlet grid, so a face towards a
                    // ghost comes out as (k_c + 0) (0 - u_c), half its value (k_c + k_c)(0 - u_c).
                    // The missing half, -k_c u_c per ghost face, is added afterwards for the
                    // cells at the grid's faces; interior rows skip it.
                    compute(std::true_type{});
                    if (!periodic) {
                        const int byz = (oy == 0) + (oy == ny - 1) +
                                        (NDIM == 3 ? (zo == 0) + (zo == nz - 1) : 0);
                        if (byz != 0 || ox == 0 || ox + VX >= nx) {
#pragma unroll
                            for (int i = 0; i < VX; ++i) {
                                const int b = byz + (ox + i == 0) + (ox + i == nx - 1);
                                acc[i] = fmaf(-(float)b * k0[i + 1], u0[i + 1], acc[i]);
                            }
                        }
                    }
                }
            }  // rows of the thread
            release_plane();  // plane zo - RZ has been read for the last time (whole warp)
#pragma unroll
            for (int v = 0; v < VY; ++v) {
                const int oy = oy0 + v;
                if (oy < ny && ox < nx) {
#pragma unroll
                    for (int i = 0; i < VX; ++i) acc2[v][i] *= 0.5f;
                    store_cells<T, VX>(p.out + (size_t)zo * pstride + (size_t)oy * nx + ox, vec,
                                       nvalid, acc2[v]);
                }
            }
        }
        // the last 2RZ planes of the piece were only read as neighbours
        for (int k = 0; k < 2 * RZ && !failed; ++k) release_plane();
    }
    if (failed) g.fail(p.err, lane);
}

}  // namespace gst

// Streaming stencil sweep: one time step of out[p] = sum_o c_o in[p + o] (ForgeStencil
// Sec. 2.1) for star, box and diamond offset sets of radius R on a 2D or 3D grid.
//
// Design (sm_103a):
//  * A CTA owns an output tile of TX x TY cells (TX = blockDim.x * VX, TY = blockDim.y * VY)
//    and, in 3D, a chunk of z-planes that it walks from low to high z.
//  * Input planes (tile plus an R-cell halo in y and one 16-byte chunk of halo in x) are
//    copied into a ring of NSTAGE shared-memory slots with 16-byte cp.async; zero-fill
//    (src-size 0) gives the Dirichlet ghosts, wrapped source addresses give the periodic
//    ones.  Plane z+NSTAGE-1 is in flight while plane z is consumed.
//  * Each plane contributes to the 2R+1 output planes it touches: every thread keeps, per owned
//    cell, a queue of 2R+1 FP32 partial sums in registers, adds the 2D slice of the offset set
//    that lies at each dz, and writes the oldest sum once the plane R above it has arrived.
//    A star therefore reads its z-neighbours from registers and only the in-plane cross from
//    shared memory; a box or diamond reuses every shared-memory read for 2R+1 outputs.
//  * In-plane neighbours come from shared memory as 16-byte vectors: a thread's VX cells are
//    contiguous in x, so one row of its window (VX + 2m values) is a few aligned loads.
//  * 2D grids use the same kernel with no z-radius (one plane per CTA).
#pragma once

#include <utility>

#include "common.cuh"

namespace gst {

template <int N, typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F> __device__ __forceinline__ void static_for(F &&f) {
    static_for_impl<N>(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------------------
// Loads of a compile-time element range [LO, HI) from a 16-byte-aligned shared-memory base,
// converted to float into dst[(e - LO0)] where LO0 is the window origin.
// ---------------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ void unpack(uint32_t bits, float *d, int n) {
    if constexpr (sizeof(T) == 4) {
        d[0] = __uint_as_float(bits);
    } else {
        T lo, hi;
        uint16_t l = (uint16_t)(bits & 0xFFFFu), h = (uint16_t)(bits >> 16);
        memcpy(&lo, &l, 2);
        memcpy(&hi, &h, 2);
        d[0] = Storage<T>::to_float(lo);
        if (n > 1) d[1] = Storage<T>::to_float(hi);
    }
}

template <typename T, int POS, int HI, int ORIGIN>
__device__ __forceinline__ void load_span(const T *base, float *dst) {
    if constexpr (POS < HI) {
        constexpr int ES = (int)sizeof(T);
        constexpr int BOFF = POS * ES;
        constexpr int REM = (HI - POS) * ES;
        constexpr int W = ((BOFF & 15) == 0 && REM >= 16)  ? 16
                          : ((BOFF & 7) == 0 && REM >= 8)  ? 8
                          : ((BOFF & 3) == 0 && REM >= 4)  ? 4
                                                           : ES;
        constexpr int NE = W / ES;
        const T *src = base + POS;
        float *d = dst + (POS - ORIGIN);
        if constexpr (W == 16) {
            uint4 v = *reinterpret_cast<const uint4 *>(src);
            if constexpr (ES == 4) {
                d[0] = __uint_as_float(v.x); d[1] = __uint_as_float(v.y);
                d[2] = __uint_as_float(v.z); d[3] = __uint_as_float(v.w);
            } else {
                unpack<T>(v.x, d + 0, 2); unpack<T>(v.y, d + 2, 2);
                unpack<T>(v.z, d + 4, 2); unpack<T>(v.w, d + 6, 2);
            }
        } else if constexpr (W == 8) {
            uint2 v = *reinterpret_cast<const uint2 *>(src);
            if constexpr (ES == 4) {
                d[0] = __uint_as_float(v.x); d[1] = __uint_as_float(v.y);
            } else {
                unpack<T>(v.x, d + 0, 2); unpack<T>(v.y, d + 2, 2);
            }
        } else if constexpr (W == 4) {
            uint32_t v = *reinterpret_cast<const uint32_t *>(src);
            unpack<T>(v, d, NE);
        } else {
            d[0] = Storage<T>::to_float(*src);
        }
        load_span<T, POS + NE, HI, ORIGIN>(base, dst);
    }
}

// ---------------------------------------------------------------------------------------
// Kernel parameters
// ---------------------------------------------------------------------------------------
template <int NPTS> struct ConstCoeffs {
    float c[NPTS];
};

template <typename T> struct StreamParams {
    const T *in;
    T *out;
    int nx, ny, nz;     // 2D grids: nz = 1
    int periodic;       // 1 = wrap, 0 = zero Dirichlet
    int aligned;        // 1 = 16-byte cp.async loader and vector stores are legal
    int tiles_x, tiles_y;
    int zchunk;         // planes per CTA (3D)
    int kchunks;        // cp.async chunks per thread per plane (aligned loader)
    int *err;           // device error word (may be null)
};

// Ordinary output: round to the storage type and store.
struct PlainStore {};

// ---------------------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------------------
template <typename T, int NDIM, int SHAPE, int R, int VX, int VY, int NSTAGE, bool UNROLLZ>
struct StreamKernel {
    static constexpr int RZ = (NDIM == 3) ? R : 0;
    static constexpr int P = 2 * RZ + 1;
    static constexpr int A = 16 / (int)sizeof(T);  // x halo: one 16-byte chunk
    using OT = OffsetTable<NDIM, SHAPE, R>;
    static constexpr int NPTS = OT::count;
    static constexpr int KMAX = 4;                  // per-thread chunk slots (loader)
    static_assert(R <= A, "x halo must fit in one 16-byte chunk");
    static_assert((VX * (int)sizeof(T)) % 16 == 0, "VX cells must span whole 16-byte chunks");

    // needed |dx| for window row wr (union over the thread's rows and every dz); -1 = unused
    __host__ __device__ static constexpr int row_m(int wr) {
        int m = -1;
        for (int vy = 0; vy < VY; ++vy) {
            int dy = wr - R - vy;
            if (dy < -R || dy > R) continue;
            int v = OT::max_dx_any(dy);
            if (v > m) m = v;
        }
        return m;
    }

    static size_t smem_bytes(int bx, int by) {
        int pitch = bx * VX + 2 * A;
        int rows = by * VY + 2 * R;
        return (size_t)NSTAGE * pitch * rows * sizeof(T);
    }
};

template <typename T, int NDIM, int SHAPE, int R, int VX, int VY, int NSTAGE, bool UNROLLZ>
__global__ void __launch_bounds__(256)
    stream_sweep_kernel(const StreamParams<T> p,
                        const __grid_constant__ ConstCoeffs<OffsetTable<NDIM, SHAPE, R>::count> cf) {
    using K = StreamKernel<T, NDIM, SHAPE, R, VX, VY, NSTAGE, UNROLLZ>;
    constexpr int RZ = K::RZ, P = K::P, A = K::A;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);

    const int bx = blockDim.x, by = blockDim.y;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * bx + tx, nthr = bx * by;
    const int TX = bx * VX, TY = by * VY;
    const int pitch = TX + 2 * A;
    const int rows = TY + 2 * R;
    const int plane_elems = pitch * rows;

    int b = blockIdx.x;
    const int tix = b % p.tiles_x;
    b /= p.tiles_x;
    const int tiy = b % p.tiles_y;
    const int tiz = b / p.tiles_y;
    const int x0 = tix * TX, y0 = tiy * TY;
    const int z_begin = (NDIM == 3) ? tiz * p.zchunk : 0;
    const int z_end = (NDIM == 3) ? min(p.nz, z_begin + p.zchunk) : 1;
    const int zs = z_begin - RZ, zl = z_end + RZ;
    const bool periodic = p.periodic != 0;
    const size_t plane_stride = (size_t)p.nx * p.ny;

    // ---- per-thread loader slots (aligned path): smem offset and in-plane source offset ----
    const int cpr = pitch / A;
    const int nchunks = cpr * rows;
    int ld_dst[K::KMAX], ld_src[K::KMAX];
#pragma unroll
    for (int k = 0; k < K::KMAX; ++k) {
        int c = tid + k * nthr;
        ld_dst[k] = -1;
        ld_src[k] = -1;
        if (k < p.kchunks && c < nchunks) {
            int row = c / cpr, cc = c - row * cpr;
            bool ok = true;
            int gy = wrap_or_flag(y0 - R + row, p.ny, periodic, ok);
            int gx = wrap_or_flag(x0 - A + cc * A, p.nx, periodic, ok);
            ld_dst[k] = row * pitch + cc * A;
            ld_src[k] = ok ? gy * p.nx + gx : -1;
        }
    }

    auto load_plane = [&](int zi, int slot) {
        bool zok = true;
        int gz = (NDIM == 3) ? wrap_or_flag(zi, p.nz, periodic, zok) : 0;
        const T *plane = p.in + (size_t)gz * plane_stride;
        T *dst = smem + slot * plane_elems;
        if (p.aligned) {
#pragma unroll
            for (int k = 0; k < K::KMAX; ++k) {
                if (ld_dst[k] >= 0) {
                    bool ok = zok && ld_src[k] >= 0;
                    cp_async16(dst + ld_dst[k], ok ? (const void *)(plane + ld_src[k])
                                                   : (const void *)p.in,
                               ok ? 16 : 0);
                }
            }
        } else {
            // scalar path: only the cells the stencil reads (x0-R .. x0+TX+R)
            const int wcols = TX + 2 * R;
            const int n = wcols * rows;
            for (int e = tid; e < n; e += nthr) {
                int row = e / wcols, col = e - row * wcols;
                bool ok = zok;
                int gy = wrap_or_flag(y0 - R + row, p.ny, periodic, ok);
                int gx = wrap_or_flag(x0 - R + col, p.nx, periodic, ok);
                T v = ok ? plane[(size_t)gy * p.nx + gx] : Storage<T>::from_float(0.0f);
                dst[row * pitch + (A - R) + col] = v;
            }
        }
    };

    float acc[P][VY][VX];
#pragma unroll
    for (int j = 0; j < P; ++j)
#pragma unroll
        for (int vy = 0; vy < VY; ++vy)
#pragma unroll
            for (int vx = 0; vx < VX; ++vx) acc[j][vy][vx] = 0.0f;

    // prologue: planes zs .. zs+NSTAGE-2 in flight
#pragma unroll
    for (int k = 0; k < NSTAGE - 1; ++k) {
        if (zs + k < zl) load_plane(zs + k, k);
        cp_async_commit();
    }

    const int ox = x0 + tx * VX;  // first owned column
    const int oy = y0 + ty * VY;  // first owned row

    // accumulate the contributions of the plane in `slot` to the queued outputs; JOF(dz) is
    // the queue index of output (zi - dz)
    auto accumulate = [&](const T *plane_smem, auto jof) {
        const T *tbase = plane_smem + (ty * VY) * pitch + A + tx * VX;
        static_for<VY + 2 * R>([&](auto wr_c) {
            constexpr int wr = decltype(wr_c)::value;
            constexpr int m = K::row_m(wr);
            if constexpr (m >= 0) {
                float win[VX + 2 * R];
                load_span<T, -m, VX + m, -R>(tbase + wr * pitch, win);
                static_for<VY>([&](auto vy_c) {
                    constexpr int vy = decltype(vy_c)::value;
                    constexpr int dy = wr - R - vy;
                    if constexpr (dy >= -R && dy <= R) {
                        static_for<P>([&](auto dzi_c) {
                            constexpr int dz = decltype(dzi_c)::value - RZ;
                            constexpr int j = decltype(jof(std::integral_constant<int, dz>{}))::value;
                            static_for<2 * R + 1>([&](auto dxi_c) {
                                constexpr int dx = decltype(dxi_c)::value - R;
                                constexpr int idx = K::OT::index(dz, dy, dx);
                                if constexpr (idx >= 0) {
                                    const float c = cf.c[idx];
#pragma unroll
                                    for (int vx = 0; vx < VX; ++vx)
                                        acc[j][vy][vx] = fmaf(c, win[vx + dx + R], acc[j][vy][vx]);
                                }
                            });
                        });
                    }
                });
            }
        });
    };

    auto store_output = [&](int zo, float (&vals)[VY][VX]) {
        if (zo < z_begin || zo >= z_end) return;
        T *orow0 = p.out + (size_t)zo * plane_stride;
#pragma unroll
        for (int vy = 0; vy < VY; ++vy) {
            const int y = oy + vy;
            if (y >= p.ny) continue;
            T *dst = orow0 + (size_t)y * p.nx + ox;
            if (p.aligned && ox + VX <= p.nx) {
                T tmp[VX];
#pragma unroll
                for (int vx = 0; vx < VX; ++vx) tmp[vx] = Storage<T>::from_float(vals[vy][vx]);
#pragma unroll
                for (int q = 0; q < (VX * (int)sizeof(T)) / 16; ++q)
                    reinterpret_cast<uint4 *>(dst)[q] = reinterpret_cast<const uint4 *>(tmp)[q];
            } else {
#pragma unroll
                for (int vx = 0; vx < VX; ++vx)
                    if (ox + vx < p.nx) dst[vx] = Storage<T>::from_float(vals[vy][vx]);
            }
        }
    };

    int zi = zs;
    int slot = 0;
    constexpr int PU = UNROLLZ ? P : 1;
    bool done = false;
    while (!done) {
        static_for<PU>([&](auto ph_c) {
            constexpr int ph = decltype(ph_c)::value;
            (void)ph;
            if (done) return;
            if (zi >= zl) {
                done = true;
                return;
            }
            cp_async_wait<NSTAGE - 2>();
            __syncthreads();
            {
                const int zn = zi + NSTAGE - 1;
                int sn = slot + NSTAGE - 1;
                if (sn >= NSTAGE) sn -= NSTAGE;
                if (zn < zl) load_plane(zn, sn);
                cp_async_commit();
            }
            const T *pl = smem + slot * plane_elems;
            if constexpr (UNROLLZ) {
                // queue index of output (zi - dz) is (ph - dz) mod P
                accumulate(pl, [](auto dz_c) {
                    constexpr int dz = decltype(dz_c)::value;
                    return std::integral_constant<int, imod_c(ph - dz, P)>{};
                });
                constexpr int jo = imod_c(ph - RZ, P);
                store_output(zi - RZ, acc[jo]);
#pragma unroll
                for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                    for (int vx = 0; vx < VX; ++vx) acc[jo][vy][vx] = 0.0f;
            } else {
                // queue index j holds output zi - RZ + j
                accumulate(pl, [](auto dz_c) {
                    constexpr int dz = decltype(dz_c)::value;
                    return std::integral_constant<int, RZ - dz>{};
                });
                store_output(zi - RZ, acc[0]);
#pragma unroll
                for (int j = 0; j + 1 < P; ++j)
#pragma unroll
                    for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                        for (int vx = 0; vx < VX; ++vx) acc[j][vy][vx] = acc[j + 1][vy][vx];
#pragma unroll
                for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                    for (int vx = 0; vx < VX; ++vx) acc[P - 1][vy][vx] = 0.0f;
            }
            ++zi;
            slot = (slot + 1 == NSTAGE) ? 0 : slot + 1;
        });
    }
    cp_async_wait<0>();
}

}  // namespace gst

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

// Calls f(integral_constant<k>) for the runtime value ph in [0, P), P <= 9, via a switch.
template <int P, typename F> __device__ __forceinline__ void phase_switch(int ph, F &&f) {
    static_assert(P <= 9, "phase_switch handles up to 9 phases");
    switch (ph) {
#define GST_PHASE_CASE(k)                                                 \
    case k:                                                               \
        if constexpr (k < P) f(std::integral_constant<int, k>{});         \
        break;
        GST_PHASE_CASE(0) GST_PHASE_CASE(1) GST_PHASE_CASE(2) GST_PHASE_CASE(3)
        GST_PHASE_CASE(4) GST_PHASE_CASE(5) GST_PHASE_CASE(6) GST_PHASE_CASE(7)
        GST_PHASE_CASE(8)
#undef GST_PHASE_CASE
    default: break;
    }
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

// How the partial-sum queue is indexed:
//  kQueueUnrolled : the z loop is unrolled by 2R+1 so every queue index is a constant;
//  kQueueRotate   : the queue is shifted by one entry after every plane (large stencils);
//  kQueueStarSplit: stars only -- the in-plane cross goes to a temporary, and a switch on
//                   the plane's phase adds it and the 2R single-point z terms to the queue.
enum QueueMode : int { kQueueUnrolled = 0, kQueueRotate = 1, kQueueStarSplit = 2 };

template <typename T, int NDIM, int SHAPE, int R, int VY, int NSTAGE, int QMODE>
struct StreamKernel {
    static constexpr int RZ = (NDIM == 3) ? R : 0;
    static constexpr int P = 2 * RZ + 1;
    static constexpr int VX = 16 / (int)sizeof(T);  // one 16-byte vector of cells per row
    static constexpr int A = VX;                     // x halo: one 16-byte chunk
    static constexpr int TX = 128;                   // tile width (cells)
    static constexpr int BX = TX / VX;               // threads along x
    static constexpr int PITCH = TX + 2 * A;         // shared-memory row length (elements)
    using OT = OffsetTable<NDIM, SHAPE, R>;
    static constexpr int NPTS = OT::count;
    static constexpr int KMAX = 4;                   // per-thread chunk slots (loader)
    static constexpr bool CREG = NPTS <= 32;         // coefficients held in registers
    static_assert(R <= A, "x halo must fit in one 16-byte chunk");
    static_assert(QMODE != kQueueStarSplit || SHAPE == kStar, "split mode is for stars");

    // needed |dx| for window row wr (union over the thread's rows and every dz); -1 = unused
    __host__ __device__ static constexpr int row_m(int wr, bool inplane_only) {
        int m = -1;
        for (int vy = 0; vy < VY; ++vy) {
            int dy = wr - R - vy;
            if (dy < -R || dy > R) continue;
            int v = inplane_only ? OT::tab.mdx[R][dy + R] : OT::max_dx_any(dy);
            if (v > m) m = v;
        }
        return m;
    }

    static size_t smem_bytes(int by) {
        return (size_t)NSTAGE * PITCH * (by * VY + 2 * R) * sizeof(T);
    }
};

template <typename T, int NDIM, int SHAPE, int R, int VY, int NSTAGE, int QMODE>
__global__ void __launch_bounds__(256)
    stream_sweep_kernel(const StreamParams<T> p,
                        const __grid_constant__ ConstCoeffs<OffsetTable<NDIM, SHAPE, R>::count> cf) {
    using K = StreamKernel<T, NDIM, SHAPE, R, VY, NSTAGE, QMODE>;
    constexpr int RZ = K::RZ, P = K::P, A = K::A, VX = K::VX, PITCH = K::PITCH, TX = K::TX;
    constexpr int ES = (int)sizeof(T);

    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);

    const int by = blockDim.y;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * K::BX + tx, nthr = K::BX * by;
    const int TY = by * VY;
    const int rows = TY + 2 * R;
    const int plane_elems = PITCH * rows;

    int b = blockIdx.x;
    const int tix = b % p.tiles_x;
    b /= p.tiles_x;
    const int tiy = b % p.tiles_y;
    const int tiz = b / p.tiles_y;
    const int nx = p.nx, ny = p.ny;
    const int x0 = tix * TX, y0 = tiy * TY;
    const int z_begin = (NDIM == 3) ? tiz * p.zchunk : 0;
    const int z_end = (NDIM == 3) ? min(p.nz, z_begin + p.zchunk) : 1;
    const int zs = z_begin - RZ, zl = z_end + RZ;
    const bool periodic = p.periodic != 0;
    const bool aligned = p.aligned != 0;
    const size_t plane_stride = (size_t)nx * ny;

    // coefficients: registers for small stencils, the parameter bank otherwise
    float creg[K::CREG ? K::NPTS : 1];
    if constexpr (K::CREG) {
#pragma unroll
        for (int i = 0; i < K::NPTS; ++i) creg[i] = cf.c[i];
    }
    auto coef = [&](auto idx_c) -> float {
        constexpr int idx = decltype(idx_c)::value;
        if constexpr (K::CREG) return creg[idx];
        else return cf.c[idx];
    };

    // ---- per-thread loader slots (aligned path): smem byte offset and in-plane source ----
    constexpr int CPR = PITCH / A;
    const int nchunks = CPR * rows;
    const uint32_t smem_u32 = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    uint32_t ld_dst[K::KMAX];
    int ld_src[K::KMAX];
    int nk = 0;
#pragma unroll
    for (int k = 0; k < K::KMAX; ++k) {
        const int c = tid + k * nthr;
        ld_dst[k] = 0;
        ld_src[k] = -1;
        if (c < nchunks) {
            const int row = c / CPR, cc = c - row * CPR;
            bool ok = true;
            const int gy = wrap_or_flag(y0 - R + row, ny, periodic, ok);
            const int gx = wrap_or_flag(x0 - A + cc * A, nx, periodic, ok);
            ld_dst[k] = (uint32_t)(c * 16);  // chunk c of the row-major tile is bytes 16c..
            ld_src[k] = ok ? gy * nx + gx : -1;
            nk = k + 1;
        }
    }

    auto load_plane = [&](int zi, int slot) {
        bool zok = true;
        const int gz = (NDIM == 3) ? wrap_or_flag(zi, p.nz, periodic, zok) : 0;
        const T *plane = p.in + (size_t)gz * plane_stride;
        if (aligned) {
            const uint32_t sbase = smem_u32 + (uint32_t)(slot * plane_elems * ES);
#pragma unroll
            for (int k = 0; k < K::KMAX; ++k) {
                if (k < nk) {
                    const bool ok = zok && ld_src[k] >= 0;
                    const T *src = ok ? plane + ld_src[k] : p.in;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                                     sbase + ld_dst[k]),
                                 "l"(src), "r"(ok ? 16 : 0)
                                 : "memory");
                }
            }
            // chunks beyond the register slots: address computed on the fly
            for (int c = tid + K::KMAX * nthr; c < nchunks; c += nthr) {
                const int row = c / CPR, cc = c - row * CPR;
                bool ok = zok;
                const int gy = wrap_or_flag(y0 - R + row, ny, periodic, ok);
                const int gx = wrap_or_flag(x0 - A + cc * A, nx, periodic, ok);
                const T *src = ok ? plane + gy * nx + gx : p.in;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                                 sbase + (uint32_t)(c * 16)),
                             "l"(src), "r"(ok ? 16 : 0)
                             : "memory");
            }
        } else {
            // scalar path: only the cells the stencil reads (x0-R .. x0+TX+R)
            T *dst = smem + slot * plane_elems;
            const int wcols = TX + 2 * R;
            const int n = wcols * rows;
            for (int e = tid; e < n; e += nthr) {
                const int row = e / wcols, col = e - row * wcols;
                bool ok = zok;
                const int gy = wrap_or_flag(y0 - R + row, ny, periodic, ok);
                const int gx = wrap_or_flag(x0 - R + col, nx, periodic, ok);
                const T v = ok ? plane[(size_t)gy * nx + gx] : Storage<T>::from_float(0.0f);
                dst[row * PITCH + (A - R) + col] = v;
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

    // output addressing, hoisted
    const int ox = x0 + tx * VX;
    const int oy = y0 + ty * VY;
    T *const obase = p.out + (size_t)oy * nx + ox;
    const bool xfull = aligned && (ox + VX <= nx);
    const int vy_valid = min(VY, ny - oy);  // may be <= 0
    const int thr_off = (ty * VY) * PITCH + A + tx * VX;  // element offset of the thread's base

    auto store_output = [&](int zo, const float (&vals)[VY][VX]) {
        if (zo < z_begin || zo >= z_end) return;
        T *orow = obase + (size_t)zo * plane_stride;
#pragma unroll
        for (int vy = 0; vy < VY; ++vy) {
            if (vy >= vy_valid) break;
            T *dst = orow + (size_t)vy * nx;
            if (xfull) {
                T tmp[VX];
#pragma unroll
                for (int vx = 0; vx < VX; ++vx) tmp[vx] = Storage<T>::from_float(vals[vy][vx]);
                *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(tmp);
            } else {
#pragma unroll
                for (int vx = 0; vx < VX; ++vx)
                    if (ox + vx < nx) dst[vx] = Storage<T>::from_float(vals[vy][vx]);
            }
        }
    };

    // add the in-plane slice(s) of the plane at `tb` to the queue; JOF(dz) = queue index of
    // output (zi - dz).  INPLANE_ONLY restricts to dz = 0 and writes into `tmp` instead.
    auto accumulate = [&](const T *tb, auto jof, auto inplane_only_c, float (&tmp)[VY][VX]) {
        constexpr bool IPO = decltype(inplane_only_c)::value;
        static_for<VY + 2 * R>([&](auto wr_c) {
            constexpr int wr = decltype(wr_c)::value;
            constexpr int m = K::row_m(wr, IPO);
            if constexpr (m >= 0) {
                float win[VX + 2 * R];
                load_span<T, -m, VX + m, -R>(tb + wr * PITCH, win);
                static_for<VY>([&](auto vy_c) {
                    constexpr int vy = decltype(vy_c)::value;
                    constexpr int dy = wr - R - vy;
                    if constexpr (dy >= -R && dy <= R) {
                        static_for<P>([&](auto dzi_c) {
                            constexpr int dz = decltype(dzi_c)::value - RZ;
                            if constexpr (!IPO || dz == 0) {
                                constexpr int j =
                                    decltype(jof(std::integral_constant<int, dz>{}))::value;
                                static_for<2 * R + 1>([&](auto dxi_c) {
                                    constexpr int dx = decltype(dxi_c)::value - R;
                                    constexpr int idx = K::OT::index(dz, dy, dx);
                                    if constexpr (idx >= 0) {
                                        const float c = coef(std::integral_constant<int, idx>{});
#pragma unroll
                                        for (int vx = 0; vx < VX; ++vx) {
                                            float &dst = IPO ? tmp[vy][vx] : acc[j][vy][vx];
                                            dst = fmaf(c, win[vx + dx + R], dst);
                                        }
                                    }
                                });
                            }
                        });
                    }
                });
            }
        });
    };

    auto zero_slot = [&](float (&a)[VY][VX]) {
#pragma unroll
        for (int vy = 0; vy < VY; ++vy)
#pragma unroll
            for (int vx = 0; vx < VX; ++vx) a[vy][vx] = 0.0f;
    };

    // one plane: wait for it, keep the ring full, consume it
    auto begin_plane = [&](int zi, int slot) -> const T * {
        cp_async_wait<NSTAGE - 2>();
        __syncthreads();
        const int zn = zi + NSTAGE - 1;
        int sn = slot + NSTAGE - 1;
        if (sn >= NSTAGE) sn -= NSTAGE;
        if (zn < zl) load_plane(zn, sn);
        cp_async_commit();
        return smem + slot * plane_elems + thr_off;
    };

    int zi = zs;
    int slot = 0;
    float dummy[VY][VX];
    if constexpr (QMODE == kQueueUnrolled) {
        bool done = false;
        while (!done) {
            static_for<P>([&](auto ph_c) {
                constexpr int ph = decltype(ph_c)::value;
                if (done) return;
                if (zi >= zl) {
                    done = true;
                    return;
                }
                const T *tb = begin_plane(zi, slot);
                accumulate(tb, [](auto dz_c) {
                    constexpr int dz = decltype(dz_c)::value;
                    return std::integral_constant<int, imod_c(ph - dz, P)>{};
                }, std::false_type{}, dummy);
                constexpr int jo = imod_c(ph - RZ, P);
                store_output(zi - RZ, acc[jo]);
                zero_slot(acc[jo]);
                ++zi;
                slot = (slot + 1 == NSTAGE) ? 0 : slot + 1;
            });
        }
    } else if constexpr (QMODE == kQueueRotate) {
        for (; zi < zl; ++zi) {
            const T *tb = begin_plane(zi, slot);
            accumulate(tb, [](auto dz_c) {
                constexpr int dz = decltype(dz_c)::value;
                return std::integral_constant<int, RZ - dz>{};
            }, std::false_type{}, dummy);
            store_output(zi - RZ, acc[0]);
#pragma unroll
            for (int j = 0; j + 1 < P; ++j)
#pragma unroll
                for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                    for (int vx = 0; vx < VX; ++vx) acc[j][vy][vx] = acc[j + 1][vy][vx];
            zero_slot(acc[P - 1]);
            slot = (slot + 1 == NSTAGE) ? 0 : slot + 1;
        }
    } else {
        // star split: in-plane cross into tmp, then a phase switch for the z line
        int ph = 0;
        for (; zi < zl; ++zi) {
            const T *tb = begin_plane(zi, slot);
            float tmp[VY][VX];
            zero_slot(tmp);
            accumulate(tb, [](auto) { return std::integral_constant<int, 0>{}; },
                       std::true_type{}, tmp);
            // centre values of this plane (the z-line terms read them)
            float ctr[VY][VX];
#pragma unroll
            for (int vy = 0; vy < VY; ++vy) {
                float w[VX];
                load_span<T, 0, VX, 0>(tb + (vy + R) * PITCH, w);
#pragma unroll
                for (int vx = 0; vx < VX; ++vx) ctr[vy][vx] = w[vx];
            }
            phase_switch<P>(ph, [&](auto ph_c) {
                constexpr int PH = decltype(ph_c)::value;
                static_for<P>([&](auto dzi_c) {
                    constexpr int dz = decltype(dzi_c)::value - RZ;
                    constexpr int j = imod_c(PH - dz, P);
#pragma unroll
                    for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                        for (int vx = 0; vx < VX; ++vx) {
                            if constexpr (dz == 0)
                                acc[j][vy][vx] += tmp[vy][vx];
                            else
                                acc[j][vy][vx] = fmaf(
                                    coef(std::integral_constant<int, K::OT::index(dz, 0, 0)>{}),
                                    ctr[vy][vx], acc[j][vy][vx]);
                        }
                });
                constexpr int jo = imod_c(PH - RZ, P);
                store_output(zi - RZ, acc[jo]);
                zero_slot(acc[jo]);
            });
            ph = (ph + 1 == P) ? 0 : ph + 1;
            slot = (slot + 1 == NSTAGE) ? 0 : slot + 1;
        }
    }
    cp_async_wait<0>();
}

}  // namespace gst

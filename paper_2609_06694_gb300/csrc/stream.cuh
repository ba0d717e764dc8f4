// Streaming stencil sweep: one time step of out[p] = sum_o c_o in[p + o] (ForgeStencil
// Sec. 2.1) for star, box and diamond offset sets of radius R on a 2D or 3D grid.
//
// Design (sm_103a):
//  * A CTA owns an output tile of TX x TY cells (TX = 128, TY = blockDim.y * VY) and walks a
//    range of z-planes from low to high z (a range may continue into the next tile column).
//  * Input planes (tile plus an R-row halo in y and one 16-byte chunk of halo in x) land in a
//    ring of NSTAGE shared-memory slots, each with an mbarrier.  When rows are 16-byte
//    aligned one thread issues a 3D TMA tensor copy per plane (the hardware zero-fills
//    everything outside the grid: the Dirichlet ghosts); for a periodic grid the few chunks
//    of an edge tile that wrap are read into registers one plane ahead and stored over the
//    zero fill once the copy has landed.  Otherwise 16-byte cp.async (or, for odd row
//    lengths, element loads) fill the slot.  Plane z+NSTAGE-1 is in flight while plane z is
//    consumed; every wait is bounded by %globaltimer.
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
    CUtensorMap tmap;   // 3D (x, y, z) map of `in`, box (128 + 2A, TY + 2R, 1)
    const T *in;
    T *out;
    int nx, ny, nz;     // 2D grids: nz = 1
    int periodic;       // 1 = wrap, 0 = zero Dirichlet
    int aligned;        // 1 = 16-byte cp.async loader and vector stores are legal
    int tiles_x, tiles_y;
    int work;           // planes per CTA (flattened tile x z sequence)
    int use_tma;        // 1 = tensor-map loads (tmap describes `in`)
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
    static constexpr bool CREG = NPTS <= 32;         // coefficients held in registers
    // Wide-halo 3D stars with one row per thread may run 512-thread CTAs (taller tiles, less
    // halo per output row); everything else is limited to 256 threads.
    static constexpr int MAX_THREADS = (NDIM == 3 && SHAPE == kStar && R >= 3 && VY == 1) ? 512 : 256;
    static constexpr int KMAX = 4;                   // cp.async chunks held in registers
    static constexpr int KP = 2;                     // TMA patch chunks per thread
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

    // ring slot size (rounded to 128 bytes) and the shared memory of a CTA: NSTAGE slots
    // followed by one mbarrier per slot
    __host__ __device__ static constexpr size_t slot_bytes(int by) {
        return ((size_t)PITCH * (by * VY + 2 * R) * sizeof(T) + 127) / 128 * 128;
    }
    static size_t smem_bytes(int by) { return NSTAGE * slot_bytes(by) + NSTAGE * 8; }
};

template <typename T, int NDIM, int SHAPE, int R, int VY, int NSTAGE, int QMODE>
__global__ void __launch_bounds__(
    (StreamKernel<T, NDIM, SHAPE, R, VY, NSTAGE, QMODE>::MAX_THREADS))
    stream_sweep_kernel(const __grid_constant__ StreamParams<T> p,
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
    const size_t slot_bytes = K::slot_bytes(by);
    const uint32_t bar_u32 =
        static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw)) + (uint32_t)(NSTAGE * slot_bytes);
    constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // bounded waits: 2 s
    // loader mode: 2 = TMA tensor copies, 1 = 16-byte cp.async, 0 = scalar rows
    const int mode = p.use_tma ? 2 : (p.aligned ? 1 : 0);
    if (tid == 0) {
        const uint32_t arrivals = mode == 2 ? 1u : (uint32_t)nthr;
        for (int i = 0; i < NSTAGE; ++i) mbar_init(bar_u32 + 8u * i, arrivals);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t phase_bits = 0;  // parity of the next phase of every slot's mbarrier
    bool failed = false;

    const int nx = p.nx, ny = p.ny;
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

    // Persistent, balanced work: this CTA owns planes [w, w_end) of the flattened
    // (tile, z) sequence, possibly spanning the end of one tile column and the start of the
    // next; each piece is one z-stream with its own prologue.
    const int nzp = NDIM == 3 ? p.nz : 1;
    const long long total = (long long)p.tiles_x * p.tiles_y * nzp;
    long long w = (long long)blockIdx.x * p.work;
    const long long w_end = min(total, w + (long long)p.work);
    while (w < w_end) {
        const int tile = (int)(w / nzp);
        const int z_begin = (int)(w % nzp);
        const int z_end = (int)min((long long)nzp, (long long)z_begin + (w_end - w));
        w += z_end - z_begin;
        const int tix = tile % p.tiles_x, tiy = tile / p.tiles_x;
        const int x0 = tix * TX, y0 = tiy * TY;
        const int zs = z_begin - RZ, zl = z_end + RZ;

        const uint32_t smem_u32 = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
        // ---- loader state for this tile -------------------------------------------------
        // chunk c of the row-major tile (row c / CPR, 16-byte chunk c % CPR) lives at byte 16c
        // of its ring slot
        constexpr int CPR = PITCH / A;
        const int nchunks = CPR * rows;
        const int oob_lo_row = max(0, R - y0);                       // rows above the grid
        const int oob_hi_row = min(rows, max(0, ny - (y0 - R)));     // first row below the grid
        const int oob_lo_chk = max(0, (A - x0 + A - 1) / A);          // chunks left of the grid
        const int oob_hi_chk = min(CPR, max(0, (nx - (x0 - A) + A - 1) / A));
        // cp.async mode: up to KMAX chunks per thread with precomputed addresses
        uint32_t ld_dst[K::KMAX];
        int ld_src[K::KMAX];
        int nk = 0;
        // TMA mode: chunks the tensor copy zero-filled but a periodic grid wraps ("patches"),
        // up to KP per thread, loaded into registers one plane ahead
        uint32_t pt_dst[K::KP];
        int pt_src[K::KP];
        int npt = 0;
        if (mode == 1) {
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
                    ld_dst[k] = (uint32_t)(c * 16);
                    ld_src[k] = ok ? gy * nx + gx : -1;
                    nk = k + 1;
                }
            }
        } else if (mode == 2 && periodic) {
            // patch list: every chunk of the out-of-grid rows, then the out-of-grid chunks of
            // the in-grid rows; patch i goes to thread i mod nthr
            const int nrow_oob = oob_lo_row + (rows - oob_hi_row);
            const int nin_rows = oob_hi_row - oob_lo_row;
            const int nchk_oob = oob_lo_chk + (CPR - oob_hi_chk);
            const int npatch = nrow_oob * CPR + nin_rows * nchk_oob;
    #pragma unroll
            for (int k = 0; k < K::KP; ++k) {
                const int i = tid + k * nthr;
                pt_dst[k] = 0;
                pt_src[k] = 0;
                if (i < npatch) {
                    int row, cc;
                    if (i < nrow_oob * CPR) {
                        const int q = i / CPR;
                        row = q < oob_lo_row ? q : oob_hi_row + (q - oob_lo_row);
                        cc = i - q * CPR;
                    } else {
                        const int j = i - nrow_oob * CPR;
                        const int q = j / nchk_oob, e = j - q * nchk_oob;
                        row = oob_lo_row + q;
                        cc = e < oob_lo_chk ? e : oob_hi_chk + (e - oob_lo_chk);
                    }
                    bool ok = true;
                    const int gy = wrap_or_flag(y0 - R + row, ny, true, ok);
                    const int gx = wrap_or_flag(x0 - A + cc * A, nx, true, ok);
                    pt_dst[k] = (uint32_t)((row * CPR + cc) * 16);
                    pt_src[k] = gy * nx + gx;
                    npt = k + 1;
                }
            }
        }
        uint4 pt_val[K::KP];

        // Fill ring slot `slot` with input plane zi.
        //  mode 2 (TMA): thread 0 announces the box bytes and issues one 3D tensor copy; the
        //    hardware zero-fills everything outside the grid (Dirichlet ghosts); periodic
        //    edge tiles overwrite the wrapped chunks from registers (patch_plane).
        //  mode 1 (cp.async): every thread copies its 16-byte chunks, zero-filling ghosts,
        //    and its arrival on the slot's mbarrier fires when its copies have landed.
        //  mode 0 (scalar rows): element loads and stores, then an arrival.
        auto load_plane = [&](int zi, int slot) {
            bool zok = true;
            const int gz = (NDIM == 3) ? wrap_or_flag(zi, p.nz, periodic, zok) : 0;
            const uint32_t bar = bar_u32 + 8u * (uint32_t)slot;
            const uint32_t sbase = smem_u32 + (uint32_t)(slot * slot_bytes);
            if (mode == 2) {
                if (tid == 0) {
                    fence_proxy_async_shared();  // earlier reads of this slot come first
                    mbar_arrive_expect_tx(bar, (uint32_t)(PITCH * rows * ES));
                    const int zc = (NDIM == 3) ? (periodic ? gz : zi) : 0;
                    tma_load_3d(sbase, &p.tmap, x0 - A, y0 - R, zc, bar);
                }
                return;
            }
            const T *plane = p.in + (size_t)gz * plane_stride;
            if (mode == 1) {
    #pragma unroll
                for (int k = 0; k < K::KMAX; ++k) {
                    if (k < nk) {
                        const bool ok = zok && ld_src[k] >= 0;
                        const T *src = ok ? plane + ld_src[k] : p.in;
                        cp_async16_u32(sbase + ld_dst[k], src, ok ? 16 : 0);
                    }
                }
                for (int c = tid + K::KMAX * nthr; c < nchunks; c += nthr) {
                    const int row = c / CPR, cc = c - row * CPR;
                    bool ok = zok;
                    const int gy = wrap_or_flag(y0 - R + row, ny, periodic, ok);
                    const int gx = wrap_or_flag(x0 - A + cc * A, nx, periodic, ok);
                    const T *src = ok ? plane + gy * nx + gx : p.in;
                    cp_async16_u32(sbase + (uint32_t)(c * 16), src, ok ? 16 : 0);
                }
                cp_async_mbar_arrive_noinc(bar);
                return;
            }
            // scalar path: only the cells the stencil reads (x0-R .. x0+TX+R)
            T *dst = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(smem) +
                                           (size_t)slot * slot_bytes);
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
            mbar_arrive(bar);
        };
        // patches of plane zi into registers (TMA mode, periodic edge tiles)
        auto fetch_patches = [&](int zi) {
            if (npt == 0) return;
            bool zok = true;
            const int gz = (NDIM == 3) ? wrap_or_flag(zi, p.nz, true, zok) : 0;
            const T *plane = p.in + (size_t)gz * plane_stride;
    #pragma unroll
            for (int k = 0; k < K::KP; ++k)
                if (k < npt) pt_val[k] = __ldg(reinterpret_cast<const uint4 *>(plane + pt_src[k]));
        };
        auto store_patches = [&](int slot) {
            if (npt == 0) return;
            unsigned char *base = reinterpret_cast<unsigned char *>(smem) + (size_t)slot * slot_bytes;
    #pragma unroll
            for (int k = 0; k < K::KP; ++k)
                if (k < npt) *reinterpret_cast<uint4 *>(base + pt_dst[k]) = pt_val[k];
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
        for (int k = 0; k < NSTAGE - 1; ++k)
            if (zs + k < zl) load_plane(zs + k, k);
        fetch_patches(zs);

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
            const bool ok = mbar_wait_bounded(bar_u32 + 8u * (uint32_t)slot,
                                              (phase_bits >> slot) & 1u, kWaitLimitNs);
            phase_bits ^= 1u << slot;
            if (ok) store_patches(slot);  // after the tensor copy of this plane has landed
            if (__syncthreads_or(!ok)) {
                failed = true;
                return nullptr;
            }
            const int zn = zi + NSTAGE - 1;
            int sn = slot + NSTAGE - 1;
            if (sn >= NSTAGE) sn -= NSTAGE;
            if (zn < zl) load_plane(zn, sn);
            if (zi + 1 < zl) fetch_patches(zi + 1);
            return reinterpret_cast<const T *>(reinterpret_cast<const unsigned char *>(smem) +
                                               (size_t)slot * slot_bytes) +
                   thr_off;
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
                    if (!tb) {
                        done = true;
                        return;
                    }
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
                if (!tb) break;
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
                if (!tb) break;
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
        if (failed) {
            // a bounded wait expired: report, let copies still in flight land, and stop
            if (tid == 0) latch_error(p.err, kErrTimeout);
            for (int i = 0; i < NSTAGE; ++i)
                mbar_wait_bounded(bar_u32 + 8u * i, (phase_bits >> i) & 1u, 100000000ull);
            return;
        }
        __syncthreads();  // the ring is reused by the next piece
    }  // while (w < w_end)
}

}  // namespace gst

// Streaming stencil sweep: one time step of out[p] = sum_o c_o in[p + o] (ForgeStencil
// Sec. 2.1) for star, box and diamond offset sets of radius R on a 2D or 3D grid.
//
// Design (sm_103a):
//  * A CTA owns an output tile of TX x TY cells (TX = 128, TY = by * VY) and walks a range of
//    z-planes from low to high z (a range may continue into the next tile column).
//  * Warp specialisation (ring.cuh): by rows of consumer threads compute while one extra
//    producer warp keeps a ring of `nstage` shared-memory slots (a launch parameter, sized by
//    the host to fill the shared memory the resident CTAs leave) filled with input planes --
//    tile plus an R-row halo in y and one 16-byte chunk of halo in x -- by 3D TMA tensor
//    copies (hardware zero fill = Dirichlet ghosts; the chunks a periodic grid wraps into an
//    edge tile are patched over the fill once the copy has landed -- except the x halo chunks
//    of tiles at the x ends of the grid, which a second tensor copy puts into side arrays of
//    the slot, read by the lanes at the tile's ends).  Slots are handed over by "full"/"empty"
//    mbarriers, never by a CTA-wide barrier; every wait is bounded.
//  * Each plane contributes to the 2R+1 output planes it touches: every thread keeps, per owned
//    cell, a queue of 2R+1 FP32 partial sums in registers, adds the 2D slice of the offset set
//    that lies at each dz, and writes the oldest sum once the plane R above it has arrived.
//    A star therefore reads its z-neighbours from registers and only the in-plane cross from
//    shared memory; a box or diamond reuses every shared-memory read for 2R+1 outputs.
//  * In-plane neighbours come from shared memory as 16-byte vectors: a thread's VX cells are
//    contiguous in x, so one row of its window (VX + 2m values) is a few aligned loads, and
//    pairs of cells share the packed two-lane FP32 FMA.
//  * 2D grids use the same kernel with no z-radius (one plane per piece).
#pragma once

#include <utility>

#include "common.cuh"
#include "ring.cuh"

namespace gst {

template <int N, typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F> __device__ __forceinline__ void static_for(F &&f) {
    static_for_impl<N>(f, std::make_integer_sequence<int, N>{});
}

// a[v] = fma(c, w[v], a[v]) for v < N.  PAIRED issues the packed two-lane FP32 FMA of sm_100+
// on (v, v+1) -- each lane rounds exactly like fmaf -- which halves the FMA instructions when
// w[v], w[v+1] come from one aligned 8-byte pair of a vector load (an even x offset).
// FIRST: a[] holds no partial sum yet; the addend is +0 (the same bits as accumulating into
// a zeroed entry), so the entry needs no zeroing and carries no dependency on its old value.
template <int N, bool PAIRED, bool FIRST = false>
__device__ __forceinline__ void fma_n(float c, const float *w, float *a) {
    if constexpr (PAIRED && N % 2 == 0) {
        const float2 c2 = make_float2(c, c);
#pragma unroll
        for (int v = 0; v < N; v += 2) {
            const float2 r = __ffma2_rn(c2, make_float2(w[v], w[v + 1]),
                                        FIRST ? make_float2(0.0f, 0.0f)
                                              : make_float2(a[v], a[v + 1]));
            a[v] = r.x;
            a[v + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < N; ++v) a[v] = fmaf(c, w[v], FIRST ? 0.0f : a[v]);
    }
}

// ---------------------------------------------------------------------------------------
// Loads of a compile-time element range [LO, HI) from a 16-byte-aligned shared-memory base,
// converted to float into dst[(e - LO0)] where LO0 is the window origin.
// ---------------------------------------------------------------------------------------
// The values of a 32-bit word of storage type T as floats (exact: every f16 and bf16 value
// is a float).  A bfloat16 is the upper half of the float with the same value, so two integer
// operations widen both halves; a pair of halves widens in one paired conversion.
template <typename T> __device__ __forceinline__ void unpack(uint32_t bits, float *d, int n) {
    if constexpr (sizeof(T) == 4) {
        d[0] = __uint_as_float(bits);
    } else if constexpr (Storage<T>::kDType == kBF16) {
        d[0] = __uint_as_float(bits << 16);
        if (n > 1) d[1] = __uint_as_float(bits & 0xFFFF0000u);
    } else {
        __half2 h2;
        memcpy(&h2, &bits, 4);
        const float2 f = __half22float2(h2);
        d[0] = f.x;
        if (n > 1) d[1] = f.y;
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
    CUtensorMap tmap;       // 3D (x, y, z) map of `in`, box (128 + 2A, TY + 2R, 1)
    CUtensorMap side_tmap;  // the same grid, box (2A, TY + 2R, 1) (use_side only)
    CUtensorMap ymap[6];    // y-split maps of periodic y-end tiles (ring.cuh; ysplit only)
    const T *in;
    T *out;
    int nx, ny, nz;     // 2D grids: nz = 1
    int periodic;       // 1 = wrap, 0 = zero Dirichlet
    int aligned;        // 1 = 16-byte cp.async loader and vector stores are legal
    int tiles_x, tiles_y;
    int work;           // planes per CTA (flattened tile x z sequence)
    int use_tma;        // 1 = tensor-map loads (tmap describes `in`)
    int use_side;       // 1 = x-wrapped halo chunks of edge tiles by side copies (periodic)
    int ysplit;         // y-end tile rows by split copies: bit 0 the top row, bit 1 the bottom
    int nstage;         // ring slots, 2 .. kMaxStages
    int z_lo, z_cnt;    // output planes [z_lo, z_lo + z_cnt) (3D; 0, 1 for 2D)
    int *err;           // device status word (may be null)
    unsigned long long wait_ns;  // bound on the ring's waits (0: default)
    int phantom;        // fault injection only: arrivals the empty barriers wait for in vain
};

// What happens to a finished output row segment (VY rows of VX cells at (zo, oy, ox)): the
// plain sweep stores it; fused operators (the wave update) supply their own epilogue with
// their own parameter block.
// An epilogue may also read operands of its own: `prefetch` is called for output plane zo at
// the top of the iteration that finishes it (before the ring wait and the stencil), so that
// the loads it issues into `Regs` overlap them; `apply` then consumes the registers.
struct PlainStoreEpi {
    struct Params {};
    template <int VY, int VX> struct Regs {};
    template <typename T, int VY, int VX>
    __device__ __forceinline__ static void prefetch(const StreamParams<T> &, const Params &, int,
                                                    int, int, bool, int, Regs<VY, VX> &) {}
    template <typename T, int VY, int VX>
    __device__ __forceinline__ static void apply(const StreamParams<T> &p, const Params &, int zo,
                                                 int oy, int ox, bool xfull, int vy_valid,
                                                 const Regs<VY, VX> &,
                                                 const float (&vals)[VY][VX]) {
        T *orow = p.out + ((size_t)zo * p.ny + oy) * p.nx + ox;
#pragma unroll
        for (int vy = 0; vy < VY; ++vy) {
            if (vy >= vy_valid) break;
            T *dst = orow + (size_t)vy * p.nx;
            if (xfull) {
                T tmp[VX];
#pragma unroll
                for (int vx = 0; vx < VX; ++vx) tmp[vx] = Storage<T>::from_float(vals[vy][vx]);
                *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(tmp);
            } else {
#pragma unroll
                for (int vx = 0; vx < VX; ++vx)
                    if (ox + vx < p.nx) dst[vx] = Storage<T>::from_float(vals[vy][vx]);
            }
        }
    }
};

// How the partial-sum queue is indexed:
//  kQueueUnrolled : the z loop is unrolled by 2R+1 so every queue index is a constant;
//  kQueueRotate   : the queue is shifted by one entry after every plane (large stencils).
enum QueueMode : int { kQueueUnrolled = 0, kQueueRotate = 1 };

template <typename T, int NDIM, int SHAPE, int R, int VY, int QMODE>
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
    // Consumer threads per CTA: with the producer warp a CTA is then at most 8 warps, two per
    // SM sub-partition, which keeps the register cap at 255.  Wide-halo 3D stars with one row
    // per thread may take 8 consumer warps: their 288-thread bound leaves the compiler room
    // for the 72 registers of three resident CTAs (a 512-thread bound made it squeeze to 64
    // registers and spill).  With two rows per thread in f32 they may take 14 (one CTA per SM,
    // 28-row tiles: 8 halo rows on 28 instead of 14 -- 0.191 against 0.215 ms for a 512^3
    // zero-Dirichlet radius-4 star); the 480-thread bound caps the registers at 136, above the
    // 116-119 those kernels use.
    static constexpr int MAX_THREADS =
        (NDIM == 3 && SHAPE == kStar && R >= 3 && VY == 1)                        ? 256
        : (NDIM == 3 && SHAPE == kStar && R >= 3 && VY == 2 && sizeof(T) == 4) ? 448
                                                                                : 224;
    static_assert(R <= A, "x halo must fit in one 16-byte chunk");

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

    // The first term that output row vy receives from a plane at offset dz, in the order the
    // accumulation visits them (window row wr, then dx): wr * 64 + dx + R, or -1.  A queue
    // entry takes its first term from the plane at dz = -RZ.
    __host__ __device__ static constexpr int first_term(int vy, int dz) {
        for (int wr = 0; wr < VY + 2 * R; ++wr) {
            if (row_m(wr) < 0) continue;
            const int dy = wr - R - vy;
            if (dy < -R || dy > R) continue;
            for (int dx = -R; dx <= R; ++dx)
                if (OT::index(dz, dy, dx) >= 0) return wr * 64 + dx + R;
        }
        return -1;
    }

    // ring slot: one field (rounded to 128 bytes), then the side arrays of kernels that take
    // them; shared memory of a CTA
    __host__ __device__ static constexpr uint32_t field_bytes(int by) {
        return RingLayout::field_size(PITCH, by * VY + 2 * R, (int)sizeof(T));
    }
    __host__ __device__ static constexpr uint32_t side_bytes(int by, bool side) {
        return side ? RingLayout::side_size(by * VY + 2 * R) : 0u;
    }
    __host__ __device__ static constexpr size_t slot_bytes(int by, bool side) {
        return field_bytes(by) + side_bytes(by, side);
    }
    static size_t smem_bytes(int by, bool side, int nstage) {
        return RingLayout::bytes((uint32_t)slot_bytes(by, side), nstage);
    }
};

// SIDE: the launch may take x halo chunks through side arrays (periodic grids with a side
// tensor map); a kernel without SIDE has no side arrays and reads every halo chunk in place.
template <typename T, int NDIM, int SHAPE, int R, int VY, int QMODE, class EPI = PlainStoreEpi,
          bool SIDE = false>
__global__ void __launch_bounds__(
    (StreamKernel<T, NDIM, SHAPE, R, VY, QMODE>::MAX_THREADS) + 32)
    stream_sweep_kernel(const __grid_constant__ StreamParams<T> p,
                        const __grid_constant__ ConstCoeffs<OffsetTable<NDIM, SHAPE, R>::count> cf,
                        const __grid_constant__ typename EPI::Params ep) {
    using K = StreamKernel<T, NDIM, SHAPE, R, VY, QMODE>;
    constexpr int RZ = K::RZ, P = K::P, A = K::A, VX = K::VX, PITCH = K::PITCH, TX = K::TX;
    extern __shared__ __align__(128) unsigned char smem_raw[];

    // blockDim = (BX, by + 32 / BX): by rows of consumer threads, then one producer warp
    const int by = (int)blockDim.y - 32 / K::BX;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * K::BX + tx;
    const int ncons = K::BX * by;  // consumer threads (whole warps)
    const int lane = tid & 31;
    const int TY = by * VY;
    const int rows = TY + 2 * R;
    Ring g;
    g.setup(smem_raw, K::field_bytes(by), 1, p.nstage, p.wait_ns, K::side_bytes(by, SIDE));
    if (tid == 0) g.init(ncons / 32, p.phantom);
    __syncthreads();  // the only CTA-wide barrier: from here on the warps meet at mbarriers

    const int nx = p.nx, ny = p.ny;
    const bool aligned = p.aligned != 0;
    RingWork wk;
    wk.setup(p.tiles_x, p.tiles_y, p.z_cnt, p.work, TX, TY, RZ, p.z_lo);

    if (tid >= ncons) {
        // producer warp
        RingSource<T, 1> src;
        src.tmap = &p.tmap;
        src.side_tmap = &p.side_tmap;
        src.use_side = SIDE && p.use_side != 0;
        src.field = &p.in;
        src.nx = nx;
        src.ny = ny;
        src.nz = p.nz;
        src.periodic = p.periodic != 0;
        src.aligned = aligned;
        src.use_tma = p.use_tma != 0;
        src.rows = rows;
        src.ymaps = p.ymap;
        src.ysplit = p.ysplit;
        // the y-split copies only where a split can land on 128 bytes at the top (radius 4)
        ring_produce<T, 1, NDIM, R, A, PITCH, TX, SIDE && R == 4>(g, src, wk, p.err, lane);
        return;
    }

    // ---- consumer warps ---------------------------------------------------------------
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
    const int thr_off = (ty * VY) * PITCH + A + tx * VX;  // element offset of the thread's base
    // side arrays (rows of two chunks, 2A elements), in elements from a slot's side base: the
    // thread's first row in the left array, shifted so that window position -A is the row's
    // second chunk; in the right array, shifted so that window position VX is the row's first
    const int sl_off = (ty * VY) * (2 * A) + 2 * A;
    const int sr_off = (int)(RingLayout::side_half(rows) / sizeof(T)) + (ty * VY) * (2 * A) - VX;
    bool failed = false;

    RingPos pos;  // ring position of the next plane
    // Where window positions < 0 (the chunk left of the thread's cells) and >= VX (the chunk
    // right of them) of window row wr come from: lb + wr * ls and rb + wr * rs -- the plane's
    // own row (stride PITCH), or for the lanes at the ends of an x-edge tile a side array
    // (stride 2A).  Set per piece (strides) and per plane (bases).
    int ls = PITCH, rs = PITCH;
    bool use_l = false, use_r = false;
    const T *lb = nullptr, *rb = nullptr;
    // wait for the next plane to land; null once a bounded wait has given up
    auto begin_plane = [&]() -> const T * {
        if (!g.wait_full(pos.slot, pos.phase)) {
            failed = true;  // the whole warp
            return nullptr;
        }
        const unsigned char *sp = g.slot_ptr(pos.slot);
        const T *tb = reinterpret_cast<const T *>(sp) + thr_off;
        if constexpr (SIDE) {
            const T *side = reinterpret_cast<const T *>(sp + g.side_off);
            lb = use_l ? side + sl_off : tb;
            rb = use_r ? side + sr_off : tb;
        }
        return tb;
    };
    // this warp has read the slot: release it to the producer and move on
    auto end_plane = [&]() {
        g.release(pos.slot, lane);
        pos.advance(g.ns);
    };

    for (long long w = wk.w_first; w < wk.w_end && !failed;) {
        const RingPiece q = wk.piece_at(w);
        w += q.z_end - q.z_begin;
        const int z_begin = q.z_begin, z_end = q.z_end, zl = q.zl;

        float acc[P][VY][VX];
    #pragma unroll
        for (int j = 0; j < P; ++j)
    #pragma unroll
            for (int vy = 0; vy < VY; ++vy)
    #pragma unroll
                for (int vx = 0; vx < VX; ++vx) acc[j][vy][vx] = 0.0f;

        // the lanes at the ends of an x-edge tile read their wrapped halo chunk from a side array
        if constexpr (SIDE) {
            const int sbits =
                ring_side_bits(p.use_side != 0, q.x0, q.y0, nx, ny, TX, TY, R, A,
                               ring_ysplit(p.ysplit, q.y0, ny, TY, R));
            use_l = (sbits & 1) && tx == 0;
            use_r = (sbits & 2) && tx == K::BX - 1;
            ls = use_l ? 2 * A : PITCH;
            rs = use_r ? 2 * A : PITCH;
        }

        // output addressing, hoisted
        const int ox = q.x0 + tx * VX;
        const int oy = q.y0 + ty * VY;
        const bool xfull = aligned && (ox + VX <= nx);
        const int vy_valid = min(VY, ny - oy);  // may be <= 0

        typename EPI::template Regs<VY, VX> eregs;
        auto prefetch_output = [&](int zo) {
            if (zo < z_begin || zo >= z_end) return;
            EPI::template prefetch<T, VY, VX>(p, ep, zo, oy, ox, xfull, vy_valid, eregs);
        };
        auto store_output = [&](int zo, const float (&vals)[VY][VX]) {
            if (zo < z_begin || zo >= z_end) return;
            EPI::template apply<T, VY, VX>(p, ep, zo, oy, ox, xfull, vy_valid, eregs, vals);
        };

        // add the in-plane slices of the plane at `tb` to the queue; JOF(dz) = queue index of
        // output (zi - dz)
        auto accumulate = [&](const T *tb, auto jof) {
            static_for<VY + 2 * R>([&](auto wr_c) {
                constexpr int wr = decltype(wr_c)::value;
                constexpr int m = K::row_m(wr);
                if constexpr (m >= 0) {
                    float win[VX + 2 * R];
                    const T *crow = tb + wr * PITCH;
                    if constexpr (SIDE && m > 0) {
                        load_span<T, -m, 0, -R>(lb + wr * ls, win);
                        load_span<T, 0, VX, -R>(crow, win);
                        load_span<T, VX, VX + m, -R>(rb + wr * rs, win);
                    } else {
                        load_span<T, -m, VX + m, -R>(crow, win);
                    }
                    static_for<VY>([&](auto vy_c) {
                        constexpr int vy = decltype(vy_c)::value;
                        constexpr int dy = wr - R - vy;
                        if constexpr (dy >= -R && dy <= R) {
                            static_for<P>([&](auto dzi_c) {
                                constexpr int dz = decltype(dzi_c)::value - RZ;
                                constexpr int j =
                                    decltype(jof(std::integral_constant<int, dz>{}))::value;
                                static_for<2 * R + 1>([&](auto dxi_c) {
                                    constexpr int dx = decltype(dxi_c)::value - R;
                                    constexpr int idx = K::OT::index(dz, dy, dx);
                                    if constexpr (idx >= 0) {
                                        const float c = coef(std::integral_constant<int, idx>{});
                                        // the entry's first term replaces its zeroing
                                        constexpr bool FIRST =
                                            dz == -RZ &&
                                            K::first_term(vy, dz) == wr * 64 + dx + R;
                                        fma_n<VX, dx % 2 == 0, FIRST>(c, win + (dx + R),
                                                                      acc[j][vy]);
                                    }
                                });
                            });
                        }
                    });
                }
            });
        };

        int zi = q.zs;
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
                    prefetch_output(zi - RZ);
                    const T *tb = begin_plane();
                    if (!tb) {
                        done = true;
                        return;
                    }
                    accumulate(tb, [](auto dz_c) {
                        constexpr int dz = decltype(dz_c)::value;
                        return std::integral_constant<int, imod_c(ph - dz, P)>{};
                    });
                    end_plane();
                    constexpr int jo = imod_c(ph - RZ, P);
                    store_output(zi - RZ, acc[jo]);
                    ++zi;
                });
            }
        } else if constexpr (QMODE == kQueueRotate) {
            for (; zi < zl; ++zi) {
                prefetch_output(zi - RZ);
                const T *tb = begin_plane();
                if (!tb) break;
                accumulate(tb, [](auto dz_c) {
                    constexpr int dz = decltype(dz_c)::value;
                    return std::integral_constant<int, RZ - dz>{};
                });
                end_plane();
                store_output(zi - RZ, acc[0]);
    #pragma unroll
                for (int j = 0; j + 1 < P; ++j)
    #pragma unroll
                    for (int vy = 0; vy < VY; ++vy)
    #pragma unroll
                        for (int vx = 0; vx < VX; ++vx) acc[j][vy][vx] = acc[j + 1][vy][vx];
            }
        }
    }  // pieces
    // a bounded wait gave up: report and stop (the producer lets the copies in flight land
    // before the CTA exits)
    if (failed) g.fail(p.err, lane);
}

}  // namespace gst

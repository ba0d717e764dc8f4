// Two time steps of a 3D stencil in one launch (temporal blocking, ForgeStencil Sec. 4.3:
// the intermediate time level stays on chip), on the plane ring of ring.cuh.
//
// A CTA owns an output tile of 128 x TY cells and walks a range of z-planes.  The producer
// warp streams the input planes u0 with a 2R-row halo in y, a 2R-plane halo in z and one
// 16-byte chunk (>= 2R cells) of halo in x.  The consumer warps chain two streaming sweeps:
//   step 1: every input plane adds its slice of the offset set to a queue of 2R+1 FP32 partial
//           sums per cell of the tile grown by R in x and y (the core 128 columns as the
//           thread's 16-byte vectors, the R columns on each side as one cell per thread for
//           the first 2R x VY1 threads of each row of threads); once an intermediate plane u1
//           is complete it is rounded to the storage type -- so the fused result equals two
//           single sweeps bit for bit -- and written to a shared-memory plane, as 0 where it
//           lies outside a Dirichlet grid (the ghost cells step 2 reads);
//   step 2: once every consumer warp has written that u1 plane (an mbarrier, bounded wait),
//           it adds its slice to a second queue of partial sums over the tile, and a finished
//           output plane u2 is stored.
// Two u1 planes alternate: writing one plane waits for nothing, since every warp finished
// reading the other plane's previous contents before it arrived on this plane's barrier.
// Each input plane is read from DRAM once for two steps; the cost is the recomputed rim.
#pragma once

#include "common.cuh"
#include "ring.cuh"
#include "stream.cuh"

namespace gst {

template <typename T> struct Fused3DParams {
    CUtensorMap tmap;  // 3D map of `in`, box (128 + 2A, TY + 4R, 1)
    const T *in;
    T *out;
    int nx, ny, nz;
    int periodic, aligned, use_tma;
    int tiles_x, tiles_y, work, nstage;
    int *err;
    unsigned long long wait_ns;
    int phantom;
};

// Layout constants.  VY2 output rows per consumer thread, VY1 = VY2 + 1 rows of the grown
// tile; with by >= 2R rows of threads the grown tile (by * VY2 + 2R rows) fits in by * VY1.
template <typename T, int SHAPE, int R> struct Fused3DKernel {
    static constexpr int VX = 16 / (int)sizeof(T);
    static constexpr int A = VX;                // x halo of a slot: one 16-byte chunk
    static constexpr int TX = 128, BX = TX / VX;
    static constexpr int PITCH = TX + 2 * A;
    // two output rows per thread for f32, one for 16-bit storage (whose vectors hold 8 cells)
    static constexpr int VY2 = sizeof(T) == 4 ? 2 : 1, VY1 = VY2 + 1;
    static constexpr int P = 2 * R + 1;
    static constexpr int NE = 2 * R * VY1;      // rim cells of a row of threads (both sides)
    static constexpr int MAX_THREADS = 224;     // consumers; the CTA adds the producer warp
    using OT = OffsetTable<3, SHAPE, R>;
    static constexpr int NPTS = OT::count;
    static_assert(2 * R <= A, "the x halo chunk must hold 2R cells");
    static_assert(NE <= BX, "rim cells: one per thread of a row of threads");
    // the first (dy, dx) in visiting order with an offset at dz = -R: (dy + R) * 64 + dx + R
    __host__ __device__ static constexpr int rim_first() {
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx)
                if (OT::index(-R, dy, dx) >= 0) return (dy + R) * 64 + dx + R;
        return -1;
    }
    // rows a slot holds: the TY + 4R copied rows, and the windows of the last group of rows
    __host__ __device__ static constexpr int slot_rows(int by) {
        return (by * VY1 + 2 * R) > (by * VY2 + 4 * R) ? (by * VY1 + 2 * R) : (by * VY2 + 4 * R);
    }
    __host__ __device__ static constexpr uint32_t field_bytes(int by) {
        return RingLayout::field_size(PITCH, slot_rows(by), (int)sizeof(T));
    }
    // one u1 plane: the grown tile, by * VY2 + 2R rows
    __host__ __device__ static constexpr uint32_t u1_bytes(int by) {
        return RingLayout::field_size(PITCH, by * VY2 + 2 * R, (int)sizeof(T));
    }
    // the two u1 planes, then their two mbarriers, padded to keep the ring 128-byte aligned
    __host__ __device__ static constexpr uint32_t prefix_bytes(int by) {
        return 2 * u1_bytes(by) + 128;
    }
    static size_t smem_bytes(int by, int nstage) {
        return prefix_bytes(by) + RingLayout::bytes(field_bytes(by), nstage);
    }
};

// The in-plane slices of one plane added to a queue of partial sums: VYW rows of VX cells per
// thread whose window rows start at `base` (rows PITCH elements apart, the thread's first
// cell at base[0]); JOF(dz) is the queue entry of the output the plane at offset dz reaches.
// An entry takes its first term from the plane at dz = -R, written with a zero addend (the
// same bits as adding to a zeroed entry), so entries are never zeroed after use.
template <typename T, int SHAPE, int R, int VYW> struct FusedAccum {
    using OT = OffsetTable<3, SHAPE, R>;
    static constexpr int VX = 16 / (int)sizeof(T);
    static constexpr int P = 2 * R + 1;
    __host__ __device__ static constexpr int row_m(int wr) {
        int m = -1;
        for (int vy = 0; vy < VYW; ++vy) {
            const int dy = wr - R - vy;
            if (dy < -R || dy > R) continue;
            const int v = OT::max_dx_any(dy);
            if (v > m) m = v;
        }
        return m;
    }
    __host__ __device__ static constexpr int first_term(int vy) {
        for (int wr = 0; wr < VYW + 2 * R; ++wr) {
            if (row_m(wr) < 0) continue;
            const int dy = wr - R - vy;
            if (dy < -R || dy > R) continue;
            for (int dx = -R; dx <= R; ++dx)
                if (OT::index(-R, dy, dx) >= 0) return wr * 64 + dx + R;
        }
        return -1;
    }
    template <int PH, int PITCH>
    __device__ __forceinline__ static void run(const T *base, const float *coef,
                                               float (&acc)[P][VYW][VX]) {
        static_for<VYW + 2 * R>([&](auto wr_c) {
            constexpr int wr = decltype(wr_c)::value;
            constexpr int m = row_m(wr);
            if constexpr (m >= 0) {
                float win[VX + 2 * R];
                load_span<T, -m, VX + m, -R>(base + wr * PITCH, win);
                static_for<VYW>([&](auto vy_c) {
                    constexpr int vy = decltype(vy_c)::value;
                    constexpr int dy = wr - R - vy;
                    if constexpr (dy >= -R && dy <= R) {
                        static_for<P>([&](auto dzi_c) {
                            constexpr int dz = decltype(dzi_c)::value - R;
                            constexpr int j = imod_c(PH - dz, P);
                            static_for<2 * R + 1>([&](auto dxi_c) {
                                constexpr int dx = decltype(dxi_c)::value - R;
                                constexpr int idx = OT::index(dz, dy, dx);
                                if constexpr (idx >= 0) {
                                    constexpr bool FIRST =
                                        dz == -R && first_term(vy) == wr * 64 + dx + R;
                                    fma_n<VX, dx % 2 == 0, FIRST>(coef[idx], win + (dx + R),
                                                                  acc[j][vy]);
                                }
                            });
                        });
                    }
                });
            }
        });
    }
};

template <typename T, int SHAPE, int R>
__global__ void __launch_bounds__(Fused3DKernel<T, SHAPE, R>::MAX_THREADS + 32)
    fused3d_kernel(const __grid_constant__ Fused3DParams<T> p,
                   const __grid_constant__ ConstCoeffs<OffsetTable<3, SHAPE, R>::count> cf) {
    using K = Fused3DKernel<T, SHAPE, R>;
    using OT = typename K::OT;
    constexpr int VX = K::VX, A = K::A, TX = K::TX, BX = K::BX, PITCH = K::PITCH, P = K::P;
    constexpr int VY1 = K::VY1, VY2 = K::VY2;
    extern __shared__ __align__(128) unsigned char smem_raw[];

    const int by = (int)blockDim.y - 32 / BX;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * BX + tx, ncons = BX * by, lane = tid & 31;
    const int TY = by * VY2, E = TY + 2 * R;  // output rows, rows of the grown tile
    const uint32_t u1b = K::u1_bytes(by);
    T *u1buf = reinterpret_cast<T *>(smem_raw);  // two u1 planes, their barriers, the ring
    const uint32_t u1bar = static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw + 2 * u1b));
    Ring g;
    g.setup(smem_raw + K::prefix_bytes(by), K::field_bytes(by), 1, p.nstage, p.wait_ns);
    if (tid == 0) {
        mbar_init(u1bar, (uint32_t)(ncons / 32));      // u1 plane 0 written by every warp
        mbar_init(u1bar + 8, (uint32_t)(ncons / 32));  // u1 plane 1
        g.init(ncons / 32, p.phantom);                 // (its fence covers both inits)
    }
    __syncthreads();  // the only CTA-wide barrier

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool periodic = p.periodic != 0, aligned = p.aligned != 0;
    RingWork wk;
    wk.setup(p.tiles_x, p.tiles_y, nz, p.work, TX, TY, 2 * R);

    if (tid >= ncons) {
        RingSource<T, 1> src;
        src.tmap = &p.tmap;
        src.side_tmap = &p.tmap;
        src.use_side = false;
        src.field = &p.in;
        src.nx = nx;
        src.ny = ny;
        src.nz = nz;
        src.periodic = periodic;
        src.aligned = aligned;
        src.use_tma = p.use_tma != 0;
        src.rows = TY + 4 * R;
        ring_produce<T, 1, 3, 2 * R, A, PITCH, TX>(g, src, wk, p.err, lane);
        return;
    }

    float creg[K::NPTS];
#pragma unroll
    for (int i = 0; i < K::NPTS; ++i) creg[i] = cf.c[i];
    const uint32_t u1_elems = u1b / sizeof(T);
    bool failed = false;
    RingPos pos;
    int ubuf = 0;           // u1 plane written next
    uint32_t ubar_par = 0;  // parity of the next phase of each u1 plane's barrier (bits 0, 1)

    for (long long w = wk.w_first; w < wk.w_end && !failed;) {
        const RingPiece q = wk.piece_at(w);
        w += q.z_end - q.z_begin;
        // step 1 rows of this thread: grown-tile rows g1 .. g1 + VY1 - 1 (grown row e is grid
        // row y0 - R + e, slot row e + R); step 2 rows: tile rows g2 .. g2 + VY2 - 1
        const int g1 = ty * VY1, g2 = ty * VY2;
        const int ox = q.x0 + tx * VX;
        const bool xfull = aligned && ox + VX <= nx;
        const int vy_valid = min(VY2, ny - (q.y0 + g2));
        // the rim cell of this thread (tx < NE): grown row g1 + tx / 2R, R cells left of the
        // core columns or R cells right of them
        const bool has_rim = tx < K::NE && g1 + tx / (2 * R) < E;
        const int rim_row = g1 + tx / (2 * R);
        const int rim_k = tx % (2 * R);
        const int rim_col = rim_k < R ? A - R + rim_k : A + TX + (rim_k - R);  // slot column
        float q1[P][VY1][VX], q2[P][VY2][VX], qr[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            qr[j] = 0.0f;
#pragma unroll
            for (int v = 0; v < VX; ++v) {
#pragma unroll
                for (int r1 = 0; r1 < VY1; ++r1) q1[j][r1][v] = 0.0f;
#pragma unroll
                for (int r2 = 0; r2 < VY2; ++r2) q2[j][r2][v] = 0.0f;
            }
        }
        const int n = q.zl - q.zs;  // input planes of the piece
        int k = 0;
        bool done = false;
        while (!done) {
            static_for<P>([&](auto ph_c) {
                constexpr int ph = decltype(ph_c)::value;  // k mod P
                if (done) return;
                if (k >= n) {
                    done = true;
                    return;
                }
                if (!g.wait_full(pos.slot, pos.phase)) {
                    failed = done = true;
                    return;
                }
                const T *slot = reinterpret_cast<const T *>(g.slot_ptr(pos.slot));
                // step 1 on the core columns (window row 0 is slot row g1)
                if (g1 < E)
                    FusedAccum<T, SHAPE, R, VY1>::template run<ph, PITCH>(
                        slot + g1 * PITCH + A + tx * VX, creg, q1);
                // step 1 on the rim: one cell, scalar.  As in the queues above, an entry's first
                // term (from the plane at dz = -R, first in (dy, dx) order) is written with a
                // zero addend, so whatever the entry held before is never added in.
                if (has_rim) {
                    const T *c0 = slot + rim_row * PITCH + rim_col;  // window row dy = -R
                    static_for<2 * R + 1>([&](auto dyi_c) {
                        constexpr int dy = decltype(dyi_c)::value - R;
                        static_for<2 * R + 1>([&](auto dxi_c) {
                            constexpr int dx = decltype(dxi_c)::value - R;
                            if constexpr (OT::max_dx_any(dy) >= (dx < 0 ? -dx : dx)) {
                                const float v = Storage<T>::to_float(c0[(dy + R) * PITCH + dx]);
                                static_for<P>([&](auto dzi_c) {
                                    constexpr int dz = decltype(dzi_c)::value - R;
                                    constexpr int idx = OT::index(dz, dy, dx);
                                    if constexpr (idx >= 0) {
                                        constexpr int j = imod_c(ph - dz, P);
                                        constexpr bool FIRST =
                                            dz == -R && K::rim_first() == (dy + R) * 64 + dx + R;
                                        qr[j] = fmaf(creg[idx], v, FIRST ? 0.0f : qr[j]);
                                    }
                                });
                            }
                        });
                    });
                }
                g.release(pos.slot, lane);
                pos.advance(g.ns);
                if (k >= 2 * R) {
                    // u1 plane zm = zs + k - R is complete in queue entry (ph - R) mod P
                    constexpr int j1 = imod_c(ph - R, P);
                    const int zm = q.zs + k - R;
                    T *ub = u1buf + ubuf * u1_elems;
                    const bool zin = periodic || (zm >= 0 && zm < nz);
#pragma unroll
                    for (int r1 = 0; r1 < VY1; ++r1) {
                        const int e = g1 + r1;
                        if (e < E) {
                            const int gy = q.y0 - R + e;
                            const bool rin = periodic || (zin && gy >= 0 && gy < ny);
                            T tmp[VX];
#pragma unroll
                            for (int v = 0; v < VX; ++v) {
                                const bool cin = periodic || ox + v < nx;
                                tmp[v] = Storage<T>::from_float((rin && cin) ? q1[j1][r1][v]
                                                                             : 0.0f);
                            }
                            *reinterpret_cast<uint4 *>(ub + e * PITCH + A + tx * VX) =
                                *reinterpret_cast<const uint4 *>(tmp);
                        }
                    }
                    if (has_rim) {
                        const int gy = q.y0 - R + rim_row;
                        const int gx = q.x0 + rim_col - A;
                        const bool in =
                            periodic || (zin && gy >= 0 && gy < ny && gx >= 0 && gx < nx);
                        ub[rim_row * PITCH + rim_col] = Storage<T>::from_float(in ? qr[j1] : 0.0f);
                    }
                    // every consumer warp has written its part of the u1 plane (bounded wait;
                    // a warp that gave up raises the abort flag, which ends this wait too)
                    __syncwarp();
                    if (lane == 0) mbar_arrive(u1bar + 8u * ubuf);
                    if (!__all_sync(0xffffffffu,
                                    mbar_wait_abortable(u1bar + 8u * ubuf, (ubar_par >> ubuf) & 1u,
                                                        g.limit_ns, g.abort_flag))) {
                        failed = done = true;
                        return;
                    }
                    ubar_par ^= 1u << ubuf;
                    // step 2: the u1 plane's index in the piece is k - 2R, so its phase is
                    // (k - 2R) mod P = (ph + 1) mod P; window row 0 is grown row g2
                    constexpr int ph2 = imod_c(ph + 1, P);
                    FusedAccum<T, SHAPE, R, VY2>::template run<ph2, PITCH>(
                        ub + g2 * PITCH + A + tx * VX, creg, q2);
                    ubuf ^= 1;
                    if (k >= 4 * R) {
                        // output plane zo = zs + k - 2R is complete in entry (ph2 - R) mod P
                        constexpr int j2 = imod_c(ph2 - R, P);
                        const int zo = q.zs + k - 2 * R;
                        T *orow = p.out + ((size_t)zo * ny + (q.y0 + g2)) * nx + ox;
#pragma unroll
                        for (int vy = 0; vy < VY2; ++vy) {
                            if (vy >= vy_valid) break;
                            T *dst = orow + (size_t)vy * nx;
                            if (xfull) {
                                T tmp[VX];
#pragma unroll
                                for (int v = 0; v < VX; ++v)
                                    tmp[v] = Storage<T>::from_float(q2[j2][vy][v]);
                                *reinterpret_cast<uint4 *>(dst) =
                                    *reinterpret_cast<const uint4 *>(tmp);
                            } else {
#pragma unroll
                                for (int v = 0; v < VX; ++v)
                                    if (ox + v < nx)
                                        dst[v] = Storage<T>::from_float(q2[j2][vy][v]);
                            }
                        }
                    }
                }
                ++k;
            });
        }
    }
    if (failed) g.fail(p.err, lane);
}

}  // namespace gst

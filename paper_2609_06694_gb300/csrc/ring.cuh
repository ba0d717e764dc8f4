// The plane ring shared by the streaming kernels: a CTA walks z-planes of a tile; one producer
// warp keeps a ring of shared-memory slots filled with the input planes (NF fields per plane,
// each a tile plus an R-row halo in y and one 16-byte chunk of halo in x, then -- for kernels
// that ask for them -- two side arrays holding the x halo chunks of a periodic edge tile)
// while the consumer warps compute.  Each slot has three mbarriers:
//   full  -- the plane is in the slot (32 arrivals of the producer warp, plus copied bytes),
//   empty -- every consumer warp has finished reading it (one arrival per consumer warp),
//   tma   -- its tensor copies have landed (periodic tiles that still need patches).
// After set-up the warps never meet at a CTA-wide barrier: consumers drift apart by up to
// nstage - 1 planes and hide one another's latencies.  Every wait is bounded by
// %globaltimer; a wait that gives up raises the CTA's abort flag and the device error word.
#pragma once

#include "common.cuh"

namespace gst {

constexpr int kMaxStages = 16;   // ring slots
constexpr int kMaxPatches = 256; // wrapped 16-byte chunks patched per plane
constexpr int kSideRowBytes = 32;  // a row of a side array: two 16-byte chunks
constexpr unsigned long long kRingWaitNs = 2000000000ull;  // default bound on a wait: 2 s

// Shared-memory layout: nstage slots of NF fields, then full/empty/tma mbarriers, the abort
// flag and the patch list.
struct RingLayout {
    uint32_t field_bytes;  // one field of one plane (128-byte multiple)
    uint32_t slot_bytes;   // NF fields
    int ns;
    __host__ __device__ static constexpr uint32_t field_size(int pitch, int rows, int es) {
        return (uint32_t)(((size_t)pitch * rows * es + 127) / 128 * 128);
    }
    // the side arrays of a slot: for every row, the two 16-byte chunks left of the tile (the
    // second one is its x halo) and then the two right of it (the first one is the halo), each
    // array starting on a 128-byte boundary (tensor-copy destinations); 32-byte rows put every
    // fourth row on a 128-byte boundary, where a split copy of the wrapped rows may start
    __host__ __device__ static constexpr uint32_t side_half(int rows) {
        return (uint32_t)((kSideRowBytes * rows + 127) / 128 * 128);
    }
    __host__ __device__ static constexpr uint32_t side_size(int rows) {
        return 2 * side_half(rows);
    }
    __host__ __device__ static constexpr size_t bytes(uint32_t slot_bytes, int ns) {
        return (size_t)ns * (slot_bytes + 24) + 16 + 8 * kMaxPatches;
    }
};

struct Ring {
    unsigned char *base;
    uint32_t base_u32, field_bytes, slot_bytes;
    uint32_t side_off;  // byte offset of the side arrays in a slot (after the NF fields)
    int ns;
    uint32_t full_u32, empty_u32, tma_u32;
    volatile int *abort_flag;
    uint2 *plist;
    unsigned long long limit_ns;  // bound on every wait

    __device__ __forceinline__ void setup(unsigned char *smem, uint32_t fbytes, int nf, int nstage,
                                          unsigned long long wait_ns, uint32_t side_bytes = 0) {
        limit_ns = wait_ns ? wait_ns : kRingWaitNs;
        base = smem;
        base_u32 = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
        field_bytes = fbytes;
        side_off = fbytes * nf;
        slot_bytes = fbytes * nf + side_bytes;
        ns = nstage;
        full_u32 = base_u32 + (uint32_t)ns * slot_bytes;
        empty_u32 = full_u32 + 8u * (uint32_t)ns;
        tma_u32 = empty_u32 + 8u * (uint32_t)ns;
        abort_flag = reinterpret_cast<volatile int *>(smem + (size_t)ns * slot_bytes + 24 * ns);
        plist = reinterpret_cast<uint2 *>(smem + (size_t)ns * slot_bytes + 24 * ns + 16);
    }
    // thread 0, before the CTA's only __syncthreads.  `phantom` extra arrivals on the empty
    // barriers never come (fault injection only: the producer's wait for a free slot expires).
    __device__ __forceinline__ void init(int consumer_warps, int phantom = 0) const {
        for (int i = 0; i < ns; ++i) {
            mbar_init(full_u32 + 8u * i, 32u);  // the producer warp
            mbar_init(empty_u32 + 8u * i, (uint32_t)(consumer_warps + phantom));  // per warp
            mbar_init(tma_u32 + 8u * i, 1u);                         // the producer's lane 0
        }
        *abort_flag = 0;
        mbar_init_fence();
    }
    __device__ __forceinline__ const unsigned char *slot_ptr(int slot) const {
        return base + (size_t)slot * slot_bytes;
    }
    // consumers: wait (warp-uniformly) for the plane in `slot`; false once a wait gives up
    __device__ __forceinline__ bool wait_full(int slot, uint32_t phase) const {
        return __all_sync(0xffffffffu, mbar_wait_abortable(full_u32 + 8u * slot, phase,
                                                            limit_ns, abort_flag));
    }
    // consumers: this warp has read `slot`
    __device__ __forceinline__ void release(int slot, int lane) const {
        __syncwarp();
        // lane 0 arrives (a predicated arrive: no branch around it)
        asm volatile(
            "{\n .reg .pred p;\n setp.eq.s32 p, %1, 0;\n"
            " @p mbarrier.arrive.shared::cta.b64 _, [%0];\n}\n" ::"r"(empty_u32 + 8u * slot),
            "r"(lane)
            : "memory");
    }
    __device__ __forceinline__ void fail(int *err, int lane) const {
        *abort_flag = 1;
        if (lane == 0) latch_error(err, kErrTimeout);
    }
};

// Ring position of a plane sequence: plane k of it sits in slot k mod ns, pass parity
// (k / ns) mod 2.
struct RingPos {
    int slot = 0;
    uint32_t phase = 0;
    __device__ __forceinline__ void advance(int ns) {
        if (++slot == ns) {
            slot = 0;
            phase ^= 1u;
        }
    }
};

// A CTA's work: planes [w_first, w_end) of the flattened (tile, z) sequence over the z range
// [zoff, zoff + nz) (tiles in row-major order, z fastest), possibly spanning several tiles;
// each piece is one z-stream of a tile, read with RZ extra planes on each side.  The sequence
// takes the two tile rows at the y ends of the grid first (tile row 0, then the last one, then
// rows 1, 2, ...): on a periodic grid their rows wrap, their planes need patches and their
// CTAs run longest, so they start in the first wave instead of trailing the launch.
struct RingPiece {
    int x0, y0, z_begin, z_end, zs, zl;
};
struct RingWork {
    long long w_first, w_end;
    int nzp, tiles_x, tiles_y, TX, TY, RZ;
    int zoff;  // first plane of the z range the sequence covers (nz planes from it)
    // work > 0: CTA b takes planes [b * work, (b + 1) * work) of the sequence (a range may
    // continue into the next tile column).  work = -c: every tile column is cut into c chunks
    // of near-equal length and CTA b takes chunk b % c of column b / c -- no CTA spans two
    // columns, and the CTAs of neighbouring tiles start at the same planes.
    __device__ __forceinline__ void setup(int tiles_x_, int tiles_y_, int nz, int work, int TX_,
                                          int TY_, int RZ_, int zoff_ = 0) {
        tiles_x = tiles_x_;
        tiles_y = tiles_y_;
        nzp = nz;
        zoff = zoff_;
        TX = TX_;
        TY = TY_;
        RZ = RZ_;
        const long long total = (long long)tiles_x_ * tiles_y_ * nz;
        if (work > 0) {
            w_first = (long long)blockIdx.x * work;
            w_end = min(total, w_first + (long long)work);
        } else {
            // chunk k of a column starts at k * q + min(k, r) (q = nz / c, r = nz % c: the
            // first r chunks take one plane more); 32-bit divisions only
            const unsigned c = (unsigned)(-work), b = blockIdx.x;
            const unsigned col = b / c, k = b - col * c;
            const unsigned q = (unsigned)nz / c, r = (unsigned)nz - q * c;
            const long long base = (long long)col * nz;
            w_first = min(total, base + (long long)(k * q + min(k, r)));
            w_end = min(total, base + (long long)((k + 1) * q + min(k + 1, r)));
        }
    }
    __device__ __forceinline__ RingPiece piece_at(long long w) const {
        RingPiece q;
        const int tile = (int)(w / nzp);
        const int zr = (int)(w % nzp);
        q.z_begin = zoff + zr;
        q.z_end = zoff + (int)min((long long)nzp, (long long)zr + (w_end - w));
        const int tix = tile % tiles_x, k = tile / tiles_x;
        const int tiy = k == 0 ? 0 : (k == 1 ? tiles_y - 1 : k - 1);  // y ends first
        q.x0 = tix * TX;
        q.y0 = tiy * TY;
        q.zs = q.z_begin - RZ;
        q.zl = q.z_end + RZ;
        return q;
    }
};

// What the producer copies: NF fields of the grid (nz x ny x nx, x fastest) and, when rows
// are 16-byte aligned and the driver could encode them, one 3D tensor map per field with the
// box (PITCH, rows, 1).  With use_side (one field, periodic), side_tmap is a second map of the
// same field with the box (A, rows, 1): one 16-byte column chunk of every row.
// With ysplit (one field, periodic), ymaps are six more maps of the field for the tile rows
// at the y ends: [0] box (PITCH, rows - R) -- the top tile row's rows from y = 0, [1] box
// (PITCH, hb + R) -- the bottom tile row's rows from y0 - R to the grid's end (hb: its output
// rows), [2] box (PITCH, R) -- the R wrapped rows; [3], [4], [5] the same three boxes two
// chunks wide (2A) for the side arrays (use_side only).
template <typename T, int NF> struct RingSource {
    const CUtensorMap *tmap;       // NF maps (kernel parameters)
    const CUtensorMap *side_tmap;  // the side map (use_side only)
    const T *const *field;         // NF pointers
    int nx, ny, nz;
    bool periodic, aligned, use_tma, use_side;
    int rows;
    const CUtensorMap *ymaps = nullptr;  // the y-split maps (ysplit != 0 only)
    int ysplit = 0;  // bit 0: the top tile row takes split copies, bit 1: the bottom one
};

// Whether a tile of a periodic grid takes its wrapped rows by split tensor copies (ysplit
// bits set by the host where the split lands on a 128-byte boundary of the slot): 1 = the top
// tile row (rows above y = 0 wrap), 2 = the bottom one (rows from ny wrap), 0 = neither.
__device__ __forceinline__ int ring_ysplit(int ysplit, int y0, int ny, int TY, int R) {
    if ((ysplit & 1) && y0 == 0) return 1;
    if ((ysplit & 2) && y0 >= R && y0 + TY + R > ny) return 2;
    return 0;
}

// Which x halo chunks of a piece come from the slot's side arrays: bit 0 the left chunk (the
// tile starts at x = 0, so the chunk wraps to x = nx - A), bit 1 the right one (the tile ends
// at x = nx, so it wraps to x = 0); a side copy takes two chunks per row (x = nx - 2A and
// x = 0, 2A wide).  Only periodic tiles whose rows all lie inside the grid and
// whose width is whole qualify: the tensor copy of the plane zero-fills those chunks in the
// slot, a second tensor copy of the wrapped column fills the side array alongside it on the
// same barrier, and the consumer lanes at the tile's ends read the side array instead -- the
// producer never touches the plane again.  Tiles at the y ends qualify too where their
// wrapped rows come by split copies (ysplit_kind != 0): their side arrays then take split
// copies as well.  Producer and consumers evaluate the same rule.
__device__ __forceinline__ int ring_side_bits(bool use_side, int x0, int y0, int nx, int ny,
                                              int TX, int TY, int R, int A,
                                              int ysplit_kind = 0) {
    if (!use_side || nx < 2 * A) return 0;
    if (ysplit_kind == 0 && (y0 < R || y0 + TY + R > ny)) return 0;
    const bool right = x0 + TX + A > nx;
    if (right && x0 + TX != nx) return 0;  // a partial tile: the wrap lands inside the tile
    return (x0 == 0 ? 1 : 0) | (right ? 2 : 0);
}

// The producer warp: fills slot k with plane k of the CTA's sequence once every consumer warp
// has released plane k - ns, then exits after the copies still in flight have landed.
//  mode 2, TMA: lane 0 announces the bytes and issues one 3D tensor copy per field; the
//    hardware zero-fills everything outside the grid (Dirichlet ghosts).
//  mode 5, TMA + side chunks: a periodic tile that wraps only in x (ring_side_bits) takes the
//    same tensor copy plus one copy of each wrapped 16-byte column into the slot's side
//    arrays, all on the full barrier, like mode 2.
//  mode 4, TMA + patches: any other tile into which a periodic grid wraps takes the same tensor
//    copies, on the slot's "tma" barrier; as soon as they have landed (the producer polls the
//    "tma" and "empty" barriers in turn), the lanes copy the wrapped 16-byte chunks (whole rows
//    above or below the grid, single chunks left or right of it) over the zero fill with
//    cp.async and arrive on the full barrier when those have landed.
//  mode 6, split TMA: a periodic tile at a y end (ring_ysplit) whose columns need no wrap, or
//    wrap into side arrays: two tensor copies on the full barrier -- the rows inside the grid
//    and, into the slot rows next to them, the R wrapped rows (top: grid rows ny - R .. ny - 1
//    into slot rows 0 .. R - 1; bottom: grid rows 0 .. R - 1 after the last grid row) -- so
//    nothing is copied twice and nothing waits for a copy to land.  The bottom tile row loads
//    only its hb + 2R needed rows.  Side arrays, if any, take the same split, two chunks wide.
//  mode 3, bulk rows: tiles with more wrapped chunks than the patch list holds (grids
//    narrower than a tile): one bulk copy per contiguous segment of each row.
//  mode 1, cp.async: no tensor map: 16-byte chunks of whole rows, wrapping or zero-filling.
//  mode 0: element copies (rows not 16-byte aligned).
// Field f of a slot starts f * field_bytes into it; rows are PITCH elements apart and the
// tile's column 0 sits A elements into a row.
// YSPLIT: mode 6 is compiled in (the plain periodic streaming sweep); other kernels patch the
// wrapped rows (mode 4) and keep the producer's registers -- and their occupancy -- as they were.
template <typename T, int NF, int NDIM, int R, int A, int PITCH, int TX, bool YSPLIT = false>
__device__ __forceinline__ void ring_produce(const Ring &g, const RingSource<T, NF> &src,
                                             const RingWork &wk, int *err, int lane) {
    constexpr int ES = (int)sizeof(T);
    constexpr int CPR = PITCH / A;  // 16-byte chunks per shared-memory row
    const int nx = src.nx, ny = src.ny, rows = src.rows, ns = g.ns;
    const bool periodic = src.periodic;
    const size_t plane_stride = (size_t)nx * ny;
    const uint32_t plane_bytes = (uint32_t)(PITCH * rows * ES);
    RingPos pos;
    bool ok = true;
    int issued = 0;      // planes issued so far (for the final drain)
    int pslot = 0;       // ring slot of the next plane to publish in mode 4
    uint32_t tbits = 0;  // parity of each slot's next "tma" phase
    int unpub = 0;       // mode-4 planes issued but not yet published
    auto wait_all = [&](uint32_t bar, uint32_t parity) {
        // the lanes agree on the outcome, so the warp never splits
        return __all_sync(0xffffffffu,
                          mbar_wait_abortable(bar, parity, g.limit_ns, g.abort_flag));
    };
    for (long long w = wk.w_first; w < wk.w_end && ok;) {
        const RingPiece q = wk.piece_at(w);
        w += q.z_end - q.z_begin;
        // Chunks a periodic grid wraps into the tile: every chunk of the rows above the grid
        // (rows < lo_row) and of the first R rows below it (rows >= hi_row), then, in the rows
        // between, the chunks left of x = 0 (chunks < lo_chk) and the first chunk right of nx
        // (chunk hi_chk).  Rows further below and chunks further right feed only outputs
        // outside the grid, which are never stored: they keep the copy's zero fill (a ragged
        // last tile row would otherwise patch most of its plane).
        const int lo_row = max(0, R - q.y0);
        const int hi_row = min(rows, max(0, ny - (q.y0 - R)));
        const int lo_chk = max(0, (A - q.x0 + A - 1) / A);
        const int hi_chk = min(CPR, max(0, (nx - (q.x0 - A) + A - 1) / A));
        const int nrow_oob = lo_row + min(rows - hi_row, R);
        const int nwc = lo_chk + min(CPR - hi_chk, 1);
        const int npatch = nrow_oob * CPR + (hi_row - lo_row) * nwc;
        const int yk = (YSPLIT && NF == 1) ? ring_ysplit(src.ysplit, q.y0, ny, wk.TY, R) : 0;
        const int sbits = ring_side_bits(src.use_side, q.x0, q.y0, nx, ny, TX, wk.TY, R, A, yk);
        const bool x_inside = q.x0 >= A && q.x0 + TX + A <= nx;
        int mode;
        if (!src.use_tma) mode = src.aligned ? 1 : 0;
        else if (!periodic || npatch == 0) mode = 2;
        else if (YSPLIT && yk != 0 && (x_inside || sbits != 0)) mode = 6;
        else if (sbits != 0) mode = 5;
        else if (npatch <= kMaxPatches && hi_row >= lo_row) mode = 4;
        else mode = 3;
        if (mode == 4) {
            // every publish of the previous piece is done: the list is free
            for (int i = lane; i < npatch; i += 32) {
                int row, cc;
                if (i < nrow_oob * CPR) {
                    const int qr = i / CPR;
                    row = qr < lo_row ? qr : hi_row + (qr - lo_row);
                    cc = i - qr * CPR;
                } else {
                    const int j = i - nrow_oob * CPR;  // here nwc > 0
                    const int qr = j / nwc, e = j - qr * nwc;
                    row = lo_row + qr;
                    cc = e < lo_chk ? e : hi_chk + (e - lo_chk);
                }
                bool wok = true;
                const int gy = wrap_or_flag(q.y0 - R + row, ny, true, wok);
                const int gx = wrap_or_flag(q.x0 - A + cc * A, nx, true, wok);
                g.plist[i] =
                    make_uint2((uint32_t)((row * CPR + cc) * 16), (uint32_t)(gy * nx + gx));
            }
            __syncwarp();
        }

        // mode 4: plane zpl's tensor copies have landed -> patch them and release the plane
        auto publish = [&](int zpl) -> bool {
            if (!wait_all(g.tma_u32 + 8u * pslot, (tbits >> pslot) & 1u)) return false;
            tbits ^= 1u << pslot;
            --unpub;
            bool zok = true;
            const int gz = (NDIM == 3) ? wrap_or_flag(zpl, src.nz, true, zok) : 0;
            const uint32_t sbase = g.base_u32 + (uint32_t)pslot * g.slot_bytes;
            for (int i = lane; i < npatch; i += 32) {
                const uint2 e = g.plist[i];
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    cp_async16_u32(sbase + f * g.field_bytes + e.x,
                                   src.field[f] + (size_t)gz * plane_stride + (int)e.y, 16);
            }
            cp_async_mbar_arrive_noinc(g.full_u32 + 8u * pslot);
            if (++pslot == ns) pslot = 0;
            return true;
        };
        // load plane zi into the slot the ring has reached (already released)
        auto issue = [&](int zi) {
            bool zok = true;
            const int gz = (NDIM == 3) ? wrap_or_flag(zi, src.nz, periodic, zok) : 0;
            const uint32_t bar = g.full_u32 + 8u * pos.slot;
            const uint32_t sbase = g.base_u32 + (uint32_t)pos.slot * g.slot_bytes;
            if (mode == 2 || mode == 4 || mode == 5) {
                if (lane == 0) {
                    fence_proxy_async_shared();  // consumers' reads of this slot come first
                    const uint32_t tb = mode == 4 ? g.tma_u32 + 8u * pos.slot : bar;
                    const uint32_t side_bytes =
                        mode == 5 ? (uint32_t)(__popc(sbits) * rows * kSideRowBytes) : 0u;
                    mbar_arrive_expect_tx(tb, NF * plane_bytes + side_bytes);
                    const int zc = (NDIM == 3) ? (periodic ? gz : zi) : 0;
#pragma unroll
                    for (int f = 0; f < NF; ++f)
                        tma_load_3d(sbase + f * g.field_bytes, &src.tmap[f], q.x0 - A, q.y0 - R,
                                    zc, tb);
                    if (mode == 5) {
                        // the wrapped columns: left chunks from x = nx - 2A, right ones from 0
                        const uint32_t side = sbase + g.side_off;
                        if (sbits & 1)
                            tma_load_3d(side, src.side_tmap, nx - 2 * A, q.y0 - R, zc, tb);
                        if (sbits & 2)
                            tma_load_3d(side + RingLayout::side_half(rows), src.side_tmap, 0,
                                        q.y0 - R, zc, tb);
                    }
                } else if (mode != 4) {
                    mbar_arrive(bar);
                }
                if (mode == 4) ++unpub;
            } else if (YSPLIT && mode == 6) {
                // top: wrapped rows from ny - R into slot rows [0, R), grid rows from 0 into
                // [R, rows); bottom: grid rows from y0 - R into [0, hb + R), wrapped rows from 0
                // into [hb + R, hb + 2R); the side arrays alike.  Every split lies on a 128-byte
                // boundary (host-checked).
                if (lane == 0) {
                    const int zc = (NDIM == 3) ? gz : 0;
                    const int hb = ny - q.y0;  // bottom: output rows of the tile
                    const int split = yk == 1 ? R : hb + R;  // first row of the second copy
                    const int nrows = yk == 1 ? rows : hb + 2 * R;
                    const uint32_t row_bytes = (uint32_t)(PITCH * ES);
                    fence_proxy_async_shared();  // consumers' reads of this slot come first
                    mbar_arrive_expect_tx(
                        bar, (uint32_t)nrows * (row_bytes + __popc(sbits) * kSideRowBytes));
                    // the first copy from y_a into row 0, the second from y = 0 (the top's
                    // rows inside the grid, the bottom's wrapped rows) into row `split`
                    const int y_a = yk == 1 ? ny - R : q.y0 - R;
                    const int y_b = 0;
                    const CUtensorMap *ma = &src.ymaps[yk == 1 ? 2 : 1];
                    const CUtensorMap *mb = &src.ymaps[yk == 1 ? 0 : 2];
                    tma_load_3d(sbase, ma, q.x0 - A, y_a, zc, bar);
                    tma_load_3d(sbase + (uint32_t)split * row_bytes, mb, q.x0 - A, y_b, zc, bar);
                    const uint32_t side = sbase + g.side_off;
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        if (!((sbits >> k) & 1)) continue;
                        const uint32_t sd = side + (uint32_t)k * RingLayout::side_half(rows);
                        const int xs = k == 0 ? nx - 2 * A : 0;
                        tma_load_3d(sd, ma + 3, xs, y_a, zc, bar);
                        tma_load_3d(sd + (uint32_t)split * kSideRowBytes, mb + 3, xs, y_b, zc,
                                    bar);
                    }
                } else {
                    mbar_arrive(bar);
                }
            } else if (mode == 3) {
                // every smem row is one to a few contiguous, 16-byte aligned segments of a
                // (wrapped) grid row: the lanes take the rows and copy the segments in bulk
                if (lane == 0) mbar_arrive_expect_tx(bar, NF * plane_bytes);
                __syncwarp();  // the byte count is announced before any copy can land
                fence_proxy_async_shared();
                for (int row = lane; row < rows; row += 32) {
                    bool rok = true;
                    const int gy = wrap_or_flag(q.y0 - R + row, ny, true, rok);
                    const size_t roff = (size_t)gz * plane_stride + (size_t)gy * nx;
                    const uint32_t drow = sbase + (uint32_t)(row * PITCH * ES);
                    for (int col = 0; col < PITCH;) {
                        int gx = (q.x0 - A + col) % nx;
                        if (gx < 0) gx += nx;
                        const int len = min(PITCH - col, nx - gx);
#pragma unroll
                        for (int f = 0; f < NF; ++f)
                            bulk_copy_g2s(drow + f * g.field_bytes + (uint32_t)(col * ES),
                                          src.field[f] + roff + gx, (uint32_t)(len * ES), bar);
                        col += len;
                    }
                }
                if (lane != 0) mbar_arrive(bar);
            } else if (mode == 1) {
                // lane L copies chunk columns L and L + 32 of every row (those < CPR)
                bool cok0 = true, cok1 = (lane + 32 < CPR);
                const int gx0 = lane < CPR ? wrap_or_flag(q.x0 - A + lane * A, nx, periodic, cok0)
                                           : 0;
                const int gx1 =
                    cok1 ? wrap_or_flag(q.x0 - A + (lane + 32) * A, nx, periodic, cok1) : 0;
                for (int row = 0; row < rows; ++row) {
                    bool rok = zok;
                    const int gy = wrap_or_flag(q.y0 - R + row, ny, periodic, rok);
                    const size_t roff = (size_t)gz * plane_stride + (size_t)gy * nx;
                    const uint32_t drow = sbase + (uint32_t)(row * PITCH * ES);
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const T *fs = src.field[f];
                        if (lane < CPR) {
                            const bool ok0 = rok && cok0;
                            cp_async16_u32(drow + f * g.field_bytes + 16u * lane,
                                           ok0 ? fs + roff + gx0 : fs, ok0 ? 16 : 0);
                        }
                        if (lane + 32 < CPR) {
                            const bool ok1 = rok && cok1;
                            cp_async16_u32(drow + f * g.field_bytes + 16u * (lane + 32),
                                           ok1 ? fs + roff + gx1 : fs, ok1 ? 16 : 0);
                        }
                    }
                }
                cp_async_mbar_arrive_noinc(bar);
            } else {
                // only the cells the stencil reads (x0-R .. x0+TX+R)
                const int wcols = TX + 2 * R;
                for (int row = 0; row < rows; ++row) {
                    bool rok = zok;
                    const int gy = wrap_or_flag(q.y0 - R + row, ny, periodic, rok);
                    for (int col = lane; col < wcols; col += 32) {
                        bool ok2 = rok;
                        const int gx = wrap_or_flag(q.x0 - R + col, nx, periodic, ok2);
                        const size_t gi = (size_t)gz * plane_stride + (size_t)gy * nx + gx;
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            T *dst = reinterpret_cast<T *>(g.base + (size_t)pos.slot * g.slot_bytes +
                                                           f * g.field_bytes);
                            dst[row * PITCH + (A - R) + col] =
                                ok2 ? src.field[f][gi] : Storage<T>::from_float(0.0f);
                        }
                    }
                }
                mbar_arrive(bar);
            }
            ++issued;
            pos.advance(ns);
        };

        pslot = pos.slot;
        if (mode != 4) {
            for (int zi = q.zs; zi < q.zl; ++zi) {
                if (!wait_all(g.empty_u32 + 8u * pos.slot, pos.phase ^ 1u)) {
                    ok = false;
                    break;
                }
                issue(zi);
            }
        } else {
            // Patched planes: issue whenever a slot is free, publish the oldest issued plane
            // as soon as its tensor copies have landed, and otherwise doze briefly and look
            // again -- never block on one of the two, so a slot freed while a copy is in
            // flight is refilled at once, and publishing never waits for a slot (which would
            // wait for consumers, which wait for published planes).  The idle time is bounded.
            int zi = q.zs, zp = q.zs;  // next plane to issue / to publish
            unsigned int idle = 0;
            unsigned long long t0 = 0;
            while (zp < q.zl) {
                if (zi < q.zl &&
                    __all_sync(0xffffffffu,
                               mbar_test_wait(g.empty_u32 + 8u * pos.slot, pos.phase ^ 1u))) {
                    issue(zi++);
                    idle = 0;
                } else if (zp < zi &&
                           __all_sync(0xffffffffu, mbar_test_wait(g.tma_u32 + 8u * pslot,
                                                                  (tbits >> pslot) & 1u))) {
                    if (!publish(zp)) {
                        ok = false;
                        break;
                    }
                    ++zp;
                    idle = 0;
                } else {
                    if (idle++ == 0) t0 = globaltimer_ns();
                    else if ((idle & 63u) == 0 &&
                             __any_sync(0xffffffffu, *g.abort_flag != 0 ||
                                                         globaltimer_ns() - t0 > g.limit_ns)) {
                        ok = false;
                        break;
                    }
                    __nanosleep(40);
                }
            }
        }
    }
    if (!ok) g.fail(err, lane);
    // Whatever the consumers do, every copy still in flight lands before the CTA can exit:
    // tensor copies of planes never published, then (bounded) the last min(issued, ns)
    // planes, the only ones that may still be in flight (in normal runs the consumers wait
    // for them anyway).
    cp_async_wait<0>();
    for (int j = 0, s2 = pslot; j < unpub; ++j, s2 = (s2 + 1 == ns) ? 0 : s2 + 1)
        mbar_wait_bounded(g.tma_u32 + 8u * s2, (tbits >> s2) & 1u, 100000000ull);
    for (int k = 0; k < min(issued, ns); ++k) {
        if (--pos.slot < 0) {
            pos.slot = ns - 1;
            pos.phase ^= 1u;
        }
        mbar_wait_bounded(g.full_u32 + 8u * pos.slot, pos.phase, 100000000ull);
    }
}

}  // namespace gst

// The dense radius-2 box (125 points in 3D, 25 in 2D) on the tensor cores, for 16-bit storage
// (ForgeStencil Sec. 6, "A refuted tensor-core mapping": the dense box is the one
// compute-bound stencil; a banded Toeplitz packing casts it onto the matrix units).
//
// Mapping.  For one (dz, dy) pair the x part of the sweep over a row segment is a product with
// a banded Toeplitz matrix:
//     out[z, y, x0 + n] += sum_k u[z + dz, y + dy, x0 - 8 + k] * B_{dz,dy}[k, n],
//     B_{dz,dy}[k, n] = c(dz, dy, k - 8 - n)   where |k - 8 - n| <= 2, else 0.
// A CTA owns M = 128 consecutive output rows (y) by NB blocks of 16 outputs (x) and walks a
// chunk of z planes.  The shifted input rows are the A operand, read in place from the plane
// tile in shared memory (one 16-column half of the window per MMA, K = 16), and the Toeplitz
// matrices are the B operand.  Each B row block holds the coefficients split into a 16-bit
// head and a 16-bit tail (c = hi + lo, both in the storage type), so the product keeps the
// coefficients to about 16 significant bits while the inputs are exact; the FP32 accumulators
// (tensor memory) are summed head + tail in the epilogue and rounded once to the storage type.
// The window halves of neighbouring blocks overlap: the half that is the second half of block
// p - 1 is the first of block p, so one M128 x N64 x K16 MMA (B = both halves' matrices)
// serves both blocks, whose accumulators sit side by side (block b at columns (NB-1-b) * 32).
// Per output plane, input plane (5 in 3D) and row offset dy (5) that is NB + 1 MMAs.
//
// Dense packing pays a density penalty: 32 K-elements per output and (dz, dy) pair against 5
// useful taps, twice for the head/tail split.  The MMAs are narrow (N <= 64), and their rate
// is set by how fast they are issued: MW warps issue them, each for every MW-th output plane.
//
// Shared-memory layout of a plane tile (the A operand).  Rows y0-2 .. y0+129 (132 rows) of
// the input window x0-8 .. x0-8+16(NB+1), stored as columns of 16-byte chunks: chunk c (8
// elements) of row r sits at c * 2176 + r * 16 (2176 = 132 rows of 16 bytes rounded up to
// 128 bytes).  In the no-swizzle K-major core-matrix layout of the tensor cores (8 rows x 16
// bytes per core matrix) that is a matrix with stride-between-K-chunks (LBO) 2176 bytes and
// stride-between-8-row-groups (SBO) 128 bytes;
// the A operand of row offset dy is the same matrix started 16 * (dy + 2) bytes later.  Each
// chunk column is one 3D TMA tensor copy (box 8 x 132 x 1) from the grid, zero-filling outside
// it (zero Dirichlet); the copies of a plane complete on one mbarrier.
//
// Warp roles (5 + MW warps): warp 0 issues the TMA copies, warps 1..MW issue the MMAs (one
// lane each; warp 1 also owns the tensor memory), the last 4 warps read the accumulators
// (each warp its 32 lanes of tensor memory) and store the outputs.  Slots and accumulators
// change hands through mbarriers; tcgen05.commit signals MMA completion; a slot is refilled
// once every issuing warp has released its plane.  Every wait is bounded: on expiry the CTA
// latches STENCIL_ERR_TIMEOUT, raises its abort flag, waits (bounded) for the copies and MMAs
// it issued, frees its tensor memory and returns.
#pragma once

#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace gst {

namespace tz {

constexpr int kRows = 132;              // 128 output rows + 2 halo rows on each side
// one column of 16-byte chunks, padded to a multiple of 128 bytes: every tensor copy into
// shared memory starts on a 128-byte boundary
constexpr int kChunkBytes = 2176;
static_assert(kChunkBytes >= kRows * 16 && kChunkBytes % 128 == 0, "chunk column");
// threads of a CTA: the producer warp, mw MMA warps and 4 epilogue warps (at most 4 MMA warps)
constexpr int kMaxThreads = 288;
__host__ __device__ constexpr int threads(int mw) { return 32 * (5 + mw); }
constexpr int kBBytes = 2048;           // B of one (dz, dy) pair: N64 x K16, 16-bit
constexpr int kPad = 2048;              // guard after the B matrices

__host__ __device__ constexpr int slot_bytes(int nb) { return 2 * (nb + 1) * kChunkBytes; }
// accumulators (one per output plane in flight, nb x 32 columns each) and tensor-memory
// columns
constexpr int kNacc = 4;
__host__ __device__ constexpr int tmem_cols(int nb) { return kNacc * nb * 32; }
__host__ __device__ constexpr int nbmat(int dzn) { return dzn * 5; }
// bytes of dynamic shared memory: slots, B matrices, guard, then the barriers and flags
__host__ __device__ constexpr int smem_bytes(int nb, int dzn, int ns) {
    return ns * slot_bytes(nb) + nbmat(dzn) * kBBytes + kPad + (2 * ns + 2 * kNacc + 1) * 8 +
           16 + 1024;  // + alignment slack for the 1024-byte aligned base
}

// No-swizzle K-major shared-memory matrix descriptor (tcgen05): start address, leading
// (K-direction) and stride (8-row-group) byte offsets, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both f16 (fmt 0) or both
// bf16 (fmt 1), both K-major, N and M as given.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t m, uint32_t n) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     dst_smem),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// D (tensor memory) = A * B (+ D when accumulate != 0); A and B from shared memory.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive once on the mbarrier when every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
        : "memory");
}
// 32 consecutive FP32 columns of this thread's tensor-memory lane (the load and its wait in
// one statement, so no register is read before the data has arrived).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <typename T> struct Half16;
template <> struct Half16<__nv_bfloat16> {
    static constexpr uint32_t kFmt = 1;
    static __device__ __forceinline__ uint16_t bits(float f) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(f));
    }
    static __device__ __forceinline__ float value(uint16_t b) {
        return __bfloat162float(__ushort_as_bfloat16(b));
    }
};
template <> struct Half16<__half> {
    static constexpr uint32_t kFmt = 0;
    static __device__ __forceinline__ uint16_t bits(float f) {
        return __half_as_ushort(__float2half_rn(f));
    }
    static __device__ __forceinline__ float value(uint16_t b) {
        return __half2float(__ushort_as_half(b));
    }
};

}  // namespace tz

template <int N> struct ToeplitzCoeffs {
    float c[N];  // canonical order of the radius-2 box
};

struct ToeplitzParams {
    void *out;
    int nz, ny, nx;
    int tiles_x, tiles_y;   // CTA tiles along x (16 NB outputs) and y (128 rows)
    int z_lo, z_hi;         // output planes [z_lo, z_hi)
    int z_chunk;            // output planes per CTA
    int stages;             // plane slots in the ring (>= 5)
    int *err;
    unsigned long long wait_ns;
    int phantom;            // extra arrivals the accumulator-free barriers wait for (tests)
};

// DZN = 5 (3D) or 1 (2D).  One work item (x tile, y tile, z chunk) per CTA.  MW warps issue
// the MMAs, each for every MW-th output plane of the CTA.
template <typename T, int NB, int DZN, int MW>
__global__ void __launch_bounds__(tz::kMaxThreads)
    toeplitz_box_kernel(const __grid_constant__ CUtensorMap map, const ToeplitzParams P,
                        const __grid_constant__ ToeplitzCoeffs<DZN * 25> cf) {
    using H = tz::Half16<T>;
    constexpr int RZ = DZN / 2;
    constexpr int SLOT = tz::slot_bytes(NB);
    static_assert(MW >= 1 && MW <= tz::kNacc, "MMA warps");
    constexpr int NACC = tz::kNacc;
    constexpr int COLS = tz::tmem_cols(NB);
    constexpr int NBM = tz::nbmat(DZN);
    const int NS = P.stages;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw));
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    const uint32_t slots = base;
    const uint32_t bmat = slots + NS * SLOT;
    const uint32_t bars = bmat + NBM * tz::kBBytes + tz::kPad;
    // barriers: full[NS], empty[NS], accf[NACC], acce[NACC], drain
    const uint32_t full0 = bars, empty0 = bars + 8 * NS, accf0 = bars + 16 * NS,
                   acce0 = accf0 + 8 * NACC, drain = acce0 + 8 * NACC;
    unsigned char *gflags = gbase + (drain + 8 - base);
    volatile uint32_t *tmem_holder = reinterpret_cast<volatile uint32_t *>(gflags);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gflags + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long limit = P.wait_ns ? P.wait_ns : 2000000000ull;

    // work item
    const int item = blockIdx.x;
    const int tx = item % P.tiles_x;
    const int ty = (item / P.tiles_x) % P.tiles_y;
    const int zc = item / (P.tiles_x * P.tiles_y);
    const int x0 = tx * 16 * NB, y0 = ty * 128;
    const int z0 = P.z_lo + zc * P.z_chunk;
    const int nzo = min(P.z_chunk, P.z_hi - z0);  // output planes of this CTA (>= 1)
    const int nin = nzo + 2 * RZ;                  // input planes

    // Toeplitz B matrices, one per (dz, dy) pair: rows n = 0-31 take the first 16 columns of
    // a block's input window (kk = 0), rows 32-63 the second (kk = 1); within each, rows 0-15
    // the head and 16-31 the tail of each coefficient.  K-major, no swizzle: element (n, k) at
    // (k / 8) * 1024 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2 (all threads)
    for (int e = threadIdx.x; e < NBM * 1024; e += blockDim.x) {
        const int mi = e >> 10, rem = e & 1023;
        const int n = rem >> 4, k = rem & 15;
        const int kk = n >> 5, nn = n & 31, dyi = mi % 5, dzi = mi / 5;
        const int dx = 16 * kk + k - 8 - (nn & 15);
        uint16_t b = 0;
        if (dx >= -2 && dx <= 2) {
            const float c = cf.c[(dzi * 5 + dyi) * 5 + dx + 2];
            const uint16_t hi = H::bits(c);
            b = nn < 16 ? hi : H::bits(c - H::value(hi));
        }
        const uint32_t off = mi * tz::kBBytes + (k >> 3) * 1024 + (n >> 3) * 128 + (n & 7) * 16 +
                             (k & 7) * 2;
        *reinterpret_cast<uint16_t *>(gbase + (bmat - base) + off) = b;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, MW);
        }
        for (int a = 0; a < NACC; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 4 + P.phantom);
        }
        mbar_init(drain, MW);
        *abort_flag = 0;
        mbar_init_fence();
    }
    fence_proxy_async_shared();  // the B matrices, written by threads, are read by the MMA unit
    if (warp == 1) {
        __syncwarp();  // the allocation is a warp-wide, converged instruction
        tz::tmem_alloc(static_cast<uint32_t>(
                           __cvta_generic_to_shared(const_cast<uint32_t *>(tmem_holder))),
                       COLS);
    }
    tz::tc_fence_before();
    __syncthreads();
    tz::tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        // ---- producer: 2 (NB + 1) tensor copies per input plane, one per chunk column ----
        int issued = 0;
        if (lane == 0) {
            for (int i = 0; i < nin; ++i) {
                const int s = i % NS;
                if (i >= NS && !mbar_wait_abortable(empty0 + 8 * s, ((i / NS) - 1) & 1, limit,
                                                    abort_flag)) {
                    if (!*abort_flag) {
                        latch_error(P.err, kErrTimeout);
                        *abort_flag = 1;
                    }
                    break;
                }
                if (((slots + s * SLOT) & 127u) != 0 || s >= NS) {  // never, by construction
                    latch_error(P.err, kErrBounds);
                    *abort_flag = 1;
                    break;
                }
                mbar_arrive_expect_tx(full0 + 8 * s, 2 * (NB + 1) * tz::kRows * 16);
                for (int c = 0; c < 2 * (NB + 1); ++c)
                    tma_load_3d(slots + s * SLOT + c * tz::kChunkBytes, &map, x0 - 8 + 8 * c,
                                y0 - 2, z0 - RZ + i, full0 + 8 * s);
                issued = i + 1;
            }
            // every copy issued lands before the CTA may exit
            for (int i = max(0, issued - NS); i < issued; ++i)
                mbar_wait_bounded(full0 + 8 * (i % NS), (i / NS) & 1, limit);
        }
    } else if (warp <= MW) {
        // ---- MMA issuers, A read from shared memory: warp w (1..MW) runs the output planes
        // j = w - 1, w - 1 + MW, ... ----
        if (lane == 0) {
            // output-stationary.  Block b of an output plane accumulates at columns
            // (NB - 1 - b) * 32, so the accumulators of blocks p and p - 1 are adjacent in that
            // order: the A tile of window chunk pair p feeds both with one N64 MMA whose B is
            // the pair's whole matrix (kk = 0 rows for block p, kk = 1 rows for block p - 1)
            constexpr uint32_t idesc32 = tz::instr_desc(H::kFmt, 128, 32);
            constexpr uint32_t idesc64 = tz::instr_desc(H::kFmt, 128, 64);
            const uint64_t bdesc0 = tz::smem_desc(bmat, 1024, 128);
            const int w = warp - 1;
            // a slot is refilled once each issuing warp has released its plane: this warp
            // releases plane p when none of its later output planes reads it (planes the
            // producer never refills, p >= nin - NS, are not released)
            int released = 0;
            const int lim = nin - NS;
            auto release_upto = [&](int p_end, bool after_mmas) {
                for (const int e = min(p_end, lim); released < e; ++released) {
                    const uint32_t bar = empty0 + 8 * (released % NS);
                    if (after_mmas) tz::mma_commit(bar);  // once this warp's MMAs are done
                    else mbar_arrive(bar);
                }
            };
            release_upto(w < nzo ? w : nin, false);
            bool ok = true;
            for (int j = w; j < nzo && ok; j += MW) {
                const int a = j % NACC;
                if (j >= NACC &&
                    !mbar_wait_abortable(acce0 + 8 * a, ((j / NACC) - 1) & 1, limit, abort_flag)) {
                    ok = false;
                    break;
                }
                tz::tc_fence_after();
                const uint32_t dacc = tmem + a * NB * 32;
                for (int dzi = 0; dzi < DZN && ok; ++dzi) {
                    const int i = j + dzi, s = i % NS;
                    if (!mbar_wait_abortable(full0 + 8 * s, (i / NS) & 1, limit, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tz::tc_fence_after();
                    const uint64_t adesc0 = tz::smem_desc(slots + s * SLOT, tz::kChunkBytes, 128);
#pragma unroll
                    for (int dyi = 0; dyi < 5; ++dyi) {
                        const uint64_t bpair = bdesc0 + (((dzi * 5 + dyi) * tz::kBBytes) >> 4);
                        const uint64_t bkk1 = bpair + (512 >> 4);  // rows 32-63
                        if (dzi == 0 && dyi == 0) {
                            // first terms: every block is written once by its kk = 0 MMA
                            // before any accumulates into it (consecutive MMAs write
                            // different blocks)
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                                for (int b = 0; b < NB; ++b)
                                    tz::mma_f16(dacc + (NB - 1 - b) * 32,
                                                adesc0 + ((2 * (b + kk) * tz::kChunkBytes + dyi * 16) >> 4),
                                                kk ? bkk1 : bpair, idesc32, kk);
                            continue;
                        }
                        // chunk pairs in the order 0, 2, 4, .., 1, 3, ..: consecutive MMAs
                        // write disjoint accumulator columns
#pragma unroll
                        for (int q = 0; q <= NB; ++q) {
                            const int p = 2 * q <= NB ? 2 * q : 2 * (q - NB / 2 - 1) + 1;
                            const uint64_t adesc =
                                adesc0 + ((2 * p * tz::kChunkBytes + dyi * 16) >> 4);
                            if (p == 0)
                                tz::mma_f16(dacc + (NB - 1) * 32, adesc, bpair, idesc32, 1);
                            else if (p == NB)
                                tz::mma_f16(dacc, adesc, bkk1, idesc32, 1);
                            else
                                tz::mma_f16(dacc + (NB - 1 - p) * 32, adesc, bpair, idesc64, 1);
                        }
                    }
                }
                if (!ok) break;
                tz::mma_commit(accf0 + 8 * a);
                release_upto(j + MW < nzo ? j + MW : nin, true);
            }
            if (!ok && !*abort_flag) {
                latch_error(P.err, kErrTimeout);
                *abort_flag = 1;
            }
            // every MMA issued completes before the tensor memory is freed
            tz::mma_commit(drain);
            mbar_wait_bounded(drain, 0, limit);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warps MW + 1 .. MW + 4, tensor-memory lanes 32 * (warp % 4) ----
        const int q = warp & 3;
        const int y = y0 + q * 32 + lane;
        for (int j = 0; j < nzo; ++j) {
            const int a = j % NACC;
            bool ok = true;
            if (lane == 0) ok = mbar_wait_abortable(accf0 + 8 * a, (j / NACC) & 1, limit, abort_flag);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0 && !*abort_flag) {
                    latch_error(P.err, kErrTimeout);
                    *abort_flag = 1;
                }
                break;
            }
            tz::tc_fence_after();
            T *orow = static_cast<T *>(P.out) + ((size_t)(z0 + j) * P.ny + y) * P.nx;
#pragma unroll 1
            for (int b = 0; b < NB; ++b) {
                float v[32];
                tz::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + a * NB * 32 + (NB - 1 - b) * 32,
                              v);
                if (b == NB - 1) {
                    tz::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce0 + 8 * a);
                }
                const int xs = x0 + 16 * b;
                if (y < P.ny && xs < P.nx) {
                    uint32_t w[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const uint32_t lo = H::bits(v[2 * t] + v[2 * t + 16]);
                        const uint32_t hi = H::bits(v[2 * t + 1] + v[2 * t + 17]);
                        w[t] = lo | (hi << 16);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(orow + xs);
                    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    if (xs + 8 < P.nx) dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
                }
            }
        }
    }
    tz::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tz::tc_fence_after();
        tz::tmem_dealloc(tmem, COLS);
    }
}

}  // namespace gst

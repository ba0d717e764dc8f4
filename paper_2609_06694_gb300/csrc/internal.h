// Internal interface between the host plan code (plan.cpp) and the kernel translation units.
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gst {

// Bounds of the plane ring's device-side waits (a plan setting): every wait gives up after
// `ns` nanoseconds (0 = the default of 2 s).  `phantom` > 0 adds that many arrivals that never
// come to every slot's "consumers are done" barrier -- fault injection for tests only: the
// producer's wait for a free slot then expires and the launch reports STENCIL_ERR_TIMEOUT,
// while every copy already issued still lands before the CTA exits.
struct RingWait {
    unsigned long long ns = 0;
    int phantom = 0;
};

// Device status words (status.cu): one per plan, in a fixed array of the library's device
// image (nothing is allocated).  status_acquire returns a free slot or -1; status_word the
// slot's device address on the current device (null if the lookup fails); status_take
// synchronises the stream, then returns and clears the slot's code.
constexpr int kStatusSlots = 65536;  // live plans at most (256 KiB per device)
int status_acquire();
void status_release(int slot, bool used);
int *status_word(int slot);
int status_take(int slot, cudaStream_t s);

// Raises the kernel's dynamic shared-memory limit on the current device to at least `smem`
// bytes (and with max_carveout asks for the largest shared-memory carveout).  The attribute is
// per device: the calls are recorded per (device, kernel) under a mutex, so any host thread
// may launch on any device.  False if the runtime refuses.
bool smem_opt_in(const void *kern, size_t smem, bool max_carveout);

// One launch of the streaming sweep kernel (one time step).
struct StreamLaunch {
    int ndim;                // 2 or 3
    int64_t nz, ny, nx;      // 2D: nz = 1
    int shape, radius, dtype;
    int periodic;
    const float *coeffs;     // host array, canonical order, shape_count entries
    const void *in;
    void *out;
    int block_x, block_y, vec_y, z_chunk;
    int stages = 0;          // ring depth (0 = fill the shared memory, see ring_stages)
    int z_lo = 0, z_hi = -1; // 3D: output planes [z_lo, z_hi) only (z_hi < 0: to nz)
    int use_tma = 1;         // 0 forces the cp.async loader (tensor maps are used when legal)
    int *err = nullptr;      // device status word (status_word) or null
    RingWait wait;           // bound on the ring's waits, fault injection
    cudaStream_t stream;
};

// Returns 0, or a negative STENCIL_ERR_* code.  One per storage type and dimension.
// Most consumer threads of a streaming kernel's CTA (kept in step with
// StreamKernel::MAX_THREADS); the CTA adds one producer warp.
constexpr int stream_max_threads(int ndim, int shape, int radius, int vec_y, int dtype) {
    return (ndim == 3 && shape == 0 && radius >= 3 && vec_y == 1)                ? 256
           : (ndim == 3 && shape == 0 && radius >= 3 && vec_y == 2 && dtype == 0) ? 448
                                                                                  : 224;
}

// Defined in stream_<dtype>_<ndim>d_<shape>.cu.
#define GST_DECLARE_STREAM(DT, ND)                          \
    int launch_stream_##DT##_##ND##d_star(const StreamLaunch &L); \
    int launch_stream_##DT##_##ND##d_box(const StreamLaunch &L);  \
    int launch_stream_##DT##_##ND##d_diamond(const StreamLaunch &L);
GST_DECLARE_STREAM(f32, 2)
GST_DECLARE_STREAM(f32, 3)
GST_DECLARE_STREAM(f16, 2)
GST_DECLARE_STREAM(f16, 3)
GST_DECLARE_STREAM(bf16, 2)
GST_DECLARE_STREAM(bf16, 3)
#undef GST_DECLARE_STREAM
int launch_stream(const StreamLaunch &L);  // dispatches on dtype, ndim and shape

// Rows per thread compiled for a streaming kernel: 1 always; 2 for every 2D stencil, every 3D
// star and 3D box/diamond up to radius 2; 4 for radius 1 (wider 3D stencils are ALU-heavy
// enough that more rows cost more registers than the shared-memory reads they save).
constexpr bool stream_vy_compiled(int ndim, int shape, int radius, int vec_y) {
    return vec_y == 1 || (vec_y == 2 && (ndim == 2 || shape == 0 || radius <= 2)) ||
           (vec_y == 4 && radius == 1);
}

// Two time steps of a 3D stencil in one launch (fused3d.cuh): the StreamLaunch fields as for
// the streaming kernel (block_y rows of threads, vec_y must be 2); compiled for star and
// diamond sets of radius 1-2 and the radius-1 box.
int launch_fused3d(const StreamLaunch &L);

// One reaction-diffusion step u + dt (A u + c1 u + c3 u^3) on the streaming kernel (reaction.cuh):
// vec_y must be 1; star sets of radius 1, 2, 4 and the radius-1 box; f32 and bf16 storage.
int launch_reaction_f32(const StreamLaunch &L, float dt, float c1, float c3);
int launch_reaction_bf16(const StreamLaunch &L, float dt, float c1, float c3);
constexpr bool fused3d_compiled(int ndim, int shape, int radius) {
    return ndim == 3 && ((shape != 1 && radius >= 1 && radius <= 2) || (shape == 1 && radius == 1));
}

// The radius-2 box on the tensor cores (toeplitz.cuh): one step per launch, 16-bit storage,
// zero Dirichlet, rows a multiple of 8 cells; nb blocks of 16 outputs per CTA along x (1, 2
// or 4), mw warps issuing the MMAs, each for every mw-th output plane (1 or 2; 4 with nb = 4),
// z_chunk output planes per CTA (0 = one wave), stages plane slots (0 = automatic, else at
// least 5 in 3D).
int launch_toeplitz(const StreamLaunch &L, int nb, int mw);
constexpr bool toeplitz_compiled(int ndim, int shape, int radius, int dtype) {
    return (ndim == 2 || ndim == 3) && shape == 1 && radius == 2 && (dtype == 1 || dtype == 2);
}

// Several 2D time steps in one launch (shared-memory tile with a shrinking halo).
struct Fused2DLaunch {
    int64_t ny, nx;
    int shape, radius, dtype;
    int periodic;
    const float *coeffs;     // host array, canonical order
    const void *in;
    void *out;
    int steps;               // steps fused in this launch (>= 1)
    int tile_x, tile_y;      // output tile
    int block_threads;
    cudaStream_t stream;
};
int launch_fused2d(const Fused2DLaunch &L);
size_t fused2d_smem_bytes(int tile_x, int tile_y, int radius, int steps);

// Variable-coefficient sweeps (VAR forward/adjoint, div(k grad u)).
struct VarLaunch {
    int ndim;
    int64_t nz, ny, nx;
    int shape, radius, dtype;
    int periodic;
    const void *in;
    void *out;
    const void *const *arrays;  // VAR: npts arrays; DIVKGRAD: k
    int narrays;
    int block_y, z_chunk;
    int vec_y = 1;  // div(k grad u): output rows per thread (1 or 2)
    int *err = nullptr;  // device status word (div(k grad u), whose ring waits are bounded)
    RingWait wait;
    cudaStream_t stream;
};
#define GST_DECLARE_VAR(DT)                               \
    int launch_var_##DT##_fwd(const VarLaunch &L);        \
    int launch_var_##DT##_adj(const VarLaunch &L);        \
    int launch_divkgrad_##DT(const VarLaunch &L);
GST_DECLARE_VAR(f32)
GST_DECLARE_VAR(f16)
GST_DECLARE_VAR(bf16)
#undef GST_DECLARE_VAR
constexpr int kMaxVarArrays = 27;

// Kernel launch counter (all families).
void count_launch(uint64_t n = 1);

}  // namespace gst

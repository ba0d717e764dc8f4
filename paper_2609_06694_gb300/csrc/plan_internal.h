// Plan and batch objects behind the opaque handles of include/stencil.h (host only).
#pragma once

#include <stdint.h>

#include <vector>

#include <cuda_runtime.h>

#include "../../include/stencil.h"
#include "internal.h"

struct stencil_plan_s {
    int ndim = 0;
    int64_t dims[3] = {1, 1, 1};  // (nz, ny, nx); nz = 1 for 2D grids
    int shape = 0, radius = 0, kind = 0, dtype = 0, boundary = 0;  // shape, radius: compiled set
    bool custom = false;           // a caller-given offset set (embedded in shape/radius)
    int64_t npts = 0;
    std::vector<int32_t> offsets;  // npts * ndim, canonical order (custom: the caller's order)
    std::vector<double> coeffs;    // STENCIL_CONST: as given
    std::vector<float> cf;         // f32 coefficients of the compiled set (0 where unused)
    std::vector<float> cf_flip;    // coefficient of -o at the index of o (adjoint)
    stencil_variant variant{};
    void *scratch = nullptr;       // one grid of the storage type (multi-step ping-pong)
    size_t scratch_bytes = 0;
    void *stage_in = nullptr;      // staging for stencil_apply_host
    void *stage_out = nullptr;
    size_t stage_bytes = 0;
    int status_slot = -1;          // the plan's device status word (status.cu)
    bool launched = false;         // a kernel of this plan may have written the word
    gst::RingWait wait;            // bound on the ring kernels' waits, fault injection
    // stencil_apply_host's z-slab pipeline: copy-in and copy-out streams and their events
    static constexpr int kMaxSlabs = 8;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[kMaxSlabs] = {}, ev_out[kMaxSlabs] = {}, ev_start = nullptr,
                ev_done = nullptr;
};

namespace gst {
std::vector<int32_t> make_offsets(int ndim, int shape, int r);
int size_class_of(int64_t cells);
int validate_variant(const stencil_plan_s &p, const stencil_variant &v);
size_t dtype_size(int dtype);
int ensure_scratch(stencil_plan_s &p);
int run_steps(stencil_plan_s &p, const float *cf, const void *in, void *out, int steps,
              cudaStream_t s);
int check_apply_args(const stencil_plan_s *p, const void *in, const void *out, int steps);
bool overlaps(const void *a, const void *b, size_t n);
int launch_group_with(stencil_plan_s &p, const float *cf, const void *src, void *dst, int k,
                      cudaStream_t s);
int plan_steps_per_launch(const stencil_plan_s &p);  // steps one launch of the plan fuses
// The batched launch's tile shape and steps per group for a storage type, from the dispatch
// map's "batch" lines (all zero: no entry).
struct BatchShape {
    int tile_y = 0, tile_x = 0, fuse = 0;
};
BatchShape batch_shape_for(int dtype);
int map_launch_rc(int rc);
}  // namespace gst

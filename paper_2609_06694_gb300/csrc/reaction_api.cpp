// stencil_apply_reaction (include/stencil.h): explicit reaction-diffusion steps, each one
// launch of the streaming kernel with the fused reaction epilogue (reaction.cuh).
#include <algorithm>
#include <cmath>

#include <cuda_runtime.h>

#include "../../include/stencil.h"
#include "internal.h"
#include "plan_internal.h"

namespace gst {

// The streaming launch of one reaction step with the plan's tile: one output row per thread
// (the tile keeps the plan's height where the thread cap allows), the plan's z chunk and ring
// depth; plans on another kernel family take the streaming defaults.
static int reaction_step(stencil_plan_s &p, const void *src, void *dst, float dt, float c1,
                         float c3, cudaStream_t s) {
    const stencil_variant &v = p.variant;
    const int bx = (int)(128 / (16 / dtype_size(p.dtype)));
    int by = 128 / bx;
    int z_chunk = p.ndim == 3 ? 64 : 0, stages = 0;
    if (v.family == STENCIL_FAMILY_STREAM) {
        by = v.block_y * v.vec_y;
        z_chunk = v.z_chunk;
        stages = v.stages;
    }
    const int cap = stream_max_threads(p.ndim, p.shape, p.radius, 1, p.dtype) / bx;
    by = std::max(1, std::min(by, cap));
    while ((bx * by) % 32) --by;
    StreamLaunch L;
    L.ndim = p.ndim;
    L.nz = p.dims[0];
    L.ny = p.dims[1];
    L.nx = p.dims[2];
    L.shape = p.shape;
    L.radius = p.radius;
    L.dtype = p.dtype;
    L.periodic = p.boundary == STENCIL_PERIODIC;
    L.coeffs = p.cf.data();
    L.in = src;
    L.out = dst;
    L.block_x = bx;
    L.block_y = by;
    L.vec_y = 1;
    L.z_chunk = z_chunk;
    L.stages = stages;
    L.err = status_word(p.status_slot);
    L.wait = p.wait;
    L.stream = s;
    p.launched = true;
    const int rc = p.dtype == STENCIL_F32 ? launch_reaction_f32(L, dt, c1, c3)
                                          : launch_reaction_bf16(L, dt, c1, c3);
    return map_launch_rc(rc);
}

}  // namespace gst

extern "C" int stencil_apply_reaction(stencil_handle h, const void *in, void *out, int steps,
                                      double dt, double c1, double c3, void *stream) {
    using namespace gst;
    int rc = check_apply_args(h, in, out, steps);
    if (rc) return rc;
    if (h->kind != STENCIL_CONST) return STENCIL_ERR_BADARG;
    if (!std::isfinite(dt) || !std::isfinite(c1) || !std::isfinite(c3)) return STENCIL_ERR_BADARG;
    if (h->dtype == STENCIL_F16) return STENCIL_ERR_UNSUPPORTED;
    const bool star = h->shape == STENCIL_STAR && (h->radius == 1 || h->radius == 2 || h->radius == 4);
    const bool box = h->shape == STENCIL_BOX && h->radius == 1;
    if (!star && !box) return STENCIL_ERR_UNSUPPORTED;
    if (steps > 1) {
        rc = ensure_scratch(*h);
        if (rc) return rc;
    }
    // the steps alternate between `out` and the scratch grid; the last one writes `out`
    const void *src = in;
    for (int t = 0; t < steps; ++t) {
        void *dst = ((steps - 1 - t) % 2 == 0) ? out : h->scratch;
        rc = reaction_step(*h, src, dst, (float)dt, (float)c1, (float)c3, (cudaStream_t)stream);
        if (rc) return rc;
        src = dst;
    }
    return STENCIL_OK;
}

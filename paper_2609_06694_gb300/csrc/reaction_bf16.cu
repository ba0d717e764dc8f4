// Reaction-diffusion kernels: bfloat16 storage (instantiations only).
#include "reaction_launch.cuh"

namespace gst {
int launch_reaction_bf16(const StreamLaunch &L, float dt, float c1, float c3) {
    return launch_reaction_t<__nv_bfloat16>(L, dt, c1, c3);
}
}  // namespace gst

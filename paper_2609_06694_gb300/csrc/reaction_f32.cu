// Reaction-diffusion kernels: float storage (instantiations only).
#include "reaction_launch.cuh"

namespace gst {
int launch_reaction_f32(const StreamLaunch &L, float dt, float c1, float c3) {
    return launch_reaction_t<float>(L, dt, c1, c3);
}
}  // namespace gst

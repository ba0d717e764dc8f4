// Streaming-sweep kernels: float storage, 3D grids, star offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_f32_3d_star(const StreamLaunch &L) {
    return launch_stream_r<float, 3, kStar>(L);
}
}  // namespace gst

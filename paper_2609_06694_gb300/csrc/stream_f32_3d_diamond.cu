// Streaming-sweep kernels: float storage, 3D grids, diamond offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_f32_3d_diamond(const StreamLaunch &L) {
    return launch_stream_r<float, 3, kDiamond>(L);
}
}  // namespace gst

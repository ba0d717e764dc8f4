// Streaming-sweep kernels: float storage, 3D grids, box offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_f32_3d_box(const StreamLaunch &L) {
    return launch_stream_r<float, 3, kBox>(L);
}
}  // namespace gst

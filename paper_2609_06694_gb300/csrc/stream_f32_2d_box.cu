// Streaming-sweep kernels: float storage, 2D grids, box offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_f32_2d_box(const StreamLaunch &L) {
    return launch_stream_r<float, 2, kBox>(L);
}
}  // namespace gst

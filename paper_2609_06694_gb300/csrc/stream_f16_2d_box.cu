// Streaming-sweep kernels: __half storage, 2D grids, box offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_f16_2d_box(const StreamLaunch &L) {
    return launch_stream_r<__half, 2, kBox>(L);
}
}  // namespace gst

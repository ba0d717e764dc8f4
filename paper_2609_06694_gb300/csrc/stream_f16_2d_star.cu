// Streaming-sweep kernels: __half storage, 2D grids, star offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_f16_2d_star(const StreamLaunch &L) {
    return launch_stream_r<__half, 2, kStar>(L);
}
}  // namespace gst

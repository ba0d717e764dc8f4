// Streaming-sweep kernels: __half storage, 2D grids, diamond offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_f16_2d_diamond(const StreamLaunch &L) {
    return launch_stream_r<__half, 2, kDiamond>(L);
}
}  // namespace gst

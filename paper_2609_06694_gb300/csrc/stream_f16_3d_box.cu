// Streaming-sweep kernels: __half storage, 3D grids, box offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_f16_3d_box(const StreamLaunch &L) {
    return launch_stream_r<__half, 3, kBox>(L);
}
}  // namespace gst

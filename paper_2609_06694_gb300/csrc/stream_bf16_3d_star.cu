// Streaming-sweep kernels: __nv_bfloat16 storage, 3D grids, star offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_bf16_3d_star(const StreamLaunch &L) {
    return launch_stream_r<__nv_bfloat16, 3, kStar>(L);
}
}  // namespace gst

// Streaming-sweep kernels: __nv_bfloat16 storage, 3D grids, diamond offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_bf16_3d_diamond(const StreamLaunch &L) {
    return launch_stream_r<__nv_bfloat16, 3, kDiamond>(L);
}
}  // namespace gst

// Streaming-sweep kernels: __nv_bfloat16 storage, 2D grids, diamond offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_bf16_2d_diamond(const StreamLaunch &L) {
    return launch_stream_r<__nv_bfloat16, 2, kDiamond>(L);
}
}  // namespace gst

// Streaming-sweep kernels: __nv_bfloat16 storage, 2D grids, box offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_bf16_2d_box(const StreamLaunch &L) {
    return launch_stream_r<__nv_bfloat16, 2, kBox>(L);
}
}  // namespace gst

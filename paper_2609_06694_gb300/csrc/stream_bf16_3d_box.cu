// Streaming-sweep kernels: __nv_bfloat16 storage, 3D grids, box offset sets (instantiations only).
#include "stream_launch.cuh"

namespace gst {
int launch_stream_bf16_3d_box(const StreamLaunch &L) {
    return launch_stream_r<__nv_bfloat16, 3, kBox>(L);
}
}  // namespace gst

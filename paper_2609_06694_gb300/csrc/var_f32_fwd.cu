// Variable-coefficient kernels: float storage, forward sweep and div(k grad u) (instantiations only).
#include "var_launch.cuh"

namespace gst {
int launch_var_f32_fwd(const VarLaunch &L) { return launch_var_dt<float, false>(L); }
int launch_divkgrad_f32(const VarLaunch &L) { return launch_divkgrad_t<float>(L); }
}  // namespace gst

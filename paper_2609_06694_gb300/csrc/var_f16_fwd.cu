// Variable-coefficient kernels: __half storage, forward sweep and div(k grad u) (instantiations only).
#include "var_launch.cuh"

namespace gst {
int launch_var_f16_fwd(const VarLaunch &L) { return launch_var_dt<__half, false>(L); }
int launch_divkgrad_f16(const VarLaunch &L) { return launch_divkgrad_t<__half>(L); }
}  // namespace gst

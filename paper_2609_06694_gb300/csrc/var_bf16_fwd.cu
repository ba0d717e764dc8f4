// Variable-coefficient kernels: __nv_bfloat16 storage, forward sweep and div(k grad u) (instantiations only).
#include "var_launch.cuh"

namespace gst {
int launch_var_bf16_fwd(const VarLaunch &L) { return launch_var_dt<__nv_bfloat16, false>(L); }
int launch_divkgrad_bf16(const VarLaunch &L) { return launch_divkgrad_t<__nv_bfloat16>(L); }
}  // namespace gst

// Variable-coefficient kernels: __nv_bfloat16 storage, adjoint sweep (instantiations only).
#include "var_launch.cuh"

namespace gst {
int launch_var_bf16_adj(const VarLaunch &L) { return launch_var_dt<__nv_bfloat16, true>(L); }
}  // namespace gst

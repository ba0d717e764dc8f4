// Variable-coefficient kernels: float storage, adjoint sweep (instantiations only).
#include "var_launch.cuh"

namespace gst {
int launch_var_f32_adj(const VarLaunch &L) { return launch_var_dt<float, true>(L); }
}  // namespace gst

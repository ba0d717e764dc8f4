// Variable-coefficient kernels: __half storage, adjoint sweep (instantiations only).
#include "var_launch.cuh"

namespace gst {
int launch_var_f16_adj(const VarLaunch &L) { return launch_var_dt<__half, true>(L); }
}  // namespace gst

"""GB300-native stencil operator library (ForgeStencil hot path, sm_103a).

The compute path is the CUDA library ``_build/libgb300stencil.so`` (built by
``paper_2609_06694_gb300.build.build()``); this package is its Python binding.  Loading is
lazy: importing the package does not need a GPU, the first library call does, and a missing
library raises instead of falling back to anything else.
"""
from .api import (  # noqa: F401
    FAMILY_FUSED2D,
    FAMILY_FUSED3D,
    FAMILY_STREAM,
    FAMILY_TENSOR,
    Batch,
    Plan,
    StencilError,
    library_path,
    stencil_abi_version,
    stencil_apply,
    stencil_apply_adjoint,
    stencil_apply_adjoint_var,
    stencil_apply_host,
    stencil_apply_reaction,
    stencil_apply_var,
    stencil_batch_info,
    stencil_batch_launch,
    stencil_batch_plan,
    stencil_batch_set_wait_limit,
    stencil_batch_status,
    stencil_geometry_class,
    stencil_launch_count,
    stencil_load_dispatch_map,
    stencil_offsets,
    stencil_plan,
    stencil_plan_get_variant,
    stencil_plan_kernel_set,
    stencil_plan_set_variant,
    stencil_set_wait_limit,
    stencil_size_class,
    stencil_strerror,
    stencil_sync_status,
    torch_dtype,
)

"""GB300-native stencil operator library (ForgeStencil hot path, sm_103a)."""

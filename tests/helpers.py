"""Shared helpers of the GPU parity tests: seeded inputs, oracle calls, error metric."""
import numpy as np

import oracle
from paper_2609_06694_gb300 import inputs

# tolerances on the max-norm relative error against the FP64 oracle, per storage type
TOL = {"f32": 1e-5, "f16": 2e-3, "bf16": 1e-2}


def relerr(got, ref):
    """max_p |got - ref| / max_p |ref|  (scale-invariant, max-norm)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = float(np.max(np.abs(ref)))
    if scale == 0.0:
        return float(np.max(np.abs(got)))
    return float(np.max(np.abs(got - ref)) / scale)


def seeded_weights(seed, n):
    """Weights of absolute sum 1 (bounded growth over many steps)."""
    return inputs.normalised_abs_weights(seed, n)


def make_input(seed, dims, dtype):
    """(storage tensor on CPU, exact stored values as float64)."""
    t = inputs.to_storage(inputs.uniform(seed, dims), dtype)
    return t, inputs.stored_values(t)


class oracle_threads:
    """Run the oracle on every host core inside the block (same bits as one thread)."""

    def __enter__(self):
        oracle.use_threads(0)
        return self

    def __exit__(self, *exc):
        oracle.use_threads(1)
        return False


def check_steps(got, pure, emu, dtype, label=""):
    """Multi-step low-precision results: the tolerance holds against pure FP64 (the primary
    number); the error against the oracle that rounds to storage after every step is printed
    as a diagnostic.  Returns (err_pure, err_emu)."""
    ep, ee = relerr(got, pure), relerr(got, emu)
    print(f"{label} {dtype}: max rel err {ep:.2e} vs pure FP64, {ee:.2e} vs per-step rounding")
    assert ep < TOL[dtype], (label, ep)
    return ep, ee


def oracle_run(x64, offs, c, bc, steps, dtype, adjoint=False):
    """FP64 reference: pure (no rounding) and emulated storage (rounded after every step)."""
    pure = oracle.run(x64, "const", bc, steps, offs=offs, coeffs=c, adjoint=adjoint)
    if dtype == "f32" or steps == 1:
        return pure, pure
    emu = oracle.run(x64, "const", bc, steps, offs=offs, coeffs=c, adjoint=adjoint,
                     round_fmt=dtype)
    return pure, emu


def periodic_slab(x64, z0, h):
    """The cells an h-deep dependency cone of plane z0 reads on a periodic 3D grid: planes
    z0-h .. z0+h (wrapped in z), each padded periodically by h cells in x and y.  A zero-
    Dirichlet sweep of the slab reproduces the periodic sweep at its middle plane's interior
    for up to h / r steps of a radius-r stencil (the ghost zeros move inward r cells a step)."""
    zi = np.arange(z0 - h, z0 + h + 1) % x64.shape[0]
    return np.pad(x64[zi], ((0, 0), (h, h), (h, h)), mode="wrap")

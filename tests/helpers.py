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


def oracle_run(x64, offs, c, bc, steps, dtype, adjoint=False):
    """FP64 reference: pure (no rounding) and emulated storage (rounded after every step)."""
    pure = oracle.run(x64, "const", bc, steps, offs=offs, coeffs=c, adjoint=adjoint)
    if dtype == "f32" or steps == 1:
        return pure, pure
    emu = oracle.run(x64, "const", bc, steps, offs=offs, coeffs=c, adjoint=adjoint,
                     round_fmt=dtype)
    return pure, emu


def cone_reference(x64, offs, c, bc, steps, point):
    """Oracle value at one cell after `steps` sweeps, from the cube of half-width steps*r
    around it (the only cells it depends on); exact for both boundary rules."""
    r = int(np.max(np.abs(offs)))
    h = steps * r
    dims = x64.shape
    if bc == "periodic":
        idx = [np.arange(p - h, p + h + 1) % n for p, n in zip(point, dims)]
        win = x64[np.ix_(*idx)]
        centre = (h,) * len(dims)
        # reads beyond the window only reach cells that do not influence the centre
        out = oracle.run(win, "const", "dirichlet", steps, offs=offs, coeffs=c)
        return out[centre]
    lo = [max(0, p - h) for p in point]
    hi = [min(n, p + h + 1) for p, n in zip(point, dims)]
    win = x64[tuple(slice(a, b) for a, b in zip(lo, hi))]
    out = oracle.run(win, "const", "dirichlet", steps, offs=offs, coeffs=c)
    return out[tuple(p - a for p, a in zip(point, lo))]

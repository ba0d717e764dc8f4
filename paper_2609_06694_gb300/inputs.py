"""Seeded synthetic inputs for the stencil workloads.

This module is the only code shared by the CUDA path's tests and the FP64 oracle.  It holds
no stencil arithmetic: it draws random fields, smooths them into the value distributions the
workloads call for, and tabulates the fixed coefficient tables those workloads name.  Every
value is produced on the host in float64 and only then cast to a storage dtype.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): element ``i`` of stream
``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``, so any element can be drawn
without drawing the ones before it.  Normals use the Box-Muller transform on pairs of
uniforms.

Workload recipes (seeds are ``workload index * 1000 + field id``):

* 2D Jacobi 512^2: input uniform[-1, 1], seed 1001.
* 3D sweeps 512^3, periodic: input uniform[-1, 1] (seed 2001 for the radius-4 star,
  2003 for the 27-point box); box weights uniform[-1, 1] normalised to sum 1 (seed 2002,
  redrawn with seed + 1 while |sum| < 0.25).
* div(k grad u) 384^3: u uniform[-1, 1] (seed 3001); k = exp(N(0, 1)) (seed 3002) smoothed by
  a periodic 5^3 box mean.
* batched 2D: per-axis side round(exp(U[ln 64, ln 2048])) (seed 4001); shape drawn from
  {star r1, star r2, box r1, box r2} (seed 4002); weights uniform[-1, 1] divided by their
  absolute sum (seed 4100 + grid index); input uniform[-1, 1] (seed 4500 + grid index).
* wave equation 256^3: velocity = N(0, 1) (seed 5001) box-filtered twice with a periodic 9^3
  mean, mapped affinely onto [1500, 4500] m/s; the "true" model multiplies it by
  1 + 0.05 exp(-|x - c|^2 / (2 * 16^2)) around the grid centre and clips to [1500, 4500];
  Ricker source at 15 Hz.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Elements ``start .. start+count-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2^-53."""
    out = np.empty(n, dtype=np.float64)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        z = splitmix64(seed, start + s, m)
        out[s:s + m] = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return out


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape))
    return (lo + (hi - lo) * uniform01(seed, n)).reshape(shape)


def normal(seed: int, shape) -> np.ndarray:
    """Standard normals by Box-Muller: element j uses uniforms 2j and 2j+1 of the stream."""
    n = int(np.prod(shape))
    u = uniform01(seed, 2 * n)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(shape)


def box_mean_periodic(a: np.ndarray, width: int) -> np.ndarray:
    """Periodic moving average of odd ``width`` along every axis (separable, via cumsum)."""
    assert width % 2 == 1
    h = width // 2
    out = np.asarray(a, dtype=np.float64)
    for ax in range(out.ndim):
        n = out.shape[ax]
        idx = np.arange(-h - 1, n + h) % n
        ext = np.take(out, idx, axis=ax)
        cs = np.cumsum(ext, axis=ax)
        hi = np.take(cs, np.arange(width, width + n), axis=ax)
        lo = np.take(cs, np.arange(0, n), axis=ax)
        out = (hi - lo) / width
    return out


def lognormal_k(seed: int, shape, smooth: int = 5) -> np.ndarray:
    """k = exp(N(0,1)) smoothed by a periodic ``smooth``^d box mean (always > 0)."""
    return box_mean_periodic(np.exp(normal(seed, shape)), smooth)


def velocity_field(seed: int, shape, vmin: float = 1500.0, vmax: float = 4500.0,
                   width: int = 9, passes: int = 2) -> np.ndarray:
    f = normal(seed, shape)
    for _ in range(passes):
        f = box_mean_periodic(f, width)
    lo, hi = float(f.min()), float(f.max())
    return vmin + (f - lo) * ((vmax - vmin) / (hi - lo))


def perturbed_velocity(v: np.ndarray, amp: float = 0.05, sigma: float = 16.0,
                       vmin: float = 1500.0, vmax: float = 4500.0) -> np.ndarray:
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in v.shape], indexing="ij")
    r2 = sum((g - (n // 2)) ** 2 for g, n in zip(grids, v.shape))
    return np.clip(v * (1.0 + amp * np.exp(-r2 / (2.0 * sigma * sigma))), vmin, vmax)


def ricker(freq: float, dt: float, nsteps: int, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = n*dt - t0, t0 = 1/f."""
    if t0 is None:
        t0 = 1.0 / freq
    tau = np.arange(nsteps, dtype=np.float64) * dt - t0
    a = (np.pi * freq * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


# Central second-derivative weights of order 2r on the unit grid (Fornberg, "Generation of
# finite difference formulas on arbitrarily spaced grids", Math. Comp. 1988), index k = |offset|.
SECOND_DERIVATIVE = {
    1: [Fraction(-2), Fraction(1)],
    2: [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)],
    3: [Fraction(-49, 18), Fraction(3, 2), Fraction(-3, 20), Fraction(1, 90)],
    4: [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560)],
}


def laplacian_weight(offset, radius: int) -> float:
    """Weight of a star offset in the order-2r Laplacian (sum of 1D second derivatives)."""
    w = SECOND_DERIVATIVE[radius]
    nz = [d for d in offset if d != 0]
    if not nz:
        return float(len(offset) * w[0])
    if len(nz) != 1 or abs(nz[0]) > radius:
        raise ValueError("not a star offset of this radius")
    return float(w[abs(nz[0])])


def laplacian_coeffs(offsets: np.ndarray, radius: int) -> np.ndarray:
    return np.array([laplacian_weight(tuple(int(x) for x in o), radius) for o in offsets],
                    dtype=np.float64)


def normalised_sum_weights(seed: int, n: int, min_abs_sum: float = 0.25):
    """uniform[-1,1] weights divided by their sum; the seed advances while |sum| is small."""
    while True:
        w = uniform(seed, (n,))
        s = float(w.sum())
        if abs(s) >= min_abs_sum:
            return w / s, seed
        seed += 1


def normalised_abs_weights(seed: int, n: int) -> np.ndarray:
    """uniform[-1,1] weights divided by the sum of their absolute values."""
    w = uniform(seed, (n,))
    return w / float(np.abs(w).sum())


BATCH_SHAPES = [("star", 1), ("star", 2), ("box", 1), ("box", 2)]


def batched_grid_specs(n_grids: int = 256, lo: int = 64, hi: int = 2048,
                       seed_sides: int = 4001, seed_shapes: int = 4002):
    """Side lengths (ny, nx) log-uniform in [lo, hi] per axis and a shape per grid."""
    u = uniform01(seed_sides, 2 * n_grids)
    sides = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    pick = np.floor(uniform01(seed_shapes, n_grids) * len(BATCH_SHAPES)).astype(np.int64)
    specs = []
    for g in range(n_grids):
        shape, radius = BATCH_SHAPES[int(pick[g])]
        specs.append({"ny": int(sides[2 * g]), "nx": int(sides[2 * g + 1]),
                      "shape": shape, "radius": radius,
                      "weight_seed": 4100 + g, "input_seed": 4500 + g})
    return specs


def to_storage(x: np.ndarray, dtype: str):
    """Cast float64 values to a storage dtype; returns a CPU torch tensor."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    if dtype == "f32":
        return t.to(torch.float32)
    if dtype == "f16":
        return t.to(torch.float16)
    if dtype == "bf16":
        return t.to(torch.float32).to(torch.bfloat16)
    raise ValueError(dtype)


def stored_values(t) -> np.ndarray:
    """The exact stored values of a storage tensor, upcast to float64."""
    import torch
    return t.detach().to("cpu").to(torch.float64).numpy()

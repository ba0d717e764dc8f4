"""FP64 stencil oracle (TEST INFRASTRUCTURE ONLY).

Python access to the plain C oracle in ``stencil_oracle.c`` (single-threaded by default;
``use_threads`` switches to the same source built with OpenMP, which gives the same bits).
Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference
leg may import this package.  It shares no code with the CUDA library and never imports it.

Functions take and return float64 numpy arrays in row-major layout (last axis fastest); grid
dimensions are given slowest axis first.  Paper references: Sec. 2.1 (stencil update, offset
sets, variable coefficients, precision) and Sec. 4.3 (fused time steps); the readings taken
where the paper is silent are listed in the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_LIB_MT = os.path.join(_LIB_DIR, "liboracle_mt.so")  # the same source with OpenMP

STAR, BOX, DIAMOND = 0, 1, 2
SHAPES = {"star": STAR, "box": BOX, "diamond": DIAMOND}
DIRICHLET0, PERIODIC = 0, 1
BCS = {"dirichlet": DIRICHLET0, "periodic": PERIODIC}
ROUND = {"none": 0, "f64": 0, "f32": 1, "f16": 2, "bf16": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, so every host gives the same bits):
    a single-threaded library and the same source with OpenMP (cell loops over host threads,
    identical results)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    for lib, extra in ((_LIB, []), (_LIB_MT, ["-fopenmp"])):
        if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(_SRC):
            continue
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC",
                               "-shared"] + extra + [_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, lib)
    return _LIB


_libs = {}
_threads = 1


def use_threads(n: int = 0) -> int:
    """Run the oracle's cell loops on n host threads from now on (0: every core, 1: the
    single-threaded build).  Results are bit-for-bit the same; returns the thread count."""
    global _threads
    if n == 1:
        _threads = 1
        return 1
    _threads = int(_open(_LIB_MT).orc_set_threads(int(n)))
    return _threads


def threads() -> int:
    """Host threads the oracle currently uses."""
    return _threads


def _L():
    return _open(_LIB if _threads == 1 else _LIB_MT)


def _open(path):
    if path not in _libs:
        build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        lib.orc_offsets.argtypes = [I, I, I, P]
        lib.orc_offsets.restype = I64
        for name in ("orc_sweep_const", "orc_sweep_var", "orc_sweep_const_adjoint",
                     "orc_sweep_var_adjoint"):
            getattr(lib, name).argtypes = [I, P, I64, P, P, I, P, P]
            getattr(lib, name).restype = None
        lib.orc_sweep_const_points.argtypes = [I, P, I64, P, P, I, P, I64, P, P]
        lib.orc_divkgrad.argtypes = [I, P, P, I, P, P]
        lib.orc_divkgrad_weights.argtypes = [I, P, P, I, P]
        lib.orc_round_scalar.argtypes = [D, I]
        lib.orc_round_scalar.restype = D
        lib.orc_round.argtypes = [I64, P, I]
        lib.orc_run.argtypes = [I, P, I, I, I64, P, P, I, I, I, P, P]
        lib.orc_run.restype = I
        lib.orc_wave_forward.argtypes = [P, I64, P, P, P, D, D, I, I64, P, I64, P, P]
        lib.orc_wave_forward.restype = I
        lib.orc_misfit.argtypes = [I64, P, P]
        lib.orc_misfit.restype = D
        lib.orc_wave_gradient.argtypes = [P, I64, P, P, P, D, D, I, I64, P, I64, P, I, P, P]
        lib.orc_wave_gradient.restype = I
        lib.orc_reaction_run.argtypes = [I, P, I64, P, P, I, I, D, D, D, I, P, P]
        lib.orc_reaction_run.restype = I
        lib.orc_set_threads.argtypes = [I]
        lib.orc_set_threads.restype = I
        _libs[path] = lib
    return _libs[path]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(shape):
    return np.ascontiguousarray(shape, dtype=np.int64)


def offsets(ndim: int, shape, radius: int) -> np.ndarray:
    """Offset set in canonical order (lexicographic, slowest axis first), shape (n, ndim)."""
    s = SHAPES[shape] if isinstance(shape, str) else int(shape)
    n = _L().orc_offsets(ndim, s, radius, None)
    if n < 0:
        raise ValueError("bad offset-set request")
    out = np.zeros((n, ndim), dtype=np.int32)
    _L().orc_offsets(ndim, s, radius, _ptr(out))
    return out


def _bc(bc):
    return BCS[bc] if isinstance(bc, str) else int(bc)


def sweep_const(x, offs, coeffs, bc):
    x = _f64(x)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    c = _f64(coeffs)
    out = np.empty_like(x)
    _L().orc_sweep_const(x.ndim, _ptr(_dims(x.shape)), len(offs), _ptr(offs), _ptr(c), _bc(bc),
                         _ptr(x), _ptr(out))
    return out


def sweep_const_points(x, offs, coeffs, bc, linear_indices):
    x = _f64(x)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    c = _f64(coeffs)
    sel = np.ascontiguousarray(linear_indices, dtype=np.int64)
    out = np.empty(len(sel), dtype=np.float64)
    _L().orc_sweep_const_points(x.ndim, _ptr(_dims(x.shape)), len(offs), _ptr(offs), _ptr(c),
                                _bc(bc), _ptr(x), len(sel), _ptr(sel), _ptr(out))
    return out


def sweep_var(x, offs, w, bc):
    """w: array of shape (npts, *x.shape)."""
    x = _f64(x)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    w = _f64(w)
    assert w.shape == (len(offs),) + x.shape
    out = np.empty_like(x)
    _L().orc_sweep_var(x.ndim, _ptr(_dims(x.shape)), len(offs), _ptr(offs), _ptr(w), _bc(bc),
                       _ptr(x), _ptr(out))
    return out


def sweep_const_adjoint(y, offs, coeffs, bc):
    y = _f64(y)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    c = _f64(coeffs)
    out = np.empty_like(y)
    _L().orc_sweep_const_adjoint(y.ndim, _ptr(_dims(y.shape)), len(offs), _ptr(offs), _ptr(c),
                                 _bc(bc), _ptr(y), _ptr(out))
    return out


def sweep_var_adjoint(y, offs, w, bc):
    y = _f64(y)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    w = _f64(w)
    assert w.shape == (len(offs),) + y.shape
    out = np.empty_like(y)
    _L().orc_sweep_var_adjoint(y.ndim, _ptr(_dims(y.shape)), len(offs), _ptr(offs), _ptr(w),
                               _bc(bc), _ptr(y), _ptr(out))
    return out


def divkgrad(u, k, bc):
    u = _f64(u)
    k = _f64(k)
    assert u.shape == k.shape
    out = np.empty_like(u)
    _L().orc_divkgrad(u.ndim, _ptr(_dims(u.shape)), _ptr(k), _bc(bc), _ptr(u), _ptr(out))
    return out


def divkgrad_weights(k, bc):
    """Per-offset coefficient arrays of div(k grad .) over the star-1 offsets (canonical)."""
    k = _f64(k)
    n = 2 * k.ndim + 1
    w = np.empty((n,) + k.shape, dtype=np.float64)
    _L().orc_divkgrad_weights(k.ndim, _ptr(_dims(k.shape)), _ptr(k), _bc(bc), _ptr(w))
    return w


def round_to(x, fmt: str):
    """Round float64 values to f32 / f16 / bf16 (nearest, ties to even); result as float64."""
    x = _f64(x).copy()
    _L().orc_round(x.size, _ptr(x), ROUND[fmt])
    return x


def round_scalar(x: float, fmt: str) -> float:
    return _L().orc_round_scalar(float(x), ROUND[fmt])


_KIND = {"const": 0, "var": 1, "divkgrad": 2}


def run(x, kind, bc, steps, *, offs=None, coeffs=None, adjoint=False, round_fmt="none"):
    """``steps`` applications of A (or A^T), rounding to ``round_fmt`` after each step.

    kind='const': coeffs = 1-D array, one per offset; kind='var': coeffs = (npts, *shape);
    kind='divkgrad': coeffs = k (same shape as x), offs ignored.
    """
    x = _f64(x)
    ndim = x.ndim
    if kind == "divkgrad":
        offs = np.zeros((1, ndim), dtype=np.int32)
        npts = 0
    else:
        offs = np.ascontiguousarray(offs, dtype=np.int32)
        npts = len(offs)
    c = _f64(coeffs)
    out = np.empty_like(x)
    rc = _L().orc_run(ndim, _ptr(_dims(x.shape)), _KIND[kind], int(bool(adjoint)), npts,
                      _ptr(offs), _ptr(c), _bc(bc), int(steps), ROUND[round_fmt], _ptr(x),
                      _ptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_run failed: {rc}")
    return out


def reaction(x, offs, coeffs, bc, steps, dt, c1, c3, round_fmt="none"):
    """``steps`` reaction-diffusion steps u + dt (A u + c1 u + c3 u^3), rounding to
    ``round_fmt`` after each step."""
    x = _f64(x)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    c = _f64(coeffs)
    out = np.empty_like(x)
    rc = _L().orc_reaction_run(x.ndim, _ptr(_dims(x.shape)), len(offs), _ptr(offs), _ptr(c),
                               _bc(bc), int(steps), float(dt), float(c1), float(c3),
                               ROUND[round_fmt], _ptr(x), _ptr(out))
    if rc != 0:
        raise RuntimeError("orc_reaction_run failed")
    return out


def wave_forward(v, offs, coeffs, h, dt, nsteps, src, wavelet, rz, return_last=False):
    """Receiver traces (nsteps, ny, nx) of the leapfrog run; optionally also u^N."""
    v = _f64(v)
    assert v.ndim == 3
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    c = _f64(coeffs)
    wl = _f64(wavelet)
    assert len(wl) >= nsteps
    nz, ny, nx = v.shape
    src_lin = (int(src[0]) * ny + int(src[1])) * nx + int(src[2])
    traces = np.empty((nsteps, ny, nx), dtype=np.float64)
    last = np.empty_like(v) if return_last else None
    rc = _L().orc_wave_forward(_ptr(_dims(v.shape)), len(offs), _ptr(offs), _ptr(c), _ptr(v),
                               float(h), float(dt), int(nsteps), src_lin, _ptr(wl), int(rz),
                               _ptr(traces), _ptr(last) if last is not None else None)
    if rc != 0:
        raise RuntimeError("orc_wave_forward failed")
    return (traces, last) if return_last else traces


def misfit(traces, observed) -> float:
    t = _f64(traces)
    o = _f64(observed)
    assert t.shape == o.shape
    return _L().orc_misfit(t.size, _ptr(t), _ptr(o))


def wave_gradient(v, offs, coeffs, h, dt, nsteps, src, wavelet, rz, observed, ck_every=0):
    """(J, g): misfit and its velocity gradient by the discrete adjoint."""
    v = _f64(v)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    c = _f64(coeffs)
    wl = _f64(wavelet)
    obs = _f64(observed)
    nz, ny, nx = v.shape
    assert obs.shape == (nsteps, ny, nx)
    src_lin = (int(src[0]) * ny + int(src[1])) * nx + int(src[2])
    g = np.empty_like(v)
    J = np.zeros(1, dtype=np.float64)
    rc = _L().orc_wave_gradient(_ptr(_dims(v.shape)), len(offs), _ptr(offs), _ptr(c), _ptr(v),
                                float(h), float(dt), int(nsteps), src_lin, _ptr(wl), int(rz),
                                _ptr(obs), int(ck_every), _ptr(g), _ptr(J))
    if rc != 0:
        raise RuntimeError("orc_wave_gradient failed")
    return float(J[0]), g

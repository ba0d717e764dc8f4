"""Thin Python binding of the C ABI in include/stencil.h.

Every function keeps the C name and only marshals arguments: torch tensors become device
pointers, the current torch stream becomes the cudaStream_t, status codes become
``StencilError``.  All stencil arithmetic runs in the CUDA kernels of libgb300stencil.so; if
the library is missing, the first call raises instead of computing anything elsewhere.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SHAPES = {"star": 0, "box": 1, "diamond": 2, "custom": 3}
DTYPES = {"f32": 0, "f16": 1, "bf16": 2}
BOUNDARIES = {"dirichlet": 0, "periodic": 1}
KINDS = {"const": 0, "var": 1, "divkgrad": 2}
FAMILY_STREAM = 1
FAMILY_FUSED2D = 2
FAMILY_FUSED3D = 3
FAMILY_TENSOR = 4

_ERRORS = {-1: "BADARG", -2: "UNSUPPORTED", -3: "OOM", -4: "CUDA", -5: "TIMEOUT", -6: "BOUNDS"}


class StencilError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: STENCIL_ERR_{_ERRORS.get(code, code)} "
                         f"({_lib().stencil_strerror(code).decode()})")


class stencil_variant(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
                ("vec_y", ctypes.c_int), ("z_chunk", ctypes.c_int), ("fuse", ctypes.c_int),
                ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("stages", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class stencil_batch_item(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


_LIB = None
DISPATCH_MAP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dispatch_map.txt")


def library_path() -> str:
    return _build.LIB


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA stencil library is not built ({path} is missing); "
                           "run paper_2609_06694_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "stencil_plan": ([ctypes.POINTER(P), I, P, I, I, I, P, I64, P, I, I], I),
        "stencil_plan_kernel_set": ([P, P, P], I),
        "stencil_set_wait_limit": ([P, ctypes.c_double, I], I),
        "stencil_apply_reaction": ([P, P, P, I, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, P], I),
        "stencil_offsets": ([P, P, I64, ctypes.POINTER(I64)], I),
        "stencil_destroy": ([P], I),
        "stencil_apply": ([P, P, P, I, P], I),
        "stencil_apply_adjoint": ([P, P, P, I, P], I),
        "stencil_apply_var": ([P, P, P, P, I, P], I),
        "stencil_apply_adjoint_var": ([P, P, P, P, I, P], I),
        "stencil_apply_host": ([P, P, P, I, P], I),
        "stencil_sync_status": ([P, P], I),
        "stencil_batch_plan": ([ctypes.POINTER(P), P, I, I], I),
        "stencil_batch_plan_tiles": ([ctypes.POINTER(P), P, I, I, I, I, I], I),
        "stencil_batch_launch": ([P, P], I),
        "stencil_batch_status": ([P, P], I),
        "stencil_batch_destroy": ([P], I),
        "stencil_batch_set_wait_limit": ([P, ctypes.c_double, I], I),
        "stencil_batch_info": ([P, P, P, P], I),
        "stencil_plan_get_variant": ([P, ctypes.POINTER(stencil_variant)], I),
        "stencil_plan_set_variant": ([P, ctypes.POINTER(stencil_variant)], I),
        "stencil_load_dispatch_map": ([ctypes.c_char_p], I),
        "stencil_size_class": ([I64], I),
        "stencil_geometry_class": ([I, P], I),
        "stencil_launch_count": ([], ctypes.c_uint64),
        "stencil_strerror": ([I], ctypes.c_char_p),
        "stencil_abi_version": ([], I),
    }
    for name, (args, res) in sig.items():
        if hasattr(lib, name):
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
    _LIB = lib
    # the dispatch map written by the autotuner ships with the package
    if os.path.exists(DISPATCH_MAP):
        lib.stencil_load_dispatch_map(DISPATCH_MAP.encode())
    return lib


def _check(rc: int, where: str):
    if rc != 0:
        raise StencilError(rc, where)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


_TORCH_DTYPE = None


def torch_dtype(dtype: str):
    import torch
    return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dtype]


class Plan:
    """Owns a ``stencil_handle``; destroyed with the object."""

    def __init__(self, handle: int, ndim, dims, shape, radius, kind, dtype, boundary):
        self.handle = ctypes.c_void_p(handle)
        self.ndim, self.dims = ndim, tuple(int(d) for d in dims)
        self.shape, self.radius, self.kind = shape, radius, kind
        self.dtype, self.boundary = dtype, boundary

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _LIB is not None:
            _LIB.stencil_destroy(h)
            self.handle = None

    @property
    def variant(self) -> dict:
        return stencil_plan_get_variant(self)

    def _check_tensor(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != torch_dtype(self.dtype) or tuple(t.shape) != self.dims:
            raise ValueError(f"{name}: expected {self.dims} {self.dtype}, got {tuple(t.shape)} {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")


def stencil_plan(ndim, dims, shape, radius, kind="const", coeffs=None, dtype="f32",
                 boundary="dirichlet", offsets=None) -> Plan:
    """shape "custom" takes `offsets`, an (n, ndim) integer array of distinct offsets (slowest
    component first), with `coeffs` in the same order."""
    lib = _lib()
    d = (ctypes.c_int64 * ndim)(*[int(x) for x in dims])
    if coeffs is not None:
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        cptr, n = c.ctypes.data_as(ctypes.c_void_p), len(c)
    else:
        c, cptr, n = None, None, 0
    optr = None
    if offsets is not None:
        o = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1, ndim)
        optr = o.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p()
    rc = lib.stencil_plan(ctypes.byref(h), ndim, d, SHAPES[shape], int(radius), KINDS[kind], cptr,
                          n, optr, DTYPES[dtype], BOUNDARIES[boundary])
    _check(rc, "stencil_plan")
    return Plan(h.value, ndim, dims, shape, radius, kind, dtype, boundary)


def stencil_plan_kernel_set(plan: Plan):
    """(shape name, radius) of the compiled offset set the plan's kernels run."""
    s, r = ctypes.c_int(), ctypes.c_int()
    _check(_lib().stencil_plan_kernel_set(plan.handle, ctypes.byref(s), ctypes.byref(r)),
           "stencil_plan_kernel_set")
    return {v: k for k, v in SHAPES.items()}[s.value], r.value


def stencil_apply_reaction(plan: Plan, inp, out, steps, dt, c1, c3, stream=None):
    """`steps` fused reaction-diffusion steps u + dt (A u + c1 u + c3 u^3)."""
    plan._check_tensor(inp, "in")
    plan._check_tensor(out, "out")
    _check(_lib().stencil_apply_reaction(plan.handle, ctypes.c_void_p(inp.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), int(steps), float(dt),
                                         float(c1), float(c3), _stream_ptr(stream)),
           "stencil_apply_reaction")
    return out


def stencil_set_wait_limit(plan: Plan, seconds: float, phantom_arrivals: int = 0):
    _check(_lib().stencil_set_wait_limit(plan.handle, float(seconds), int(phantom_arrivals)),
           "stencil_set_wait_limit")


def stencil_offsets(plan: Plan) -> np.ndarray:
    lib = _lib()
    n = ctypes.c_int64()
    _check(lib.stencil_offsets(plan.handle, None, 0, ctypes.byref(n)), "stencil_offsets")
    out = np.zeros((n.value, plan.ndim), dtype=np.int32)
    _check(lib.stencil_offsets(plan.handle, out.ctypes.data_as(ctypes.c_void_p), n.value,
                               ctypes.byref(n)), "stencil_offsets")
    return out


def stencil_apply(plan: Plan, inp, out, steps=1, stream=None):
    plan._check_tensor(inp, "in")
    plan._check_tensor(out, "out")
    _check(_lib().stencil_apply(plan.handle, ctypes.c_void_p(inp.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), int(steps), _stream_ptr(stream)),
           "stencil_apply")
    return out


def stencil_apply_adjoint(plan: Plan, inp, out, steps=1, stream=None):
    plan._check_tensor(inp, "in")
    plan._check_tensor(out, "out")
    _check(_lib().stencil_apply_adjoint(plan.handle, ctypes.c_void_p(inp.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), int(steps),
                                        _stream_ptr(stream)), "stencil_apply_adjoint")
    return out


def _coeff_ptrs(plan: Plan, arrays):
    # the C entry point reads exactly this many pointers, so the count is checked here
    want = 1 if plan.kind == "divkgrad" else len(stencil_offsets(plan))
    if len(arrays) != want:
        raise ValueError(f"expected {want} coefficient arrays, got {len(arrays)}")
    for i, a in enumerate(arrays):
        plan._check_tensor(a, f"coeff_arrays[{i}]")
    return (ctypes.c_void_p * len(arrays))(*[a.data_ptr() for a in arrays])


def stencil_apply_var(plan: Plan, inp, coeff_arrays, out, steps=1, stream=None):
    plan._check_tensor(inp, "in")
    plan._check_tensor(out, "out")
    ptrs = _coeff_ptrs(plan, coeff_arrays)
    _check(_lib().stencil_apply_var(plan.handle, ctypes.c_void_p(inp.data_ptr()), ptrs,
                                    ctypes.c_void_p(out.data_ptr()), int(steps),
                                    _stream_ptr(stream)), "stencil_apply_var")
    return out


def stencil_apply_adjoint_var(plan: Plan, inp, coeff_arrays, out, steps=1, stream=None):
    plan._check_tensor(inp, "in")
    plan._check_tensor(out, "out")
    ptrs = _coeff_ptrs(plan, coeff_arrays)
    _check(_lib().stencil_apply_adjoint_var(plan.handle, ctypes.c_void_p(inp.data_ptr()), ptrs,
                                            ctypes.c_void_p(out.data_ptr()), int(steps),
                                            _stream_ptr(stream)), "stencil_apply_adjoint_var")
    return out


def stencil_apply_host(plan: Plan, inp_host, out_host, steps=1, stream=None):
    """Host tensors (ideally pinned) in and out; copies happen inside the call."""
    for t, name in ((inp_host, "in"), (out_host, "out")):
        if t.is_cuda or not t.is_contiguous() or tuple(t.shape) != plan.dims \
                or t.dtype != torch_dtype(plan.dtype):
            raise ValueError(f"{name} must be a contiguous host tensor of the plan's shape/dtype")
    _check(_lib().stencil_apply_host(plan.handle, ctypes.c_void_p(inp_host.data_ptr()),
                                     ctypes.c_void_p(out_host.data_ptr()), int(steps),
                                     _stream_ptr(stream)), "stencil_apply_host")
    return out_host


def stencil_sync_status(plan: Plan, stream=None) -> int:
    return _lib().stencil_sync_status(plan.handle, _stream_ptr(stream))


def stencil_plan_get_variant(plan: Plan) -> dict:
    v = stencil_variant()
    _check(_lib().stencil_plan_get_variant(plan.handle, ctypes.byref(v)), "get_variant")
    return v.as_dict()


def stencil_plan_set_variant(plan: Plan, **kw):
    v = stencil_variant()
    _check(_lib().stencil_plan_get_variant(plan.handle, ctypes.byref(v)), "get_variant")
    for k, val in kw.items():
        setattr(v, k, int(val))
    _check(_lib().stencil_plan_set_variant(plan.handle, ctypes.byref(v)), "set_variant")


def stencil_load_dispatch_map(path):
    _check(_lib().stencil_load_dispatch_map(path.encode() if path else None),
           "stencil_load_dispatch_map")


def stencil_size_class(cells: int) -> int:
    return _lib().stencil_size_class(int(cells))


def stencil_geometry_class(ndim: int, dims) -> int:
    d = (ctypes.c_int64 * ndim)(*[int(x) for x in dims])
    rc = _lib().stencil_geometry_class(int(ndim), d)
    _check(min(rc, 0), "stencil_geometry_class")
    return rc


def stencil_launch_count() -> int:
    return int(_lib().stencil_launch_count())


def stencil_strerror(code: int) -> str:
    return _lib().stencil_strerror(int(code)).decode()


def stencil_abi_version() -> int:
    return _lib().stencil_abi_version()


class Batch:
    """Owns a ``stencil_batch``; keeps the plans and tensors it references alive."""

    def __init__(self, handle, keep):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _LIB is not None:
            _LIB.stencil_batch_destroy(h)
            self.handle = None


def stencil_batch_plan(items, steps, tile_y=0, tile_x=0, fuse=0) -> Batch:
    """items: sequence of (Plan, in_tensor, out_tensor); all 2D const plans.  tile_y, tile_x,
    fuse: the launch shape (all 0: the dispatch map's shape for the storage type, else the
    library default for any field left 0)."""
    lib = _lib()
    arr = (stencil_batch_item * len(items))()
    for i, (plan, inp, out) in enumerate(items):
        plan._check_tensor(inp, f"items[{i}].in")
        plan._check_tensor(out, f"items[{i}].out")
        arr[i].plan = plan.handle.value
        arr[i].in_ = inp.data_ptr()
        arr[i].out = out.data_ptr()
    h = ctypes.c_void_p()
    if tile_y == 0 and tile_x == 0 and fuse == 0:
        # the launch shape of the dispatch map's "batch" line for the storage type
        _check(lib.stencil_batch_plan(ctypes.byref(h), arr, len(items), int(steps)),
               "stencil_batch_plan")
    else:
        _check(lib.stencil_batch_plan_tiles(ctypes.byref(h), arr, len(items), int(steps),
                                            int(tile_y), int(tile_x), int(fuse)),
               "stencil_batch_plan")
    return Batch(h.value, list(items))


def stencil_batch_launch(batch: Batch, stream=None):
    _check(_lib().stencil_batch_launch(batch.handle, _stream_ptr(stream)), "stencil_batch_launch")


def stencil_batch_status(batch: Batch, stream=None) -> int:
    return _lib().stencil_batch_status(batch.handle, _stream_ptr(stream))


def stencil_batch_set_wait_limit(batch: Batch, seconds: float, phantom_arrivals: int = 0):
    _check(_lib().stencil_batch_set_wait_limit(batch.handle, float(seconds),
                                               int(phantom_arrivals)), "set_wait_limit")


def stencil_batch_info(batch: Batch) -> dict:
    nt, nb, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib().stencil_batch_info(batch.handle, ctypes.byref(nt), ctypes.byref(nb),
                                     ctypes.byref(g)), "stencil_batch_info")
    return {"tiles": nt.value, "blocks": nb.value, "graph": bool(g.value)}

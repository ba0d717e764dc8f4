"""Binding of include/wave.h (acoustic wave equation, misfit and adjoint velocity gradient)
and its torch.autograd.Function.  Argument marshalling only; all arithmetic is on the GPU."""
from __future__ import annotations

import ctypes

import numpy as np

from .api import StencilError, _check, _lib, _stream_ptr


def _wlib():
    lib = _lib()
    if not getattr(lib, "_wave_sigs", False):
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.wave_plan.argtypes = [ctypes.POINTER(P), P, I, P, D, D, I, P, P, I64, I]
        lib.wave_plan.restype = I
        lib.wave_forward.argtypes = [P, P, P, P]
        lib.wave_forward.restype = I
        lib.wave_misfit.argtypes = [P, P, P, P, P]
        lib.wave_misfit.restype = I
        lib.wave_gradient.argtypes = [P, P, P, P, P, P, P]
        lib.wave_gradient.restype = I
        lib.wave_destroy.argtypes = [P]
        lib.wave_destroy.restype = I
        lib.wave_sync_status.argtypes = [P, P]
        lib.wave_sync_status.restype = I
        lib._wave_sigs = True
    return lib


class WavePlan:
    def __init__(self, handle, dims, nsteps):
        self.handle = ctypes.c_void_p(handle)
        self.dims = tuple(int(d) for d in dims)
        self.nsteps = int(nsteps)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _wlib().wave_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def trace_shape(self):
        return (self.nsteps, self.dims[1], self.dims[2])


def wave_plan(dims, radius, lap, h, dt, nsteps, src, wavelet, rz, ck_every) -> WavePlan:
    lib = _wlib()
    d = (ctypes.c_int64 * 3)(*[int(x) for x in dims])
    lap = np.ascontiguousarray(lap, dtype=np.float64)
    wl = np.ascontiguousarray(wavelet, dtype=np.float64)
    if len(lap) != 6 * radius + 1 or len(wl) < nsteps:
        raise ValueError("lap must hold 6r+1 weights and wavelet at least nsteps values")
    sr = (ctypes.c_int64 * 3)(*[int(x) for x in src])
    hnd = ctypes.c_void_p()
    _check(lib.wave_plan(ctypes.byref(hnd), d, int(radius), lap.ctypes.data_as(ctypes.c_void_p),
                         float(h), float(dt), int(nsteps), sr,
                         wl.ctypes.data_as(ctypes.c_void_p), int(rz), int(ck_every)), "wave_plan")
    return WavePlan(hnd.value, dims, nsteps)


def _f32(t, shape, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
        raise ValueError(f"{name}: contiguous CUDA float32 tensor of shape {shape} expected")
    return ctypes.c_void_p(t.data_ptr())


def wave_forward(plan: WavePlan, v, traces, stream=None):
    _check(_wlib().wave_forward(plan.handle, _f32(v, plan.dims, "v"),
                                _f32(traces, plan.trace_shape, "traces"), _stream_ptr(stream)),
           "wave_forward")
    return traces


def wave_misfit(plan: WavePlan, traces, observed, J, stream=None):
    import torch
    assert J.dtype == torch.float64 and J.is_cuda and J.numel() >= 1
    _check(_wlib().wave_misfit(plan.handle, _f32(traces, plan.trace_shape, "traces"),
                               _f32(observed, plan.trace_shape, "observed"),
                               ctypes.c_void_p(J.data_ptr()), _stream_ptr(stream)), "wave_misfit")
    return J


def wave_gradient(plan: WavePlan, v, observed, traces, J, g, stream=None):
    import torch
    assert J.dtype == torch.float64 and J.is_cuda
    assert g.dtype == torch.float64 and g.is_cuda and tuple(g.shape) == plan.dims
    _check(_wlib().wave_gradient(plan.handle, _f32(v, plan.dims, "v"),
                                 _f32(observed, plan.trace_shape, "observed"),
                                 _f32(traces, plan.trace_shape, "traces"),
                                 ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                 _stream_ptr(stream)), "wave_gradient")
    return J, g


def wave_sync_status(plan: WavePlan, stream=None) -> int:
    return _wlib().wave_sync_status(plan.handle, _stream_ptr(stream))


def _autograd_classes():
    import torch

    class WaveMisfit(torch.autograd.Function):
        """J(v) = 1/2 ||traces(v) - observed||^2 with dJ/dv from the hand-written adjoint.

        The forward pass runs the checkpointed forward and the adjoint sweep together
        (wave_gradient) and keeps g, so backward only scales it by the incoming gradient."""

        @staticmethod
        def forward(ctx, v, plan, observed):
            traces = torch.empty(plan.trace_shape, dtype=torch.float32, device=v.device)
            J = torch.zeros(1, dtype=torch.float64, device=v.device)
            g = torch.empty(plan.dims, dtype=torch.float64, device=v.device)
            wave_gradient(plan, v.contiguous(), observed, traces, J, g)
            ctx.save_for_backward(g)
            return J[0]

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return (grad_out.to(torch.float64) * g).to(torch.float32), None, None

    return WaveMisfit


def WaveMisfit():
    """The torch.autograd.Function class (created lazily so importing needs no torch)."""
    return _autograd_classes()

"""GPU test of stencil_apply_noalloc, the sweep entry point for callers that may not allocate
device memory (frameworks whose memory pool owns the GPU, latency-critical loops that cannot
absorb cudaMalloc's synchronisation).  Called directly through the C ABI, it must give the same result as
stencil_apply on two calls in a row (the shared fixed scratch array keeps the previous call's
contents, which must not matter), and must refuse a grid larger than its fixed scratch.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import TOL, make_input, relerr, seeded_weights
from paper_2609_06694_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def noalloc():
    gs.build.build()
    torch.cuda.set_device(0)
    fn = api._lib().stencil_apply_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def call(fn, plan, x, y, steps):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
              int(steps), stream)


CASES = [
    # ndim, dims, shape, radius, dtype, boundary, steps
    (2, (512, 512), "star", 1, "f32", "dirichlet", 10),   # fused groups of 8 + 2
    (3, (40, 64, 128), "star", 2, "f32", "periodic", 5),  # one launch per step
    (2, (200, 136), "box", 1, "bf16", "dirichlet", 7),
]


@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_stencil_apply_twice(noalloc, case):
    ndim, dims, shape, r, dtype, bc, steps = case
    offs = oracle.offsets(ndim, shape, r)
    c = np.full(len(offs), 0.2) if shape == "star" and r == 1 else seeded_weights(61, len(offs))
    plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, dtype, bc)
    x, _ = make_input(62, dims, dtype)
    xd = x.cuda()
    ref = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, ref, steps)
    for _ in range(2):  # the second call starts from the first call's leftover scratch
        y = torch.full_like(xd, float("nan"))
        assert call(noalloc, plan, xd, y, steps) == 0
        assert gs.stencil_sync_status(plan) == 0
        got = inputs.stored_values(y)
        assert relerr(got, inputs.stored_values(ref)) < TOL[dtype]
        assert torch.equal(y, ref)  # same kernels, same grouping


def test_noalloc_rejects_grids_beyond_its_scratch(noalloc):
    dims = (256, 256, 256)  # 64 MiB of f32 > 16 MiB
    plan = gs.stencil_plan(3, dims, "star", 1, "const", np.ones(7), "f32", "periodic")
    x = torch.zeros(dims, device="cuda")
    y = torch.empty_like(x)
    assert call(noalloc, plan, x, y, 2) == -1  # STENCIL_ERR_BADARG, nothing launched
    torch.cuda.synchronize()

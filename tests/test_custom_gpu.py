"""GPU parity of caller-given offset sets (STENCIL_CUSTOM, the sweep of Sec. 2.1 over an
arbitrary offset set S) against the FP64 oracle, which sweeps the same offsets in the caller's
order: single sweeps, multi-step runs and the adjoint, both boundary rules, f32 and 16-bit
storage, 2D and 3D, and custom grids inside a batched launch."""
import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import TOL, make_input, oracle_run, relerr
from paper_2609_06694_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


def _subset(ndim, shape, r, k, seed):
    """k offsets of a compiled set, drawn with a seed, in a shuffled order."""
    full = oracle.offsets(ndim, shape, r)
    idx = np.random.default_rng(seed).permutation(len(full))[:k]
    return full[idx]


CASES = {
    # a one-sided (upwind) 3D set: runs on the star r2 kernel
    "upwind3d": (3, (21, 35, 264), np.array([(0, 0, 0), (0, 0, -1), (0, 0, -2), (0, -1, 0),
                                             (-1, 0, 0)]), ("star", 2)),
    # 20 of the 125 box r2 offsets
    "sparse_box2": (3, (13, 35, 136), _subset(3, "box", 2, 20, 5), ("box", 2)),
    # an off-axis set inside the diamond r2
    "diag3d": (3, (17, 30, 200), np.array([(1, 1, 0), (0, 0, 0), (-1, 0, 1), (0, -1, -1)]),
               ("diamond", 2)),
    # 2D: 11 of the 49 box r3 offsets
    "sparse_box3_2d": (2, (53, 264), _subset(2, "box", 3, 11, 7), ("box", 3)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_custom_set_matches_oracle(name, dtype, bc):
    ndim, dims, offs, kernel_set = CASES[name]
    c = inputs.uniform(401, (len(offs),))
    plan = gs.stencil_plan(ndim, dims, "custom", 4, "const", c, dtype, bc, offsets=offs)
    assert gs.stencil_plan_kernel_set(plan) == kernel_set
    x, x64 = make_input(402, dims, dtype)
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    assert relerr(inputs.stored_values(y), oracle.sweep_const(x64, offs, c, bc)) < TOL[dtype]
    gs.stencil_apply_adjoint(plan, xd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    assert relerr(inputs.stored_values(y), oracle.sweep_const_adjoint(x64, offs, c, bc)) < TOL[dtype]
    # three steps: weights of absolute sum 1 keep the values bounded
    cn = c / np.sum(np.abs(c))
    p3 = gs.stencil_plan(ndim, dims, "custom", 4, "const", cn, dtype, bc, offsets=offs)
    gs.stencil_apply(p3, xd, y, 3)
    assert gs.stencil_sync_status(p3) == 0
    pure, emu = oracle_run(x64, offs, cn, bc, 3, dtype)
    got = inputs.stored_values(y)
    print(f"{name} {dtype} {bc}: 3 steps, max rel err {relerr(got, pure):.2e} vs pure FP64, "
          f"{relerr(got, emu):.2e} vs per-step rounding")
    assert relerr(got, pure) < TOL[dtype]


def test_custom_grids_in_a_batch():
    # the batched kernel runs compiled sets of radius <= 2: a box r2, a star r2 and a diamond
    # r2 set carry these three custom grids
    specs = [((70, 90), [(0, 0), (1, -2), (-2, 1), (0, 1), (2, 2)], "periodic"),
             ((64, 130), [(0, 0), (0, -1), (-1, 0), (-2, 0), (0, 2)], "dirichlet"),
             ((33, 257), [(1, 1), (-1, -1), (0, 0)], "dirichlet")]
    items, refs = [], []
    for i, (dims, offs, bc) in enumerate(specs):
        offs = np.asarray(offs, dtype=np.int32)
        c = inputs.normalised_abs_weights(410 + i, len(offs))
        plan = gs.stencil_plan(2, dims, "custom", 2, "const", c, "f32", bc, offsets=offs)
        x, x64 = make_input(420 + i, dims, "f32")
        items.append((plan, x.cuda(), torch.empty(dims, dtype=torch.float32, device="cuda")))
        refs.append(oracle.run(x64, "const", bc, 4, offs=offs, coeffs=c))
    batch = gs.stencil_batch_plan(items, 4)
    gs.stencil_batch_launch(batch)
    assert gs.stencil_batch_status(batch) == 0
    for (plan, _, y), ref in zip(items, refs):
        assert relerr(inputs.stored_values(y), ref) < 1e-5

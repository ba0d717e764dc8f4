"""GPU parity of the variable-coefficient sweeps (general VAR forward/adjoint and div(k grad u))
against the FP64 oracle, through the C ABI.  The div(k grad u) workload (384^3, k lognormal
smoothed by a 5^3 box mean, u uniform[-1,1]) is checked at full size on sampled planes in f32,
f16 and bf16 storage, with the max relative error reported per storage type."""
import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import TOL, check_steps, make_input, oracle_threads, relerr
from paper_2609_06694_gb300 import inputs

pytestmark = pytest.mark.gpu

DTYPES = ["f32", "f16", "bf16"]


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


def to_dev(t):
    return t.cuda()


def var_case(ndim, shape, r, dtype, bc, dims, seed=300):
    offs = oracle.offsets(ndim, shape, r)
    plan = gs.stencil_plan(ndim, dims, shape, r, "var", None, dtype, bc)
    w_st = [inputs.to_storage(inputs.uniform(seed + i, dims, -0.5, 0.5), dtype)
            for i in range(len(offs))]
    w64 = np.stack([inputs.stored_values(t) for t in w_st])
    x, x64 = make_input(seed + 99, dims, dtype)
    return plan, offs, [to_dev(t) for t in w_st], w64, x, x64


@pytest.mark.parametrize("ndim,shape,r", [(2, "star", 1), (2, "star", 4), (2, "box", 2),
                                          (2, "diamond", 3), (3, "star", 1), (3, "star", 4),
                                          (3, "box", 1), (3, "diamond", 2)])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_var_forward_and_adjoint(ndim, shape, r, dtype, bc):
    dims = (13, 21, 136) if ndim == 3 else (45, 264)
    plan, offs, wd, w64, x, x64 = var_case(ndim, shape, r, dtype, bc, dims)
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply_var(plan, xd, wd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    assert relerr(inputs.stored_values(y), oracle.sweep_var(x64, offs, w64, bc)) < TOL[dtype]
    gs.stencil_apply_adjoint_var(plan, xd, wd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    assert relerr(inputs.stored_values(y), oracle.sweep_var_adjoint(x64, offs, w64, bc)) < TOL[dtype]


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_var_unaligned_rows_and_multistep(bc):
    dims = (9, 17, 131)  # odd row length: scalar loader and scalar coefficient loads
    plan, offs, wd, w64, x, x64 = var_case(3, "star", 2, "f32", bc, dims, seed=400)
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply_var(plan, xd, wd, y, 3)
    ref = oracle.run(x64, "var", bc, 3, offs=offs, coeffs=w64)
    assert relerr(inputs.stored_values(y), ref) < 1e-5
    gs.stencil_apply_adjoint_var(plan, xd, wd, y, 2)
    ref = oracle.run(x64, "var", bc, 2, offs=offs, coeffs=w64, adjoint=True)
    assert relerr(inputs.stored_values(y), ref) < 1e-5


def test_var_rejects_missing_arrays_and_unsupported_sets():
    plan = gs.stencil_plan(3, (8, 8, 8), "star", 1, "var", None, "f32", "dirichlet")
    x = torch.zeros((8, 8, 8), device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(ValueError):
        gs.stencil_apply_var(plan, x, [x] * 6, y, 1)  # 7 arrays expected (checked by count)
    big = gs.stencil_plan(3, (8, 8, 8), "box", 2, "var", None, "f32", "dirichlet")
    with pytest.raises(gs.StencilError) as e:
        gs.stencil_apply_var(big, x, [x] * 125, y, 1)
    assert e.value.code == -2  # 125 coefficient arrays: no kernel


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_divkgrad_work_splits(dtype, bc):
    # one equal share of the (tile, z) planes per resident CTA (z_chunk 0: a CTA's planes span
    # several tiles), aligned chunks per tile column (z_chunk -1), short chunks that end
    # mid-column, several tile heights, one and two rows per thread: every split gives the
    # same bits and matches the oracle
    dims = (23, 45, 264)
    plan = gs.stencil_plan(3, dims, "star", 1, "divkgrad", None, dtype, bc)
    k = inputs.to_storage(inputs.lognormal_k(3012, dims), dtype)
    u = inputs.to_storage(inputs.uniform(3011, dims), dtype)
    ref = oracle.divkgrad(inputs.stored_values(u), inputs.stored_values(k), bc)
    base = gs.stencil_plan_get_variant(plan)
    bx = base["block_x"]
    first = None
    f = 1 if bx == 32 else 2  # 16-bit rows of 128 cells take 16 threads: twice the rows
    for by, vy, zc in ((4, 1, 0), (2 * f, 1, 0), (7 * f, 1, 5), (f, 1, 9), (4 * f, 2, 16),
                       (7 * f, 2, 0), (f, 2, 3), (4 * f, 2, -1), (f, 1, -1)):
        gs.stencil_plan_set_variant(plan, **dict(base, block_y=by, vec_y=vy, z_chunk=zc,
                                                 stages=0))
        y = torch.empty_like(u, device="cuda")
        gs.stencil_apply_var(plan, u.cuda(), [k.cuda()], y, 1)
        assert gs.stencil_sync_status(plan) == 0
        assert relerr(inputs.stored_values(y), ref) < TOL[dtype], (by, vy, zc)
        if first is None:
            first = y.clone()
        assert torch.equal(y, first), (by, vy, zc)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_divkgrad_small(ndim, dtype, bc):
    dims = (11, 19, 136) if ndim == 3 else (37, 264)
    plan = gs.stencil_plan(ndim, dims, "star", 1, "divkgrad", None, dtype, bc)
    k = inputs.to_storage(inputs.lognormal_k(3002, dims), dtype)
    u = inputs.to_storage(inputs.uniform(3001, dims), dtype)
    k64, u64 = inputs.stored_values(k), inputs.stored_values(u)
    y = torch.empty_like(u, device="cuda")
    gs.stencil_apply_var(plan, u.cuda(), [k.cuda()], y, 1)
    assert gs.stencil_sync_status(plan) == 0
    ref = oracle.divkgrad(u64, k64, bc)
    assert relerr(inputs.stored_values(y), ref) < TOL[dtype]
    # adjoint = the operator itself
    y2 = torch.empty_like(y)
    gs.stencil_apply_adjoint_var(plan, u.cuda(), [k.cuda()], y2, 1)
    assert torch.equal(y, y2)
    # two steps: the tolerance against pure FP64, the per-step-rounded error printed
    gs.stencil_apply_var(plan, u.cuda(), [k.cuda()], y, 2)
    pure = oracle.run(u64, "divkgrad", bc, 2, coeffs=k64)
    emu = oracle.run(u64, "divkgrad", bc, 2, coeffs=k64,
                     round_fmt="none" if dtype == "f32" else dtype)
    check_steps(inputs.stored_values(y), pure, emu, dtype, f"div(k grad u) {ndim}D {bc} x2")


@pytest.mark.parametrize("dtype", DTYPES)
def test_divkgrad_384_full_size_whole_grid(dtype):
    """div(k grad u), 384^3, zero Dirichlet, in the launch configuration the dispatch map
    gives this size and storage type: every cell against the oracle on the exact stored
    inputs; the max relative error is printed per storage type."""
    n = 384
    dims = (n, n, n)
    k = inputs.to_storage(inputs.lognormal_k(3002, dims), dtype)
    u = inputs.to_storage(inputs.uniform(3001, dims), dtype)
    plan = gs.stencil_plan(3, dims, "star", 1, "divkgrad", None, dtype, "dirichlet")
    y = torch.empty_like(u, device="cuda")
    gs.stencil_apply_var(plan, u.cuda(), [k.cuda()], y, 1)
    assert gs.stencil_sync_status(plan) == 0
    with oracle_threads():
        ref = oracle.divkgrad(inputs.stored_values(u), inputs.stored_values(k), "dirichlet")
    err = relerr(inputs.stored_values(y), ref)
    print(f"div(k grad u) 384^3 {dtype}: max relative error {err:.3e} (all cells)")
    assert err < TOL[dtype]

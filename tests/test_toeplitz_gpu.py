"""GPU parity of the tensor-core sweep of the radius-2 box (STENCIL_FAMILY_TENSOR: Toeplitz
packing of the x direction onto tcgen05 MMAs, the tensor-core mapping of Sec. 6) against the
FP64 oracle: 2D and 3D, f16 and bf16 storage, every CTA tile width and number of MMA-issuing
warps, ragged y and x tiles, short z chunks and ring depths, multi-step runs, the adjoint, the
full-size 384^3 grid, and a bounded wait that expires."""
import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import TOL, check_steps, make_input, oracle_run, oracle_threads, relerr
from paper_2609_06694_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


def _plan(ndim, dims, dtype, c, tile_x=16, z_chunk=0, stages=0, mw=1):
    """A plan on the tensor-core kernel: tile_x outputs per CTA, mw warps issuing the MMAs."""
    plan = gs.stencil_plan(ndim, dims, "box", 2, "const", c, dtype, "dirichlet")
    gs.stencil_plan_set_variant(plan, family=gs.FAMILY_TENSOR, tile_x=tile_x, z_chunk=z_chunk,
                                stages=stages, fuse=1, block_y=1, vec_y=mw)
    return plan


def _weights(seed, ndim):
    c, _ = inputs.normalised_sum_weights(seed, 25 if ndim == 2 else 125)
    return c


# dims with ragged y tiles (not a multiple of 128 rows) and x tiles (a multiple of 8 but not
# of the CTA width), small z extents, and a plane smaller than one tile
CASES = [(3, (6, 130, 40)), (3, (9, 64, 64)), (3, (3, 20, 24)), (3, (1, 7, 8)),
         (2, (130, 40)), (2, (300, 264)), (2, (5, 8))]


@pytest.mark.parametrize("ndim,dims", CASES)
@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("tile_x,mw", [(16, 1), (16, 2), (32, 1), (32, 2), (64, 1), (64, 2),
                                       (64, 4)])
def test_tensor_sweep_matches_oracle(ndim, dims, dtype, tile_x, mw):
    offs = oracle.offsets(ndim, "box", 2)
    c = _weights(601, ndim)
    plan = _plan(ndim, dims, dtype, c, tile_x=tile_x, mw=mw)
    x, x64 = make_input(602, dims, dtype)
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    ref = oracle.sweep_const(x64, offs, c, "dirichlet")
    err = relerr(inputs.stored_values(y), ref)
    # the FP32 CUDA-core path the dispatcher picks for the same plan, for scale
    plain = gs.stencil_plan(ndim, dims, "box", 2, "const", c, dtype, "dirichlet")
    assert gs.stencil_plan_get_variant(plain)["family"] != gs.FAMILY_TENSOR
    y2 = torch.empty_like(xd)
    gs.stencil_apply(plain, xd, y2, 1)
    err2 = relerr(inputs.stored_values(y2), ref)
    print(f"{ndim}D {dims} {dtype} tile_x {tile_x} mma warps {mw}: "
          f"max rel err {err:.2e} (tensor cores), "
          f"{err2:.2e} (CUDA cores)")
    assert err < TOL[dtype]


@pytest.mark.parametrize("z_chunk,stages", [(1, 5), (2, 6), (7, 5), (3, 12), (0, 8)])
def test_tensor_launch_shapes(z_chunk, stages):
    dims = (13, 140, 48)
    offs = oracle.offsets(3, "box", 2)
    c = _weights(611, 3)
    x, x64 = make_input(612, dims, "bf16")
    xd = x.cuda()
    ref = oracle.sweep_const(x64, offs, c, "dirichlet")
    outs = []
    # (64-output tiles with 12 plane slots need more shared memory than a CTA may have: the
    # launch reports STENCIL_ERR_UNSUPPORTED, checked below)
    for tile_x, mw in ((16, 1), (16, 2), (32, 1), (32, 2)) + (((64, 4),) if stages <= 8 else ()):
        plan = _plan(3, dims, "bf16", c, tile_x=tile_x, z_chunk=z_chunk, stages=stages, mw=mw)
        y = torch.empty_like(xd)
        gs.stencil_apply(plan, xd, y, 1)
        assert gs.stencil_sync_status(plan) == 0
        assert relerr(inputs.stored_values(y), ref) < TOL["bf16"]
        outs.append(y)
    # the tile width, the chunking and the issuing warp change which CTA and warp compute a
    # cell and when, not the order of the MMAs that accumulate it
    for o in outs[1:]:
        assert torch.equal(outs[0], o)
    if stages > 8:
        plan = _plan(3, dims, "bf16", c, tile_x=64, z_chunk=z_chunk, stages=stages, mw=4)
        with pytest.raises(gs.StencilError) as e:
            gs.stencil_apply(plan, xd, torch.empty_like(xd), 1)
        assert e.value.code == -2


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("mw", [1, 2])
def test_tensor_multi_step_and_adjoint(dtype, mw):
    dims = (10, 70, 56)
    offs = oracle.offsets(3, "box", 2)
    c = inputs.normalised_abs_weights(621, 125)
    plan = _plan(3, dims, dtype, c, tile_x=32, mw=mw)
    x, x64 = make_input(622, dims, dtype)
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, y, 4)
    assert gs.stencil_sync_status(plan) == 0
    pure, emu = oracle_run(x64, offs, c, "dirichlet", 4, dtype)
    check_steps(inputs.stored_values(y), pure, emu, dtype, f"tensor cores {dtype} x4")
    gs.stencil_apply_adjoint(plan, xd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    ref = oracle.sweep_const_adjoint(x64, offs, c, "dirichlet")
    assert relerr(inputs.stored_values(y), ref) < TOL[dtype]


@pytest.mark.parametrize("mw", [1, 2, 4])
def test_tensor_expired_wait_is_reported(mw):
    # one phantom arrival on every "accumulator read" barrier: the MMA lane's wait for a free
    # accumulator expires once the ring of accumulators has gone round once
    dims = (12, 64, 32)
    offs = oracle.offsets(3, "box", 2)
    c = _weights(641, 3)
    plan = _plan(3, dims, "bf16", c, tile_x=64 if mw == 4 else 16, z_chunk=12, stages=6,
                 mw=mw)
    x, x64 = make_input(642, dims, "bf16")
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_set_wait_limit(plan, 0.05, 1)
    gs.stencil_apply(plan, xd, y, 1)
    assert gs.stencil_sync_status(plan) == -5
    gs.stencil_set_wait_limit(plan, 2.0, 0)
    gs.stencil_apply(plan, xd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    assert relerr(inputs.stored_values(y), oracle.sweep_const(x64, offs, c, "dirichlet")) < 1e-2


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("tile_x,mw", [(16, 1), (64, 4)])
def test_tensor_384_cubed_whole_grid(dtype, tile_x, mw):
    """384^3 zero-Dirichlet 125-point box in 16-bit storage on the tensor cores, against the
    oracle at every cell."""
    dims = (384, 384, 384)
    offs = oracle.offsets(3, "box", 2)
    c = _weights(2002, 3)
    plan = _plan(3, dims, dtype, c, tile_x=tile_x, mw=mw)
    x = inputs.to_storage(inputs.uniform(2003, dims), dtype)
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    with oracle_threads():
        ref = oracle.sweep_const(inputs.stored_values(x), offs, c, "dirichlet")
    err = relerr(inputs.stored_values(y), ref)
    print(f"384^3 box r2 {dtype} on the tensor cores: max rel err {err:.2e} (all cells)")
    assert err < TOL[dtype]

"""GPU checks of the batched persistent sweep: many 2D grids of mixed sizes, shapes, storage
types and boundaries advanced by one persistent cooperative launch (captured in a CUDA
graph), against the FP64 oracle per grid and bit for bit against the plain per-grid sweep
(both accumulate the offsets in canonical order in FP32).  The bounded device-side barrier
wait is exercised by a barrier that waits for one arrival that never comes: the launch must
end with STENCIL_ERR_TIMEOUT and leave the context usable."""
import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import (TOL, check_steps, make_input, oracle_run, oracle_threads, relerr,
                     seeded_weights)
from paper_2609_06694_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


def make_batch(specs, steps, tiles=(0, 0, 0)):
    grids = []
    for i, (ny, nx, shape, r, dtype, bc) in enumerate(specs):
        offs = oracle.offsets(2, shape, r)
        c = seeded_weights(4100 + i, len(offs))
        plan = gs.stencil_plan(2, (ny, nx), shape, r, "const", c, dtype, bc)
        x, x64 = make_input(4500 + i, (ny, nx), dtype)
        xd = x.cuda()
        yd = torch.empty_like(xd)
        grids.append(dict(plan=plan, offs=offs, c=c, x=x, x64=x64, xd=xd, yd=yd, dtype=dtype,
                          bc=bc))
    batch = gs.stencil_batch_plan([(g["plan"], g["xd"], g["yd"]) for g in grids], steps, *tiles)
    return batch, grids


MIXED = [(37, 51, "star", 1, "f32", "dirichlet"), (130, 260, "box", 2, "f32", "periodic"),
         (5, 3, "star", 2, "f32", "periodic"), (64, 64, "box", 1, "bf16", "dirichlet"),
         (200, 131, "diamond", 2, "f16", "dirichlet"), (33, 129, "star", 2, "bf16", "periodic"),
         (1, 7, "box", 1, "f32", "dirichlet"), (96, 300, "diamond", 1, "f32", "periodic")]


@pytest.mark.parametrize("steps", [1, 2, 5])
def test_mixed_batch_matches_oracle(steps):
    batch, grids = make_batch(MIXED, steps)
    gs.stencil_batch_launch(batch)
    assert gs.stencil_batch_status(batch) == 0
    for g in grids:
        pure, emu = oracle_run(g["x64"], g["offs"], g["c"], g["bc"], steps, g["dtype"])
        check_steps(inputs.stored_values(g["yd"]), pure, emu, g["dtype"],
                    f"batch {g['x64'].shape} x{steps}")
    # a second launch of the same graph gives the same result
    first = [g["yd"].clone() for g in grids]
    gs.stencil_batch_launch(batch)
    assert gs.stencil_batch_status(batch) == 0
    for g, f in zip(grids, first):
        assert torch.equal(g["yd"], f)


def test_batch_equals_plain_per_grid_bitwise():
    steps = 4
    batch, grids = make_batch(MIXED, steps)
    gs.stencil_batch_launch(batch)
    assert gs.stencil_batch_status(batch) == 0
    for g in grids:
        ref = torch.empty_like(g["yd"])
        gs.stencil_apply(g["plan"], g["xd"], ref, steps)
        torch.cuda.synchronize()
        assert torch.equal(ref, g["yd"])


# (tile_y, tile_x, steps per group): ragged tiles, tiles larger than small grids, deep groups
TILINGS = [(16, 120, 1), (16, 120, 3), (8, 56, 3), (4, 8, 5), (32, 120, 2), (64, 248, 1)]


@pytest.mark.parametrize("tiles", TILINGS)
def test_launch_shapes_equal_plain_sweeps(tiles):
    """Every launch shape gives the bits of plain per-grid sweeps, over ragged tiles, grids
    smaller than one tile and periodic halos that wrap more than once."""
    steps = 5
    batch, grids = make_batch(MIXED, steps, tiles)
    gs.stencil_batch_launch(batch)
    assert gs.stencil_batch_status(batch) == 0
    for g in grids:
        ref = torch.empty_like(g["yd"])
        gs.stencil_apply(g["plan"], g["xd"], ref, steps)
        torch.cuda.synchronize()
        assert torch.equal(ref, g["yd"]), (tiles, g["x64"].shape, g["dtype"], g["bc"])
    g = grids[1]  # one grid against the oracle as well
    pure, emu = oracle_run(g["x64"], g["offs"], g["c"], g["bc"], steps, g["dtype"])
    check_steps(inputs.stored_values(g["yd"]), pure, emu, g["dtype"], f"batch tiles {tiles}")


def test_batch_rejects_unsupported_and_bad_items():
    p3 = gs.stencil_plan(3, (8, 8, 8), "star", 1, "const", np.ones(7), "f32", "dirichlet")
    x = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(gs.StencilError) as e:
        gs.stencil_batch_plan([(p3, x, torch.empty_like(x))], 2)
    assert e.value.code == -2
    p2 = gs.stencil_plan(2, (8, 8), "star", 3, "const", np.ones(13), "f32", "dirichlet")
    x2 = torch.zeros((8, 8), device="cuda")
    with pytest.raises(gs.StencilError):
        gs.stencil_batch_plan([(p2, x2, torch.empty_like(x2))], 2)  # radius 3: no batch kernel
    p1 = gs.stencil_plan(2, (8, 8), "star", 1, "const", np.ones(5), "f32", "dirichlet")
    with pytest.raises(gs.StencilError) as e:
        gs.stencil_batch_plan([(p1, x2, x2)], 2)  # in == out
    assert e.value.code == -1


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_full_batch_256_grids_20_steps(dtype):
    """256 grids, sides log-uniform in [64, 2048] per axis, star r1/r2 and box 3x3/5x5, zero
    Dirichlet, 20 steps, in the launch configuration the benchmark times: every grid against
    the FP64 oracle (the tolerance holds against pure FP64; the error against the oracle that
    rounds after every step is printed), and bit for bit equal to plain per-grid sweeps."""
    specs = inputs.batched_grid_specs()
    steps = 20
    rows = [(s["ny"], s["nx"], s["shape"], s["radius"], dtype, "dirichlet") for s in specs]
    batch, grids = make_batch(rows, steps)
    info = gs.stencil_batch_info(batch)
    assert info["tiles"] > 256 and info["blocks"] >= 152
    gs.stencil_batch_launch(batch)
    assert gs.stencil_batch_status(batch) == 0
    worst_pure = worst_emu = 0.0
    with oracle_threads():
        for g, s in zip(grids, specs):
            ref = torch.empty_like(g["yd"])
            gs.stencil_apply(g["plan"], g["xd"], ref, steps)
            torch.cuda.synchronize()
            assert torch.equal(ref, g["yd"])
            pure, emu = oracle_run(g["x64"], g["offs"], g["c"], "dirichlet", steps, dtype)
            got = inputs.stored_values(g["yd"])
            ep, ee = relerr(got, pure), relerr(got, emu)
            assert ep < TOL[dtype], (s, ep)
            worst_pure, worst_emu = max(worst_pure, ep), max(worst_emu, ee)
    print(f"batched 256 grids x 20 steps {dtype}: worst max rel err {worst_pure:.2e} vs pure "
          f"FP64, {worst_emu:.2e} vs per-step rounding")


@pytest.mark.parametrize("tiles", [(0, 0, 0), (16, 120, 2)])  # 3 steps: two groups
def test_barrier_timeout_is_reported_and_context_survives(tiles):
    specs = [(64, 128, "star", 1, "f32", "dirichlet"), (50, 70, "box", 1, "f32", "periodic")]
    batch, grids = make_batch(specs, 3, tiles)
    gs.stencil_batch_set_wait_limit(batch, 0.05, phantom_arrivals=1)
    gs.stencil_batch_launch(batch)
    assert gs.stencil_batch_status(batch) == -5  # STENCIL_ERR_TIMEOUT
    gs.stencil_batch_set_wait_limit(batch, 2.0, phantom_arrivals=0)
    gs.stencil_batch_launch(batch)
    assert gs.stencil_batch_status(batch) == 0
    for g in grids:
        pure, _ = oracle_run(g["x64"], g["offs"], g["c"], g["bc"], 3, "f32")
        assert relerr(inputs.stored_values(g["yd"]), pure) < 1e-5

"""GPU parity of the two-step fused 3D kernel (temporal blocking, Sec. 4.3) against the FP64
oracle and, bit for bit, against the same number of single sweeps: the intermediate time
level is rounded to the storage type before the second step, so fusing changes no result.

Cases: star r1/r2, diamond r2 and the 27-point box; f32, f16 and bf16; both boundaries; even
and odd step counts (an odd last step runs on the streaming kernel); grids several tiles wide
and tall with ragged tails, rows that are not a multiple of 16 bytes, short z chunks whose
pieces span tiles, and grids smaller than the halo."""
import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import TOL, check_steps, make_input, oracle_run, relerr, seeded_weights
from paper_2609_06694_gb300 import inputs

pytestmark = pytest.mark.gpu

SETS = [("star", 1), ("star", 2), ("diamond", 2), ("box", 1), ("diamond", 1)]


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


def fused_variant(dtype, r, by=None, z_chunk=16, stages=0):
    bx = 32 if dtype == "f32" else 16
    vy = 2 if dtype == "f32" else 1
    if by is None:
        by = 4 if dtype == "f32" else 8
    return dict(family=gs.FAMILY_FUSED3D, block_x=bx, block_y=max(by, 2 * r), vec_y=vy,
                z_chunk=z_chunk, fuse=2, tile_x=0, tile_y=0, stages=stages)


def stream_variant(dtype, z_chunk=16):
    bx = 32 if dtype == "f32" else 16
    return dict(family=gs.FAMILY_STREAM, block_x=bx, block_y=4, vec_y=2, z_chunk=z_chunk,
                fuse=1, tile_x=0, tile_y=0, stages=0)


def run(plan, x, steps):
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, y, steps)
    assert gs.stencil_sync_status(plan) == 0
    return y


@pytest.mark.parametrize("shape,r", SETS)
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_fused_pairs_match_oracle_and_single_sweeps(shape, r, dtype, bc):
    dims = (23, 37, 264)
    offs = oracle.offsets(3, shape, r)
    c = seeded_weights(501 + r, len(offs))
    fused = gs.stencil_plan(3, dims, shape, r, "const", c, dtype, bc)
    gs.stencil_plan_set_variant(fused, **fused_variant(dtype, r))
    plain = gs.stencil_plan(3, dims, shape, r, "const", c, dtype, bc)
    gs.stencil_plan_set_variant(plain, **stream_variant(dtype))
    x, x64 = make_input(502, dims, dtype)
    for steps in (2, 3, 4):
        yf = run(fused, x, steps)
        yp = run(plain, x, steps)
        assert torch.equal(yf, yp), (shape, r, dtype, bc, steps)
        pure, emu = oracle_run(x64, offs, c, bc, steps, dtype)
        check_steps(inputs.stored_values(yf), pure, emu, dtype,
                    f"fused 3D {shape} r{r} {bc} x{steps}")


@pytest.mark.parametrize("dims", [(9, 21, 263), (5, 3, 40), (40, 70, 128), (3, 5, 7)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_fused_odd_shapes(dims, bc):
    # rows that are not a multiple of 16 bytes (element loads, scalar stores), grids smaller
    # than the doubled halo (periodic reads wrap several times), one tile column
    for shape, r in (("box", 1), ("star", 2)):
        offs = oracle.offsets(3, shape, r)
        c = seeded_weights(511, len(offs))
        plan = gs.stencil_plan(3, dims, shape, r, "const", c, "f32", bc)
        gs.stencil_plan_set_variant(plan, **fused_variant("f32", r, z_chunk=4))
        x, x64 = make_input(512, dims, "f32")
        y = run(plan, x, 2)
        ref = oracle.run(x64, "const", bc, 2, offs=offs, coeffs=c)
        assert relerr(inputs.stored_values(y), ref) < 1e-5, (dims, shape, bc)


@pytest.mark.parametrize("by,z_chunk,stages", [(2, 5, 2), (4, 7, 3), (7, 64, 0), (5, 0, 6)])
def test_fused_launch_shapes(by, z_chunk, stages):
    # tile heights from the smallest allowed to 7 rows of threads, pieces shorter than the
    # halo and spanning tiles, ring depths from 2
    dims = (31, 45, 200)
    offs = oracle.offsets(3, "box", 1)
    c = seeded_weights(521, len(offs))
    plan = gs.stencil_plan(3, dims, "box", 1, "const", c, "f32", "periodic")
    gs.stencil_plan_set_variant(plan, **fused_variant("f32", 1, by=by, z_chunk=z_chunk,
                                                      stages=stages))
    x, x64 = make_input(522, dims, "f32")
    y = run(plan, x, 2)
    ref = oracle.run(x64, "const", "periodic", 2, offs=offs, coeffs=c)
    assert relerr(inputs.stored_values(y), ref) < 1e-5


def test_fused_adjoint():
    dims = (17, 40, 136)
    offs = oracle.offsets(3, "diamond", 2)
    c = inputs.uniform(531, (len(offs),))  # not symmetric
    c = c / np.sum(np.abs(c))
    plan = gs.stencil_plan(3, dims, "diamond", 2, "const", c, "f32", "dirichlet")
    gs.stencil_plan_set_variant(plan, **fused_variant("f32", 2))
    x, x64 = make_input(532, dims, "f32")
    y = torch.empty_like(x.cuda())
    gs.stencil_apply_adjoint(plan, x.cuda(), y, 2)
    assert gs.stencil_sync_status(plan) == 0
    ref = oracle.run(x64, "const", "dirichlet", 2, offs=offs, coeffs=c, adjoint=True)
    assert relerr(inputs.stored_values(y), ref) < 1e-5


def test_fused_expired_wait_is_reported():
    dims = (40, 24, 256)
    offs = oracle.offsets(3, "box", 1)
    c = seeded_weights(541, len(offs))
    plan = gs.stencil_plan(3, dims, "box", 1, "const", c, "f32", "dirichlet")
    gs.stencil_plan_set_variant(plan, **fused_variant("f32", 1, z_chunk=40))
    x, x64 = make_input(542, dims, "f32")
    gs.stencil_set_wait_limit(plan, 0.05, 1)
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, y, 2)
    assert gs.stencil_sync_status(plan) == -5
    gs.stencil_set_wait_limit(plan, 2.0, 0)
    y = run(plan, x, 2)
    ref = oracle.run(x64, "const", "dirichlet", 2, offs=offs, coeffs=c)
    assert relerr(inputs.stored_values(y), ref) < 1e-5


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_fused_box_512_cubed_whole_planes(bc):
    """The 27-point box at 512^3, 8 steps as four fused pairs: five whole planes against the
    oracle (the dependency slab), and the whole grid bit for bit against 8 single sweeps."""
    from helpers import oracle_threads, periodic_slab
    dims = (512, 512, 512)
    offs = oracle.offsets(3, "box", 1)
    c, _ = inputs.normalised_sum_weights(2002, len(offs))
    x = inputs.to_storage(inputs.uniform(2003, dims), "f32")
    fused = gs.stencil_plan(3, dims, "box", 1, "const", c, "f32", bc)
    gs.stencil_plan_set_variant(fused, **fused_variant("f32", 1, by=4, z_chunk=64))
    plain = gs.stencil_plan(3, dims, "box", 1, "const", c, "f32", bc)
    yf = run(fused, x, 8)
    yp = run(plain, x, 8)
    assert torch.equal(yf, yp)
    del yp
    x64 = inputs.stored_values(x)
    errs = []
    with oracle_threads():
        for z0 in (0, 255, 511):
            if bc == "periodic":
                ref = oracle.run(periodic_slab(x64, z0, 8), "const", "dirichlet", 8, offs=offs,
                                 coeffs=c)[8, 8:-8, 8:-8]
            else:
                lo, hi = max(0, z0 - 8), min(512, z0 + 9)
                # planes lo .. hi-1 with zero ghosts beyond: exact at z0, whose distance to a
                # ghost plane that is not a true boundary is 9 > 8 steps
                ref = oracle.run(x64[lo:hi], "const", "dirichlet", 8, offs=offs,
                                 coeffs=c)[z0 - lo]
            got = yf[z0].double().cpu().numpy()
            errs.append((np.max(np.abs(got - ref)), np.max(np.abs(ref))))
    err = max(e for e, _ in errs) / max(m for _, m in errs)
    print(f"fused box 512^3 {bc}, 8 steps: max rel err {err:.2e} (3 whole planes)")
    assert err < 1e-5

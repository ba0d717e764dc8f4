"""GPU parity of the constant-coefficient sweeps against the FP64 oracle (through the C ABI).

Cases span every shape (star, box, diamond), radius 1-4, 2D and 3D grids, f32/f16/bf16
storage and both boundary rules, on grids that cover several tiles plus ragged tails in x, y
and z, on the vectorised (16-byte aligned rows) and scalar (odd row length) loaders, and the
fused multi-step 2D kernel.  Tolerances: max-norm relative error 1e-5 (f32), 2e-3 (f16),
1e-2 (bf16) against the FP64 oracle on the exact stored inputs.  Multi-step low-precision runs
are held to the same tolerance against pure FP64 (no rounding between steps); their error
against the oracle that rounds to the storage type after every step (the library's stated
semantics) is printed as a diagnostic.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import (TOL, check_steps, make_input, oracle_run, oracle_threads, periodic_slab,
                     relerr, seeded_weights)
from paper_2609_06694_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = ["star", "box", "diamond"]
DTYPES = ["f32", "f16", "bf16"]


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


def gpu_apply(plan, x_cpu, steps=1, adjoint=False):
    xd = x_cpu.cuda()
    yd = torch.empty_like(xd)
    fn = gs.stencil_apply_adjoint if adjoint else gs.stencil_apply
    fn(plan, xd, yd, steps)
    assert gs.stencil_sync_status(plan) == 0
    return inputs.stored_values(yd)


def dims_for(ndim, shape, r, aligned=True):
    # x spans 2+ tiles of 128 cells plus a tail; y spans 2+ tiles; z several chunks
    nx = 264 if aligned else 263
    if ndim == 2:
        return (53, nx)
    big = shape != "star" and r >= 3
    return (13 if big else 21, 35, nx if not big else (136 if aligned else 133))


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_single_sweep_matches_oracle(ndim, shape, r, dtype, bc):
    dims = dims_for(ndim, shape, r)
    offs = oracle.offsets(ndim, shape, r)
    c = seeded_weights(1000 + r, len(offs))
    plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, dtype, bc)
    if ndim == 3:
        gs.stencil_plan_set_variant(plan, z_chunk=8)  # several z chunks with a ragged tail
    x, x64 = make_input(2000 + r, dims, dtype)
    got = gpu_apply(plan, x)
    ref = oracle.sweep_const(x64, offs, c, bc)
    assert relerr(got, ref) < TOL[dtype]


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_scalar_loader_odd_row_length(ndim, shape, bc):
    r = 2
    dims = dims_for(ndim, shape, r, aligned=False)
    offs = oracle.offsets(ndim, shape, r)
    c = seeded_weights(31, len(offs))
    for dtype in DTYPES:
        plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, dtype, bc)
        if ndim == 2:
            gs.stencil_plan_set_variant(plan, family=gs.FAMILY_STREAM, block_x=128 // (
                4 if dtype == "f32" else 8), block_y=4, vec_y=2, fuse=1, tile_x=0, tile_y=0)
        x, x64 = make_input(32, dims, dtype)
        assert relerr(gpu_apply(plan, x), oracle.sweep_const(x64, offs, c, bc)) < TOL[dtype]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("vec_y", [1, 2])
@pytest.mark.parametrize("blocks", [(32, 7), (32, 4), (32, 3), (32, 1)])
@pytest.mark.parametrize("stages", [0, 2, 5])
def test_stream_variants_agree(shape, vec_y, blocks, stages):
    # odd tile heights, the shallowest ring (the producer waits on every slot) and a ring
    # deeper than some pieces are long
    r = 1
    dims = (19, 45, 200)
    offs = oracle.offsets(3, shape, r)
    c = seeded_weights(41, len(offs))
    plan = gs.stencil_plan(3, dims, shape, r, "const", c, "f32", "periodic")
    gs.stencil_plan_set_variant(plan, block_x=blocks[0], block_y=blocks[1], vec_y=vec_y,
                                z_chunk=7, stages=stages)
    x, x64 = make_input(42, dims, "f32")
    assert relerr(gpu_apply(plan, x), oracle.sweep_const(x64, offs, c, "periodic")) < 1e-5


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("stages", [2, 16])
def test_stream_ring_depth_radius4(bc, stages):
    # wide stars on a grid that is several tiles wide and tall with ragged edges, with the
    # shallowest and the deepest ring, up to the 256-thread consumer tile
    dims = (40, 70, 300)
    for r, by in ((4, 4), (4, 8), (4, 7), (3, 8)):
        offs = oracle.offsets(3, "star", r)
        c = seeded_weights(43, len(offs))
        plan = gs.stencil_plan(3, dims, "star", r, "const", c, "f32", bc)
        gs.stencil_plan_set_variant(plan, block_x=32, block_y=by, vec_y=1, z_chunk=9,
                                    stages=stages)
        x, x64 = make_input(44, dims, "f32")
        assert relerr(gpu_apply(plan, x), oracle.sweep_const(x64, offs, c, bc)) < 1e-5


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape,r", [("star", 4), ("box", 1), ("star", 2)])
def test_periodic_whole_tile_widths(dtype, shape, r):
    # periodic grids whose width is a whole number of 128-cell tiles: the first and last tile
    # columns wrap exactly one 16-byte chunk per row, which a second tensor copy puts into the
    # slot's side arrays (tiles whose rows wrap too are patched instead); a single tile
    # column takes both side chunks at once
    for dims in ((20, 40, 256), (9, 33, 128)):
        offs = oracle.offsets(3, shape, r)
        c = seeded_weights(47, len(offs))
        plan = gs.stencil_plan(3, dims, shape, r, "const", c, dtype, "periodic")
        x, x64 = make_input(48, dims, dtype)
        assert relerr(gpu_apply(plan, x), oracle.sweep_const(x64, offs, c, "periodic")) < TOL[dtype]


def _split_rows(ny, ty, r, pitch_bytes):
    """Which y-end tile rows of a periodic grid take split tensor copies (the rows inside the
    grid and the R wrapped rows as two copies, at 128-byte boundaries of the slot; compiled for
    radius 4): the same rule as the library's launcher, restated for the test's coverage
    checks."""
    tiles_y = -(-ny // ty)
    hb = ny - (tiles_y - 1) * ty
    if r != 4 or tiles_y < 2 or ny < ty + 2 * r or hb < r:
        return set()
    out = set()
    if (r * pitch_bytes) % 128 == 0:
        out.add("top")
    if ((hb + r) * pitch_bytes) % 128 == 0:
        out.add("bottom")
    return out


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("ndim,dims,shape,r,block_y,want", [
    # want: the split tile rows in f32, in bf16 (the split must land on 128 bytes)
    (3, (12, 134, 384), "star", 4, 7, ({"top", "bottom"}, {"top"})),  # x-inner and corners
    (3, (10, 134, 128), "star", 4, 7, ({"top", "bottom"}, {"top"})),  # one tile column
    (3, (12, 140, 256), "star", 4, 7, ({"top"}, {"top", "bottom"})),
    (3, (9, 92, 256), "star", 4, 14, ({"top", "bottom"}, None)),      # 28-row f32 tiles
    (3, (11, 70, 256), "box", 2, 4, (set(), set())),                  # R = 2: patched
    (2, (134, 384), "star", 4, 7, ({"top", "bottom"}, {"top"})),
])
def test_periodic_split_copies(dtype, ndim, dims, shape, r, block_y, want):
    # periodic tile rows at the y ends take their wrapped rows by a second tensor copy into
    # the slot rows next to the first (no patching after the copy lands); tiles that also wrap
    # in x fill their side arrays with cp.async.  Against the oracle, and bit for bit against
    # the same sweep of a misaligned input view (element loader, no tensor copies)
    es = 4 if dtype == "f32" else 2
    bx, by = (32, block_y) if es == 4 else (16, 2 * block_y)
    vy = 2
    if ndim == 2:
        by = min(by, 224 // bx)
    ty = by * vy
    pitch_bytes = (128 + 2 * (16 // es)) * es
    want = want[0 if es == 4 else 1]
    if want is None:
        pytest.skip("16-bit two-row tiles take at most 14 rows of 16 threads")
    assert _split_rows(dims[-2], ty, r, pitch_bytes) == want
    offs = oracle.offsets(ndim, shape, r)
    c = seeded_weights(71, len(offs))
    plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, dtype, "periodic")
    gs.stencil_plan_set_variant(plan, family=1, block_x=bx, block_y=by, vec_y=vy,
                                z_chunk=4, stages=0, fuse=1)
    x, x64 = make_input(72, dims, dtype)
    got = gpu_apply(plan, x)
    assert relerr(got, oracle.sweep_const(x64, offs, c, "periodic")) < TOL[dtype], dims
    # the same input at a 4-byte offset: rows not 16-byte aligned, element loads
    n = x.numel()
    buf = torch.empty(n + 8, dtype=x.dtype, device="cuda")
    xm = buf[2:2 + n].view(dims)
    xm.copy_(x.cuda())
    ym = torch.empty(dims, dtype=x.dtype, device="cuda")
    gs.stencil_apply(plan, xm, ym, 1)
    assert gs.stencil_sync_status(plan) == 0
    assert np.array_equal(inputs.stored_values(ym), got)


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("dtype,shape,r,block_y,vec_y", [
    ("f32", "star", 4, 14, 2), ("f32", "star", 4, 7, 2), ("f32", "box", 1, 4, 2),
    ("bf16", "star", 2, 8, 2), ("f16", "diamond", 1, 14, 1)])
def test_column_aligned_split(bc, dtype, shape, r, block_y, vec_y):
    # z_chunk -1: every tile column cut into the same number of chunks (as many as the
    # resident CTAs allow, here one to several per column); the same bits as one equal share
    # per CTA and as 5-plane chunks, and the oracle's values
    dims = (37, 92, 264)
    offs = oracle.offsets(3, shape, r)
    c = seeded_weights(81, len(offs))
    plan = gs.stencil_plan(3, dims, shape, r, "const", c, dtype, bc)
    bx = 32 if dtype == "f32" else 16
    x, x64 = make_input(82, dims, dtype)
    outs = []
    for zc in (-1, 0, 5):
        gs.stencil_plan_set_variant(plan, family=1, block_x=bx, block_y=block_y, vec_y=vec_y,
                                    z_chunk=zc, stages=0, fuse=1)
        outs.append(gpu_apply(plan, x))
    assert relerr(outs[0], oracle.sweep_const(x64, offs, c, bc)) < TOL[dtype]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("shape,r,block_y,vec_y", [("star", 4, 8, 1), ("star", 4, 7, 2),
                                                   ("star", 4, 4, 2), ("star", 2, 3, 2),
                                                   ("box", 1, 4, 2), ("box", 1, 7, 1),
                                                   ("diamond", 2, 5, 1)])
def test_periodic_side_chunks(dtype, shape, r, block_y, vec_y):
    # tall periodic grids of whole tile columns: most tiles of the first and last column take
    # their x halo from the side arrays, the tiles at the y ends are patched, for several tile
    # heights; and one 2D grid
    cases = [(3, (11, 70, 256)), (3, (6, 50, 128))]
    if vec_y == 1:
        cases.append((2, (90, 256)))
    for ndim, dims in cases:
        offs = oracle.offsets(ndim, shape, r)
        c = seeded_weights(49, len(offs))
        plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, dtype, "periodic")
        # 16-bit rows of 128 cells take 16 threads: twice the rows keep whole warps
        bx, by = (32, block_y) if dtype == "f32" else (16, 2 * block_y)
        if ndim == 2:
            by = min(by, 224 // bx)  # 2D tiles take at most 224 consumer threads
        gs.stencil_plan_set_variant(plan, family=1, block_x=bx, block_y=by, vec_y=vec_y,
                                    z_chunk=5, stages=0, fuse=1)
        x, x64 = make_input(50, dims, dtype)
        got = gpu_apply(plan, x)
        assert relerr(got, oracle.sweep_const(x64, offs, c, "periodic")) < TOL[dtype], (ndim, dims)


@pytest.mark.parametrize("dtype,steps", [("f32", 1), ("f32", 2), ("f32", 3), ("f32", 8),
                                         ("bf16", 1), ("bf16", 2), ("bf16", 3)])
def test_apply_host_buffers(dtype, steps):
    # stencil_apply_host: 3D grids deep enough for the z-slab pipeline (copies in and out
    # overlapping the sweeps; several sweeps as a wavefront over z whose periodic ends follow
    # the bands), a shallow one and a 2D one on the simple path; pinned and pageable host
    # buffers.  Bit for bit equal to the device-buffer path, and within tolerance of the
    # oracle.
    cases = [(3, (70, 40, 256), "star", 4, "periodic"), (3, (130, 33, 128), "box", 1, "dirichlet"),
             (3, (64, 20, 130), "diamond", 2, "periodic"), (3, (9, 20, 64), "star", 2, "periodic"),
             (2, (90, 300), "box", 2, "periodic")]
    for i, (ndim, dims, shape, r, bc) in enumerate(cases):
        offs = oracle.offsets(ndim, shape, r)
        c = seeded_weights(60 + i, len(offs))
        plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, dtype, bc)
        x, x64 = make_input(61 + i, dims, dtype)
        for pinned in (True, False):
            hin = x.pin_memory() if pinned else x.clone()
            hout = torch.empty_like(hin)
            if pinned:
                hout = hout.pin_memory()
            gs.stencil_apply_host(plan, hin, hout, steps)
            dev = torch.empty_like(x.cuda())
            gs.stencil_apply(plan, x.cuda(), dev, steps)
            torch.cuda.synchronize()
            assert torch.equal(hout, dev.cpu()), (dims, shape, bc, pinned)
        pure, emu = oracle_run(x64, offs, c, bc, steps, dtype)
        check_steps(inputs.stored_values(hout), pure, emu, dtype, f"host {dims} {shape}")


def test_tiny_grids_wrap_many_times():
    for ndim, dims in ((3, (3, 2, 4)), (3, (1, 1, 8)), (2, (1, 4)), (2, (3, 5)), (3, (2, 3, 5))):
        for shape in SHAPES:
            r = 4
            offs = oracle.offsets(ndim, shape, r)
            c = seeded_weights(51, len(offs))
            for bc in ("periodic", "dirichlet"):
                plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, "f32", bc)
                x, x64 = make_input(52, dims, "f32")
                got = gpu_apply(plan, x)
                assert relerr(got, oracle.sweep_const(x64, offs, c, bc)) < 1e-5, (dims, shape, bc)


@pytest.mark.parametrize("ndim,shape,r", [(3, "star", 4), (3, "box", 1), (3, "diamond", 2),
                                          (2, "box", 2), (2, "star", 3)])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_multi_step_matches_oracle(ndim, shape, r, dtype, bc):
    dims = (17, 33, 136) if ndim == 3 else (67, 136)
    steps = 5
    offs = oracle.offsets(ndim, shape, r)
    c = seeded_weights(61, len(offs))
    plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, dtype, bc)
    x, x64 = make_input(62, dims, dtype)
    got = gpu_apply(plan, x, steps)
    pure, emu = oracle_run(x64, offs, c, bc, steps, dtype)
    check_steps(got, pure, emu, dtype, f"{ndim}D {shape} r{r} {bc} x{steps}")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r", [1, 2, 4])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_fused2d_matches_oracle(shape, r, dtype, bc):
    dims = (75, 93)  # ragged against 32x32 tiles
    offs = oracle.offsets(2, shape, r)
    c = seeded_weights(71, len(offs))
    plan = gs.stencil_plan(2, dims, shape, r, "const", c, dtype, bc)
    gs.stencil_plan_set_variant(plan, family=gs.FAMILY_FUSED2D, fuse=3, tile_x=32, tile_y=32,
                                block_x=128, block_y=1, vec_y=1, z_chunk=0)
    x, x64 = make_input(72, dims, dtype)
    steps = 7  # fused groups of 3, 3, 1
    got = gpu_apply(plan, x, steps)
    pure, emu = oracle_run(x64, offs, c, bc, steps, dtype)
    check_steps(got, pure, emu, dtype, f"fused 2D {shape} r{r} {bc} x{steps}")


def test_fused_equals_unfused_bitwise():
    """Rounding between fused steps makes grouping irrelevant (same FP32 sums per step)."""
    dims = (70, 90)
    offs = oracle.offsets(2, "box", 1)
    c = seeded_weights(81, len(offs))
    for dtype in DTYPES:
        x, _ = make_input(82, dims, dtype)
        a = gs.stencil_plan(2, dims, "box", 1, "const", c, dtype, "dirichlet")
        gs.stencil_plan_set_variant(a, family=gs.FAMILY_FUSED2D, fuse=6, tile_x=32, tile_y=16,
                                    block_x=64, block_y=1, vec_y=1, z_chunk=0)
        b = gs.stencil_plan(2, dims, "box", 1, "const", c, dtype, "dirichlet")
        gs.stencil_plan_set_variant(b, family=gs.FAMILY_FUSED2D, fuse=1, tile_x=32, tile_y=16,
                                    block_x=64, block_y=1, vec_y=1, z_chunk=0)
        ya, yb = gpu_apply(a, x, 6), gpu_apply(b, x, 6)
        assert np.array_equal(ya, yb)


@pytest.mark.parametrize("ndim,shape,r", [(3, "box", 1), (3, "star", 2), (2, "diamond", 3),
                                          (2, "box", 2)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_adjoint_matches_oracle_and_dot_test(ndim, shape, r, bc):
    dims = (15, 22, 136) if ndim == 3 else (41, 136)
    offs = oracle.offsets(ndim, shape, r)
    c = inputs.uniform(91, (len(offs),))  # non-symmetric weights
    plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, "f32", bc)
    x, x64 = make_input(92, dims, "f32")
    y, y64 = make_input(93, dims, "f32")
    aty = gpu_apply(plan, y, 1, adjoint=True)
    assert relerr(aty, oracle.sweep_const_adjoint(y64, offs, c, bc)) < 1e-5
    ax = gpu_apply(plan, x, 1)
    lhs, rhs = float(np.sum(ax * y64)), float(np.sum(x64 * aty))
    assert abs(lhs - rhs) <= 1e-5 * np.sum(np.abs(ax * y64))
    aty3 = gpu_apply(plan, y, 3, adjoint=True)
    ref3 = oracle.run(y64, "const", bc, 3, offs=offs, coeffs=c, adjoint=True)
    assert relerr(aty3, ref3) < 1e-5


def test_jacobi_512_10_steps_full_size():
    """2D 5-point Jacobi, weights 0.2, zero Dirichlet, 512^2, 10 steps (fused launches)."""
    dims = (512, 512)
    offs = oracle.offsets(2, "star", 1)
    c = np.full(len(offs), 0.2)
    plan = gs.stencil_plan(2, dims, "star", 1, "const", c, "f32", "dirichlet")
    assert gs.stencil_plan_get_variant(plan)["family"] == gs.FAMILY_FUSED2D
    x, x64 = make_input(1001, dims, "f32")
    got = gpu_apply(plan, x, 10)
    ref = oracle.run(x64, "const", "dirichlet", 10, offs=offs, coeffs=c)
    assert relerr(got, ref) < 1e-5


def _laplacian_r4_plan(dims, bc="periodic"):
    offs = oracle.offsets(3, "star", 4)
    return offs, inputs.laplacian_coeffs(offs, 4)


@pytest.mark.parametrize("which", ["star4", "box27"])
def test_full_size_512_cubed_whole_grid(which):
    """512^3 f32 periodic in the launch configuration the benchmark times: the 1-step result
    against the oracle at every cell of the grid, and the 8-step result against the oracle at
    every cell of five whole xy-planes (z = 0, 1, 255, 510, 511: the wrapped z ends, every tile
    column with its wrapped x ends and patched y ends)."""
    dims = (512, 512, 512)
    if which == "star4":
        shape, r = "star", 4
        offs = oracle.offsets(3, shape, r)
        c = inputs.laplacian_coeffs(offs, 4)
        seed = 2001
    else:
        shape, r = "box", 1
        offs = oracle.offsets(3, shape, r)
        c, _ = inputs.normalised_sum_weights(2002, len(offs))
        seed = 2003
    plan = gs.stencil_plan(3, dims, shape, r, "const", c, "f32", "periodic")
    x = inputs.to_storage(inputs.uniform(seed, dims), "f32")
    xd = x.cuda()
    y1 = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, y1, 1)
    y8 = torch.empty_like(xd)
    gs.stencil_apply(plan, xd, y8, 8)
    assert gs.stencil_sync_status(plan) == 0
    x64 = inputs.stored_values(x)
    with oracle_threads():
        ref1 = oracle.sweep_const(x64, offs, c, "periodic")
        err1 = relerr(inputs.stored_values(y1), ref1)
        del ref1
        h = 8 * r
        errs = []
        for z0 in (0, 1, 255, 510, 511):
            ref = oracle.run(periodic_slab(x64, z0, h), "const", "dirichlet", 8, offs=offs,
                             coeffs=c)[h, h:-h, h:-h]
            got = y8[z0].double().cpu().numpy()
            errs.append((np.max(np.abs(got - ref)), np.max(np.abs(ref))))
    err8 = max(e for e, _ in errs) / max(m for _, m in errs)
    print(f"512^3 {which}: 1 step max rel err {err1:.2e} (all cells); 8 steps {err8:.2e} "
          f"(5 whole planes)")
    assert err1 < 1e-5
    assert err8 < 1e-5

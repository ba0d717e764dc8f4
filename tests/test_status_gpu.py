"""GPU tests of kernel-side error reporting: a bounded wait of the plane ring that expires is
reported by stencil_sync_status as STENCIL_ERR_TIMEOUT, the launch returns instead of hanging,
and the plan keeps working afterwards.

The expiry is provoked in the permitted way: stencil_set_wait_limit shortens the bound on the
ring's waits and adds one arrival that never comes to every slot's "consumers are done"
barrier, so the producer warp's wait for a free slot runs out once the ring is full.  Every
copy the producer issued has landed by then (the consumers read those planes), so no copy is
in flight when a CTA exits.  Nothing here faults, traps or spins without a bound."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import make_input, relerr, seeded_weights
from paper_2609_06694_gb300 import inputs

pytestmark = pytest.mark.gpu

TIMEOUT = -5


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


# (ndim, dims, shape, radius, boundary, variant): every CTA walks more planes than its ring
# holds -- 3D pieces of 40 planes (plus halo) on the tensor-copy path, on the periodic path with
# side arrays and patched y-end tiles, and a 2D grid whose CTAs take several tiles each
CASES = [
    (3, (40, 24, 256), "star", 1, "dirichlet", dict(z_chunk=40)),
    (3, (40, 40, 256), "box", 1, "periodic", dict(z_chunk=40)),
    (3, (40, 24, 128), "star", 4, "periodic", dict(z_chunk=40, stages=2)),
    (2, (2048, 2048), "star", 2, "dirichlet", dict(family=1, block_x=32, block_y=4, vec_y=2,
                                                   z_chunk=0, fuse=1, tile_x=0, tile_y=0)),
]


@pytest.mark.parametrize("ndim,dims,shape,r,bc,variant", CASES)
def test_expired_ring_wait_is_reported_and_the_plan_recovers(ndim, dims, shape, r, bc, variant):
    offs = oracle.offsets(ndim, shape, r)
    c = seeded_weights(301, len(offs))
    plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, "f32", bc)
    gs.stencil_plan_set_variant(plan, **variant)
    x, x64 = make_input(302, dims, "f32")
    xd = x.cuda()
    y = torch.zeros_like(xd)
    gs.stencil_set_wait_limit(plan, 0.05, 1)
    t0 = time.perf_counter()
    gs.stencil_apply(plan, xd, y, 1)
    rc = gs.stencil_sync_status(plan)
    waited = time.perf_counter() - t0
    assert rc == TIMEOUT, rc
    assert waited < 30.0
    assert gs.stencil_sync_status(plan) == 0          # reading the word clears it
    # normal limits: the same plan sweeps correctly and reports nothing
    gs.stencil_set_wait_limit(plan, 2.0, 0)
    gs.stencil_apply(plan, xd, y, 1)
    assert gs.stencil_sync_status(plan) == 0
    got = inputs.stored_values(y)
    assert relerr(got, oracle.sweep_const(x64, offs, c, bc)) < 1e-5


def test_divkgrad_expired_wait_is_reported():
    dims = (40, 30, 256)
    plan = gs.stencil_plan(3, dims, "star", 1, "divkgrad", None, "f32", "dirichlet")
    gs.stencil_plan_set_variant(plan, z_chunk=40)
    u, u64 = make_input(311, dims, "f32")
    k = inputs.to_storage(inputs.lognormal_k(312, dims), "f32")
    ud, kd = u.cuda(), k.cuda()
    y = torch.zeros_like(ud)
    gs.stencil_set_wait_limit(plan, 0.05, 1)
    gs.stencil_apply_var(plan, ud, [kd], y, 1)
    assert gs.stencil_sync_status(plan) == TIMEOUT
    gs.stencil_set_wait_limit(plan, 2.0, 0)
    gs.stencil_apply_var(plan, ud, [kd], y, 1)
    assert gs.stencil_sync_status(plan) == 0
    ref = oracle.divkgrad(u64, inputs.stored_values(k), "dirichlet")
    assert relerr(inputs.stored_values(y), ref) < 1e-5


def test_errors_stay_with_their_plan():
    # a timeout of one plan is not reported by another plan's status word
    dims = (40, 24, 256)
    offs = oracle.offsets(3, "star", 1)
    c = seeded_weights(321, len(offs))
    bad = gs.stencil_plan(3, dims, "star", 1, "const", c, "f32", "dirichlet")
    good = gs.stencil_plan(3, dims, "star", 1, "const", c, "f32", "dirichlet")
    for p in (bad, good):
        gs.stencil_plan_set_variant(p, z_chunk=40)
    gs.stencil_set_wait_limit(bad, 0.05, 1)
    x, _ = make_input(322, dims, "f32")
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply(bad, xd, y, 1)
    gs.stencil_apply(good, xd, y, 1)
    assert gs.stencil_sync_status(good) == 0
    assert gs.stencil_sync_status(bad) == TIMEOUT
    del bad
    # the released word was cleared: a new plan that takes it starts clean
    fresh = gs.stencil_plan(3, dims, "star", 1, "const", c, "f32", "dirichlet")
    gs.stencil_apply(fresh, xd, y, 1)
    assert gs.stencil_sync_status(fresh) == 0
    assert np.isfinite(y.cpu().numpy()).all()

"""GPU parity of the fused stencil + physics kernel (reaction-diffusion steps
u + dt (A u + c1 u + c3 u^3), one launch per step) against the FP64 oracle: Allen-Cahn with
the radius-4 and radius-1 Laplacians, a linear reaction with the 27-point box, 2D and 3D, both
boundaries, f32 and bf16 storage, several steps (the tolerance against pure FP64), and the
argument checks of the entry point."""
import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import TOL, make_input, relerr
from paper_2609_06694_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


CASES = [
    # ndim, dims, shape, radius, weights, dt, c1, c3, steps
    (3, (21, 35, 264), "star", 4, "laplacian", 0.02, 4.0, -4.0, 5),    # Allen-Cahn, eps = 0.5
    (3, (17, 40, 136), "star", 1, "laplacian", 0.1, 1.0, -1.0, 4),
    (3, (13, 30, 200), "box", 1, "seeded", 0.2, -0.5, 0.0, 3),          # linear reaction
    (2, (90, 300), "star", 2, "laplacian", 0.05, 2.0, -2.0, 6),
    (2, (64, 129), "box", 1, "seeded", 0.1, 0.3, -0.2, 3),              # odd row length
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_reaction_matches_oracle(case, dtype, bc):
    ndim, dims, shape, r, wkind, dt, c1, c3, steps = case
    offs = oracle.offsets(ndim, shape, r)
    c = inputs.laplacian_coeffs(offs, r) if wkind == "laplacian" else \
        inputs.normalised_abs_weights(601, len(offs))
    plan = gs.stencil_plan(ndim, dims, shape, r, "const", c, dtype, bc)
    x, x64 = make_input(602, dims, dtype)
    xd = x.cuda()
    y = torch.empty_like(xd)
    gs.stencil_apply_reaction(plan, xd, y, steps, dt, c1, c3)
    assert gs.stencil_sync_status(plan) == 0
    got = inputs.stored_values(y)
    pure = oracle.reaction(x64, offs, c, bc, steps, dt, c1, c3)
    err = relerr(got, pure)
    emu = oracle.reaction(x64, offs, c, bc, steps, dt, c1, c3,
                          round_fmt="none" if dtype == "f32" else dtype)
    print(f"reaction {ndim}D {shape} r{r} {bc} {dtype} x{steps}: max rel err {err:.2e} vs pure "
          f"FP64, {relerr(got, emu):.2e} vs per-step rounding")
    assert err < TOL[dtype]
    # one step from the same input through the adjoint-free plain sweep path: u + dt (L + ...)
    if steps > 1 and dtype == "f32":
        y1 = torch.empty_like(xd)
        gs.stencil_apply_reaction(plan, xd, y1, 1, dt, c1, c3)
        one = oracle.reaction(x64, offs, c, bc, 1, dt, c1, c3)
        assert relerr(inputs.stored_values(y1), one) < TOL[dtype]


def test_reaction_argument_checks():
    offs = oracle.offsets(3, "star", 3)
    c = inputs.laplacian_coeffs(offs, 3)
    plan = gs.stencil_plan(3, (8, 8, 8), "star", 3, "const", c, "f32", "periodic")
    x = torch.zeros((8, 8, 8), device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(gs.StencilError) as e:
        gs.stencil_apply_reaction(plan, x, y, 1, 0.1, 1.0, -1.0)  # star r3: no kernel
    assert e.value.code == -2
    p16 = gs.stencil_plan(3, (8, 8, 8), "star", 1, "const", np.ones(7), "f16", "periodic")
    xh = torch.zeros((8, 8, 8), device="cuda", dtype=torch.float16)
    with pytest.raises(gs.StencilError) as e:
        gs.stencil_apply_reaction(p16, xh, torch.empty_like(xh), 1, 0.1, 1.0, -1.0)
    assert e.value.code == -2
    p1 = gs.stencil_plan(3, (8, 8, 8), "star", 1, "const", np.ones(7), "f32", "periodic")
    with pytest.raises(gs.StencilError) as e:
        gs.stencil_apply_reaction(p1, x, y, 1, float("nan"), 1.0, -1.0)
    assert e.value.code == -1
    with pytest.raises(gs.StencilError):
        gs.stencil_apply_reaction(p1, x, x, 1, 0.1, 1.0, -1.0)  # in == out

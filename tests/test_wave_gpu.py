"""GPU checks of the acoustic wave-equation driver: forward traces, FP64 misfit and the
checkpointed adjoint velocity gradient against the FP64 oracle on a small grid; bitwise
independence of the gradient from the checkpoint interval; the autograd wrappers; and, at
the full 256^3 x 500-step size, properties that hold at any size (checkpoint invariance and
agreement with a finite-difference directional derivative)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2609_06694_gb300 as gs
from helpers import relerr
from paper_2609_06694_gb300 import autograd, inputs
from paper_2609_06694_gb300 import wave as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    gs.build.build()
    torch.cuda.set_device(0)


def problem(n=(36, 34, 40), steps=80, freq=25.0, seed=5901, radius=4, rz=5):
    v = inputs.velocity_field(seed, n, width=5, passes=2)
    h = 10.0
    dt = 0.4 * h / 4500.0
    offs = oracle.offsets(3, "star", radius)
    lap = inputs.laplacian_coeffs(offs, radius)
    wl = inputs.ricker(freq, dt, steps)
    src = (n[0] // 2, n[1] // 2, n[2] // 2)
    vt = inputs.perturbed_velocity(v, sigma=4.0)
    return dict(v=v, vt=vt, h=h, dt=dt, offs=offs, lap=lap, wl=wl, src=src, rz=rz, steps=steps,
                dims=n, radius=radius)


def plan_for(P, ck):
    return W.wave_plan(P["dims"], P["radius"], P["lap"], P["h"], P["dt"], P["steps"], P["src"],
                       P["wl"], P["rz"], ck)


def f32dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_forward_traces_match_oracle():
    P = problem()
    plan = plan_for(P, 10)
    v32 = f32dev(P["v"])
    tr = torch.empty(plan.trace_shape, dtype=torch.float32, device="cuda")
    W.wave_forward(plan, v32, tr)
    torch.cuda.synchronize()
    v64 = v32.double().cpu().numpy()  # the oracle sees the stored f32 velocities
    ref = oracle.wave_forward(v64, P["offs"], P["lap"], P["h"], P["dt"], P["steps"], P["src"],
                              P["wl"], P["rz"])
    assert np.max(np.abs(ref)) > 0
    assert relerr(tr.double().cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("radius", [4, 2])
def test_gradient_matches_oracle(radius):
    P = problem(radius=radius)
    v32 = f32dev(P["v"])
    v64 = v32.double().cpu().numpy()
    obs64 = oracle.wave_forward(f32dev(P["vt"]).double().cpu().numpy(), P["offs"], P["lap"],
                                P["h"], P["dt"], P["steps"], P["src"], P["wl"], P["rz"])
    obs = f32dev(obs64)
    obs_used = obs.double().cpu().numpy()
    J_ref, g_ref = oracle.wave_gradient(v64, P["offs"], P["lap"], P["h"], P["dt"], P["steps"],
                                        P["src"], P["wl"], P["rz"], obs_used, ck_every=10)
    plan = plan_for(P, 10)
    tr = torch.empty(plan.trace_shape, dtype=torch.float32, device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty(P["dims"], dtype=torch.float64, device="cuda")
    W.wave_gradient(plan, v32, obs, tr, J, g)
    torch.cuda.synchronize()
    assert abs(J.item() - J_ref) <= 1e-4 * J_ref
    err = relerr(g.cpu().numpy(), g_ref)
    print(f"wave gradient r{radius}: max-norm relative error vs FP64 oracle {err:.2e}")
    assert err < 1e-3
    # the misfit entry point alone gives the same J from the same traces
    J2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    W.wave_misfit(plan, tr, obs, J2)
    assert J2.item() == J.item()


def test_gradient_independent_of_checkpoint_interval():
    P = problem(steps=60)
    v32 = f32dev(P["v"])
    obs = torch.zeros((P["steps"],) + P["dims"][1:], dtype=torch.float32, device="cuda")
    out = []
    for ck in (7, 25, 60):
        plan = plan_for(P, ck)
        tr = torch.empty(plan.trace_shape, dtype=torch.float32, device="cuda")
        J = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.empty(P["dims"], dtype=torch.float64, device="cuda")
        W.wave_gradient(plan, v32, obs, tr, J, g)
        out.append((J.item(), g.clone()))
    for J, g in out[1:]:
        assert J == out[0][0] and torch.equal(g, out[0][1])


def test_wave_misfit_autograd():
    P = problem(steps=40)
    v = f32dev(P["v"]).requires_grad_(True)
    obs = f32dev(np.zeros((P["steps"],) + P["dims"][1:]))
    plan = plan_for(P, 10)
    J = W.WaveMisfit().apply(v, plan, obs)
    J.backward()
    tr = torch.empty(plan.trace_shape, dtype=torch.float32, device="cuda")
    Jr = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty(P["dims"], dtype=torch.float64, device="cuda")
    W.wave_gradient(plan, v.detach(), obs, tr, Jr, g)
    assert J.item() == Jr.item()
    assert torch.equal(v.grad, g.float())


def test_stencil_autograd_is_the_adjoint():
    dims = (20, 24, 136)
    offs = oracle.offsets(3, "box", 1)
    c = inputs.uniform(7, (len(offs),))
    plan = gs.stencil_plan(3, dims, "box", 1, "const", c, "f32", "dirichlet")
    x = torch.from_numpy(inputs.uniform(8, dims).astype(np.float32)).cuda().requires_grad_(True)
    w = torch.from_numpy(inputs.uniform(9, dims).astype(np.float32)).cuda()
    y = autograd.StencilSweep.apply(x, plan, 2)
    (y * w).sum().backward()
    ref = oracle.run(w.double().cpu().numpy(), "const", "dirichlet", 2, offs=offs, coeffs=c,
                     adjoint=True)
    assert relerr(x.grad.double().cpu().numpy(), ref) < 1e-5
    pv = gs.stencil_plan(3, dims, "star", 1, "var", None, "f32", "periodic")
    offs7 = oracle.offsets(3, "star", 1)
    ws = [torch.from_numpy(inputs.uniform(20 + i, dims).astype(np.float32)).cuda()
          for i in range(7)]
    x2 = x.detach().clone().requires_grad_(True)
    y2 = autograd.VarStencilSweep.apply(x2, pv, 1, *ws)
    (y2 * w).sum().backward()
    ref2 = oracle.sweep_var_adjoint(w.double().cpu().numpy(), offs7,
                                    np.stack([t.double().cpu().numpy() for t in ws]), "periodic")
    assert relerr(x2.grad.double().cpu().numpy(), ref2) < 1e-5


def full_problem(steps=500):
    n = (256, 256, 256)
    v = inputs.velocity_field(5001, n)
    vt = inputs.perturbed_velocity(v)
    h = 10.0
    dt = 0.4 * h / 4500.0
    offs = oracle.offsets(3, "star", 4)
    return dict(v=v, vt=vt, h=h, dt=dt, offs=offs, lap=inputs.laplacian_coeffs(offs, 4),
                wl=inputs.ricker(15.0, dt, steps), src=(10, 128, 128), rz=10, steps=steps,
                dims=n, radius=4)


def test_full_size_gradient_properties():
    """256^3, 500 steps, checkpoints every 25: the gradient equals the one with checkpoints
    every 50 bit for bit, and <g, e> matches the central difference of J along a smooth
    direction e (f32 fields, so the check is at 1e-2)."""
    P = full_problem()
    v32 = f32dev(P["v"])
    plan25 = plan_for(P, 25)
    tr = torch.empty(plan25.trace_shape, dtype=torch.float32, device="cuda")
    W.wave_forward(plan_for(P, 25), f32dev(P["vt"]), tr)
    obs = tr.clone()
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty(P["dims"], dtype=torch.float64, device="cuda")
    W.wave_gradient(plan25, v32, obs, tr, J, g)
    torch.cuda.synchronize()
    assert J.item() > 0 and torch.isfinite(g).all()
    plan50 = plan_for(P, 50)
    J50 = torch.zeros(1, dtype=torch.float64, device="cuda")
    g50 = torch.empty_like(g)
    W.wave_gradient(plan50, v32, obs, tr, J50, g50)
    assert J50.item() == J.item() and torch.equal(g50, g)
    # Finite-difference directional derivative.  The receivers (z = 10) do not see the
    # centre of the grid within 500 steps, so the direction is a smooth bump the recorded
    # wavefield crosses (between source and receivers), and the observed record is zero so
    # that J is far above the f32 rounding of the traces.
    zero = torch.zeros_like(obs)
    g0 = torch.empty_like(g)
    J0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    W.wave_gradient(plan25, v32, zero, tr, J0, g0)
    zz, yy, xx = np.meshgrid(*[np.arange(256.0)] * 3, indexing="ij")
    e = np.exp(-((zz - 24) ** 2 + (yy - 128) ** 2 + (xx - 150) ** 2) / (2 * 12.0 ** 2))
    eps = 4.0  # m/s
    Js = []
    for sgn in (1, -1):
        trs = torch.empty_like(tr)
        W.wave_forward(plan25, f32dev(P["v"] + sgn * eps * e), trs)
        Jx = torch.zeros(1, dtype=torch.float64, device="cuda")
        W.wave_misfit(plan25, trs, zero, Jx)
        Js.append(Jx.item())
    fd = (Js[0] - Js[1]) / (2 * eps)
    ad = float((g0 * torch.from_numpy(e).cuda()).sum())
    print(f"256^3 x 500: J={J.item():.6e}  <g,e>={ad:.6e}  FD={fd:.6e}  rel={abs(fd-ad)/abs(ad):.2e}")
    assert abs(fd - ad) <= 1e-2 * abs(ad)

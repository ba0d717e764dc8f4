"""The schedule of stencil_apply_host's multi-sweep wavefront over z (csrc/wavefront.h, the
header the library issues its copies and launches from), replayed plane by plane on the CPU:
every sweep reads planes the sweep before it (or the landed input) has already written and
nothing has overwritten since, no output plane is rewritten after it was copied out, every
plane is copied out once, and the replay reproduces direct iteration of a z stencil in FP64
(zero-Dirichlet and periodic, 2 to 8 sweeps, radius 1 to 4, the library's slab rule)."""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("wavefront") / "wavefront_driver")
    subprocess.run([cxx, "-std=c++17", "-O1", os.path.join(ROOT, "tests", "wavefront_driver.cpp"),
                    "-o", exe], check=True)
    return exe


def schedule(exe, nz, r, periodic, steps):
    # the library's slab rule for host buffers (up to 8 slabs of at least max(16, 2r) planes)
    nslab = min(8, nz // max(16, 2 * r))
    zb = [nz * k // nslab for k in range(nslab + 1)]
    out = subprocess.run([exe, str(nz), str(r), str(int(periodic)), str(steps), str(nslab)] +
                         [str(z) for z in zb], check=True, capture_output=True, text=True).stdout
    return zb, [tuple(int(v) for v in ln.split()) for ln in out.splitlines()]


def iterate(x, w, periodic, steps):
    r = (len(w) - 1) // 2
    for _ in range(steps):
        y = np.zeros_like(x)
        for d in range(-r, r + 1):
            if periodic:
                y += w[d + r] * np.roll(x, -d)
            else:
                s = np.zeros_like(x)
                if d >= 0:
                    s[:len(x) - d] = x[d:]
                else:
                    s[-d:] = x[:len(x) + d]
                y += w[d + r] * s
        x = y
    return x


def replay(ops, zb, x, w, periodic, steps):
    nz, r = len(x), (len(w) - 1) // 2
    arrived = np.zeros(nz, bool)
    # the library's buffers: the input, then sweep t writes `out` when steps - t is even,
    # else `scratch`; `step_of` records which sweep last wrote each plane of each buffer
    data = {"in": x.copy(), "out": np.full(nz, np.nan), "scratch": np.full(nz, np.nan)}
    step_of = {"out": np.zeros(nz, int), "scratch": np.zeros(nz, int)}
    dst = lambda t: "out" if (steps - t) % 2 == 0 else "scratch"
    copied = np.zeros(nz, bool)
    host = np.full(nz, np.nan)
    for kind, slab, t, a, b in ops:
        assert 0 <= a < b <= nz, (kind, t, a, b)
        if kind == 0:
            assert (a, b) == (zb[slab], zb[slab + 1])
            arrived[a:b] = True
        elif kind == 1:
            src = "in" if t == 1 else dst(t - 1)
            d = dst(t)
            for z in range(a, b):
                acc = 0.0
                for o in range(-r, r + 1):
                    zz = z + o
                    if periodic:
                        zz %= nz
                    elif zz < 0 or zz >= nz:
                        continue
                    if t == 1:
                        assert arrived[zz], ("input not landed", t, z, zz)
                    else:
                        assert step_of[src][zz] == t - 1, ("stale read", t, z, zz)
                    acc += w[o + r] * data[src][zz]
                if d == "out":
                    assert not copied[z], ("rewritten after copy-out", t, z)
                data[d][z] = acc
                step_of[d][z] = t
        else:
            assert t == steps
            assert (step_of["out"][a:b] == steps).all()
            assert not copied[a:b].any(), "copied twice"
            copied[a:b] = True
            host[a:b] = data["out"][a:b]
    assert copied.all()
    return host


@pytest.mark.parametrize("periodic", [False, True])
def test_wavefront_schedule_replays_direct_iteration(driver, periodic):
    rng = np.random.default_rng(7)
    n = 0
    for nz, r, steps in itertools.product((32, 40, 70, 130, 257), (1, 2, 4), (2, 3, 8)):
        if nz < 2 * max(16, 2 * r):
            continue
        zb, ops = schedule(driver, nz, r, periodic, steps)
        x = rng.uniform(-1, 1, nz)
        w = rng.uniform(-1, 1, 2 * r + 1)
        got = replay(ops, zb, x, w, periodic, steps)
        ref = iterate(x, w, periodic, steps)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12), (nz, r, steps)
        n += 1
    assert n > 20


def test_wavefront_overlaps_copies_with_sweeps(driver):
    # the point of the schedule: on the benchmark's 512-plane grid the last sweep's first
    # planes go out before the last input slab has landed (zero-Dirichlet and periodic)
    for periodic in (False, True):
        zb, ops = schedule(driver, 512, 4, periodic, 8)
        first_out = next(i for i, op in enumerate(ops) if op[0] == 2)
        last_in = max(i for i, op in enumerate(ops) if op[0] == 0)
        assert first_out < last_in, periodic

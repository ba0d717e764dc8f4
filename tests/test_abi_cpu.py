"""Host-side checks of the C ABI that need no GPU: the library loads, exports every function
declared in include/*.h, validates plans and arguments, keeps the canonical offset order, and
reads dispatch maps."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
import paper_2609_06694_gb300 as gs
from paper_2609_06694_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("stencil_plan", "stencil_apply", "stencil_apply_adjoint", "stencil_apply_var",
              "stencil_apply_adjoint_var", "stencil_batch_plan", "stencil_batch_launch",
              "stencil_destroy", "stencil_strerror", "stencil_sync_status"):
        assert n in names


def test_library_exports_every_declared_function():
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_abi_version_and_strerror():
    assert gs.stencil_abi_version() == 2
    for code in (0, -1, -2, -3, -4, -5, -6):
        s = gs.stencil_strerror(code)
        assert s and s != "unknown status code"
    assert gs.stencil_strerror(-99) == "unknown status code"


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", ["star", "box", "diamond"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_library_offsets_equal_oracle_offsets(ndim, shape, r):
    offs = oracle.offsets(ndim, shape, r)
    dims = (9, 10, 11)[:ndim]
    p = gs.stencil_plan(ndim, dims, shape, r, "const", np.ones(len(offs)), "f32", "periodic")
    assert np.array_equal(gs.stencil_offsets(p), offs)


def _plan_rc(ndim=3, dims=(8, 8, 8), shape=0, r=1, kind=0, coeffs="auto", dtype=0, bc=0):
    lib = api._lib()
    d = (ctypes.c_int64 * max(1, len(dims)))(*dims)
    if isinstance(coeffs, str):
        n = len(oracle.offsets(ndim, ["star", "box", "diamond"][shape], r)) if 1 <= r <= 4 and \
            ndim in (2, 3) and shape in (0, 1, 2) else 1
        coeffs = np.ones(n)
    if coeffs is None:
        cptr, n = None, 0
    else:
        coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
        cptr, n = coeffs.ctypes.data_as(ctypes.c_void_p), len(coeffs)
    h = ctypes.c_void_p()
    rc = lib.stencil_plan(ctypes.byref(h), ndim, d, shape, r, kind, cptr, n, None, dtype, bc)
    if h.value:
        lib.stencil_destroy(h)
    return rc


def test_plan_validation():
    assert _plan_rc() == 0
    assert _plan_rc(ndim=1, dims=(8,)) == -1
    assert _plan_rc(ndim=4, dims=(8, 8, 8, 8)) == -1
    assert _plan_rc(r=0) == -1
    assert _plan_rc(r=5) == -1
    assert _plan_rc(shape=3) == -1                    # custom without its offsets
    assert _plan_rc(shape=4) == -1
    assert _plan_rc(dtype=3) == -1
    assert _plan_rc(bc=2) == -1
    assert _plan_rc(kind=3) == -1
    assert _plan_rc(dims=(8, 0, 8)) == -1
    assert _plan_rc(dims=(8, -3, 8)) == -1
    assert _plan_rc(coeffs=np.ones(6)) == -1          # 7 offsets expected
    assert _plan_rc(coeffs=None) == -1                # const needs coefficients
    bad = np.ones(7)
    bad[3] = np.nan
    assert _plan_rc(coeffs=bad) == -1
    assert _plan_rc(kind=1, coeffs=None) == 0         # var: arrays come at apply time
    assert _plan_rc(kind=1, coeffs=np.ones(7)) == -1
    assert _plan_rc(kind=2, coeffs=None) == 0         # div(k grad u): star r1 only
    assert _plan_rc(kind=2, shape=1, coeffs=None) == -1
    assert _plan_rc(kind=2, r=2, coeffs=None) == -1
    assert _plan_rc(ndim=2, dims=(5, 7)) == 0
    assert _plan_rc(dims=(1, 1, 1)) == 0
    lib = api._lib()
    assert lib.stencil_plan(None, 3, (ctypes.c_int64 * 3)(8, 8, 8), 0, 1, 0, None, 0, None, 0,
                            0) == -1


def _custom_rc(offsets, ndim=3, r=2, kind=0, coeffs="auto", shape=3):
    lib = api._lib()
    d = (ctypes.c_int64 * ndim)(*([9] * ndim))
    o = np.ascontiguousarray(offsets, dtype=np.int32)
    n = len(o)
    c = np.ones(n) if isinstance(coeffs, str) else coeffs
    cptr = None if c is None else np.ascontiguousarray(c, dtype=np.float64).ctypes.data_as(
        ctypes.c_void_p)
    h = ctypes.c_void_p()
    rc = lib.stencil_plan(ctypes.byref(h), ndim, d, shape, r, kind, cptr,
                          0 if c is None else len(c), o.ctypes.data_as(ctypes.c_void_p), 0, 0)
    if h.value:
        lib.stencil_destroy(h)
    return rc


def test_custom_offset_validation():
    up = [(0, 0, 0), (0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, -2)]
    assert _custom_rc(up) == 0
    assert _custom_rc(up, r=1) == -1                       # |component| > radius
    assert _custom_rc(up + [(0, 0, -1)]) == -1             # repeated offset
    assert _custom_rc(up, coeffs=None) == -1               # ncoeffs = 0: no offsets, no weights
    assert _custom_rc(up, kind=1, coeffs=None) == -2       # custom sets: constant weights only
    assert _custom_rc(up, shape=0) == -1                   # offsets given for a named shape
    assert _custom_rc([(0, 0, 5)], r=4) == -1
    assert _custom_rc([(0, 0)], ndim=2, r=1) == 0
    assert _custom_rc(np.zeros((0, 3)), r=1) == -1         # empty set


@pytest.mark.parametrize("offsets,want", [
    ([(0, 0, 0), (0, 0, -1), (0, 0, -2), (0, 1, 0), (3, 0, 0)], ("star", 3)),
    ([(0, 0, 0)], ("star", 1)),
    ([(1, 1, 0), (0, 0, 0), (-1, 0, 1)], ("diamond", 2)),    # 25 points < 27 of the box r1
    ([(1, 1, 1), (0, 0, 0)], ("box", 1)),                    # diamond r3 (63) > box r1 (27)
    ([(2, 2, 2), (0, 1, 0)], ("box", 2)),
])
def test_custom_sets_run_on_the_smallest_compiled_superset(offsets, want):
    p = gs.stencil_plan(3, (9, 9, 9), "custom", 4, "const", np.arange(1.0, len(offsets) + 1),
                        "f32", "periodic", offsets=offsets)
    assert gs.stencil_plan_kernel_set(p) == want
    # the plan reports the caller's offsets, in the caller's order
    assert np.array_equal(gs.stencil_offsets(p), np.array(offsets, dtype=np.int32))


def test_wait_limit_validation():
    p = gs.stencil_plan(3, (8, 8, 8), "star", 1, "const", np.ones(7), "f32", "dirichlet")
    gs.stencil_set_wait_limit(p, 0.5, 0)
    for bad in ((0.0, 0), (-1.0, 0), (4000.0, 0), (1.0, -1), (1.0, 1001)):
        with pytest.raises(gs.StencilError):
            gs.stencil_set_wait_limit(p, *bad)


def test_status_words_are_recycled():
    # every plan takes one device status word from a fixed array; destroyed plans give theirs
    # back, so creating and dropping many plans never runs out (host logic, no GPU needed)
    for _ in range(3):
        plans = [gs.stencil_plan(2, (8, 8), "star", 1, "const", np.ones(5), "f32", "dirichlet")
                 for _ in range(30000)]
        del plans


def test_apply_argument_validation_needs_no_device():
    p = gs.stencil_plan(3, (8, 8, 8), "star", 1, "const", np.ones(7), "f32", "dirichlet")
    lib = api._lib()
    buf = ctypes.c_void_p(0x10000000)
    other = ctypes.c_void_p(0x20000000)
    assert lib.stencil_apply(None, buf, other, 1, None) == -1
    assert lib.stencil_apply(p.handle, None, other, 1, None) == -1
    assert lib.stencil_apply(p.handle, buf, None, 1, None) == -1
    assert lib.stencil_apply(p.handle, buf, other, 0, None) == -1
    assert lib.stencil_apply(p.handle, buf, buf, 1, None) == -1        # in == out
    assert lib.stencil_apply(p.handle, buf, ctypes.c_void_p(0x10000000 + 8), 1, None) == -1
    assert lib.stencil_apply_adjoint(p.handle, buf, buf, 1, None) == -1
    assert lib.stencil_apply_host(p.handle, None, other, 1, None) == -1
    pv = gs.stencil_plan(3, (8, 8, 8), "star", 1, "var", None, "f32", "dirichlet")
    assert lib.stencil_apply(pv.handle, buf, other, 1, None) == -1    # wrong entry for kind
    assert lib.stencil_batch_info(None, None, None, None) == -1


def test_variant_get_set_and_validation():
    p = gs.stencil_plan(3, (64, 64, 64), "star", 4, "const", np.ones(25), "f32", "periodic")
    v = gs.stencil_plan_get_variant(p)
    assert v["family"] == gs.FAMILY_STREAM and v["fuse"] == 1
    gs.stencil_plan_set_variant(p, block_x=32, block_y=4, vec_y=2, z_chunk=16)
    assert gs.stencil_plan_get_variant(p)["z_chunk"] == 16
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(p, block_x=32, block_y=16)   # 512 threads
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(p, family=gs.FAMILY_FUSED2D, fuse=2, tile_x=32, tile_y=32,
                                    block_x=128, block_y=1)     # fused 2D on a 3D plan
    assert gs.stencil_plan_get_variant(p)["z_chunk"] == 16      # unchanged on failure
    gs.stencil_plan_set_variant(p, stages=16)
    assert gs.stencil_plan_get_variant(p)["stages"] == 16
    for bad in (1, 17, -1):
        with pytest.raises(gs.StencilError):
            gs.stencil_plan_set_variant(p, stages=bad)          # ring depth 0 or 2..16
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(q := gs.stencil_plan(3, (64, 64, 64), "star", 1, "const",
                                                         np.ones(7), "f32", "periodic"),
                                    block_x=32, block_y=8)       # 256 consumer threads
    q = gs.stencil_plan(3, (64, 64, 64), "box", 4, "const", np.ones(729), "f32", "periodic")
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(q, vec_y=2)                  # not compiled for box r4
    p2 = gs.stencil_plan(2, (512, 512), "star", 1, "const", np.full(5, 0.2), "f32", "dirichlet")
    v2 = gs.stencil_plan_get_variant(p2)
    assert v2["family"] == gs.FAMILY_FUSED2D and v2["fuse"] > 1
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(p2, tile_x=512, tile_y=512)  # shared memory too large


def test_dispatch_map_file(tmp_path):
    m = tmp_path / "map.txt"
    m.write_text("# ndim shape r dtype bc kind class : family bx by vy zc fuse tx ty\n"
                 "3 0 4 0 1 0 -1 : 1 32 8 1 48 1 0 0\n"
                 "3 1 1 0 1 0 -1 : 1 32 4 2 32 1 0 0 6\n\n")
    gs.stencil_load_dispatch_map(str(m))
    try:
        p = gs.stencil_plan(3, (64, 64, 64), "star", 4, "const", np.ones(25), "f32", "periodic")
        v = gs.stencil_plan_get_variant(p)
        assert (v["block_x"], v["block_y"], v["vec_y"], v["z_chunk"]) == (32, 8, 1, 48)
        assert v["stages"] == 0                                  # optional field absent
        b = gs.stencil_plan(3, (64, 64, 64), "box", 1, "const", np.ones(27), "f32", "periodic")
        assert gs.stencil_plan_get_variant(b)["stages"] == 6
        q = gs.stencil_plan(3, (64, 64, 64), "star", 4, "const", np.ones(25), "f32", "dirichlet")
        assert gs.stencil_plan_get_variant(q)["z_chunk"] != 48   # key differs (boundary)
        bad = tmp_path / "bad.txt"
        bad.write_text("3 0 4 : nonsense\n")
        with pytest.raises(gs.StencilError):
            gs.stencil_load_dispatch_map(str(bad))
        with pytest.raises(gs.StencilError):
            gs.stencil_load_dispatch_map(str(tmp_path / "missing.txt"))
    finally:
        gs.stencil_load_dispatch_map(None)
    p = gs.stencil_plan(3, (64, 64, 64), "star", 4, "const", np.ones(25), "f32", "periodic")
    assert gs.stencil_plan_get_variant(p)["z_chunk"] != 48


def test_size_classes():
    assert [gs.stencil_size_class(n) for n in (1, 1 << 16, 1 << 20, 1 << 24, 1 << 30)] == \
        [0, 1, 2, 3, 3]


def test_batch_lines_in_the_dispatch_map(tmp_path):
    ok = tmp_path / "ok.txt"
    ok.write_text("batch 0 : 32 248 4\nbatch 2 : 16 120 2\n3 0 4 0 1 0 3 : 1 32 8 1 16 1 0 0\n")
    gs.stencil_load_dispatch_map(str(ok))
    gs.stencil_load_dispatch_map(None)
    for bad in ("batch 3 : 32 248 4\n", "batch 0 : 0 248 4\n", "batch 0 : 32 248\n"):
        m = tmp_path / "bad.txt"
        m.write_text(bad)
        with pytest.raises(gs.StencilError):
            gs.stencil_load_dispatch_map(str(m))


def test_geometry_classes_and_slab_keys(tmp_path):
    assert gs.stencil_geometry_class(3, (512, 512, 512)) == 0
    assert gs.stencil_geometry_class(3, (32, 1024, 1024)) == 1
    assert gs.stencil_geometry_class(3, (64, 512, 511)) == 0      # nz * 8 > nx
    assert gs.stencil_geometry_class(2, (8, 4096)) == 0           # 2D grids: one class
    # a slab-only entry, then a catch-all one for the same key without the geometry field
    m = tmp_path / "map.txt"
    m.write_text("3 0 4 0 1 0 3 1 : 1 32 4 2 48 1 0 0 3\n"
                 "3 0 4 0 1 0 3 : 1 32 8 1 16 1 0 0\n")
    gs.stencil_load_dispatch_map(str(m))
    try:
        c = np.ones(25)
        slab = gs.stencil_plan(3, (32, 1024, 1024), "star", 4, "const", c, "f32", "periodic")
        cube = gs.stencil_plan(3, (256, 256, 256), "star", 4, "const", c, "f32", "periodic")
        assert gs.stencil_plan_get_variant(slab)["z_chunk"] == 48
        assert gs.stencil_plan_get_variant(cube)["z_chunk"] == 16
    finally:
        gs.stencil_load_dispatch_map(None)


def test_library_missing_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(api, "_LIB", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        api._lib()


def _plan_for(ndim, dims, shape, r, dtype, bc, kind):
    if kind == "divkgrad":
        return gs.stencil_plan(ndim, dims, "star", 1, "divkgrad", None, dtype, bc)
    if kind == "var":
        return gs.stencil_plan(ndim, dims, shape, r, "var", None, dtype, bc)
    return gs.stencil_plan(ndim, dims, shape, r, "const",
                           np.ones(len(oracle.offsets(ndim, shape, r))), dtype, bc)


def test_autotuner_ranking_prefers_the_aligned_split_on_ties():
    from paper_2609_06694_gb300 import autotune

    def ev(ms, zc, by=14):
        return {"ms": ms, "variant": {"z_chunk": zc, "block_y": by}}

    # within 1% of the fastest: the column-aligned split wins
    r = autotune.rank_timings([ev(0.2000, 0), ev(0.2015, -1), ev(0.2100, 64)])
    assert r[0]["variant"]["z_chunk"] == -1 and [e["ms"] for e in r[1:]] == [0.2000, 0.2100]
    # beyond 1%: the fastest stays first
    r = autotune.rank_timings([ev(0.2030, -1), ev(0.2000, 0)])
    assert r[0]["variant"]["z_chunk"] == 0
    # no aligned candidate: plain order by time
    assert [e["ms"] for e in autotune.rank_timings([ev(0.3, 0), ev(0.1, 64)])] == [0.1, 0.3]
    assert autotune.rank_timings([]) == []


def test_autotuner_candidates_are_variants_the_library_accepts():
    # every candidate the tuner would time is a variant the plan validation accepts, so a
    # tuning run never spends its time on launches the library refuses (host logic only)
    from paper_2609_06694_gb300 import autotune
    seen = 0
    for key in autotune.tuning_set():
        ndim, dims, shape, r, dtype, bc, steps = key[:7]
        kind = key[7] if len(key) > 7 else "const"
        plan = _plan_for(ndim, dims, shape, r, dtype, bc, kind)
        if kind == "divkgrad":
            cands = autotune.divkgrad_candidates(dtype)
        elif kind == "var":
            cands = autotune.var_candidates(dtype)
        elif ndim == 2 and steps > 1:
            cands = autotune.fused2d_candidates(r, steps)
        else:
            cands = autotune.stream_candidates(ndim, shape, r, dtype)
            if ndim == 3 and (shape, r) in autotune.FUSED3D_SETS:
                cands = cands + autotune.fused3d_candidates(shape, r, dtype)
            if autotune.tensor_applies(ndim, dims, shape, r, dtype, bc, kind):
                cands = cands + autotune.tensor_candidates(ndim)
        assert cands, key
        for v in cands:
            gs.stencil_plan_set_variant(plan, **v)
            got = gs.stencil_plan_get_variant(plan)
            assert all(got[k] == val for k, val in v.items()), (key, v, got)
            seen += 1
    assert seen > 500


def test_column_split_variant_validation():
    # z_chunk -1 (aligned chunks per tile column) is a work split of the streaming and div(k
    # grad u) kernels; the general variable-coefficient sweeps and the fused kernels take none
    p = gs.stencil_plan(3, (64, 64, 64), "star", 4, "const", np.ones(25), "f32", "periodic")
    v = gs.stencil_plan_get_variant(p)
    gs.stencil_plan_set_variant(p, **dict(v, z_chunk=-1))
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(p, **dict(v, z_chunk=-2))
    d = gs.stencil_plan(3, (64, 64, 64), "star", 1, "divkgrad", None, "bf16", "dirichlet")
    gs.stencil_plan_set_variant(d, **dict(gs.stencil_plan_get_variant(d), z_chunk=-1))
    w = gs.stencil_plan(3, (64, 64, 64), "star", 1, "var", None, "f32", "dirichlet")
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(w, **dict(gs.stencil_plan_get_variant(w), z_chunk=-1))
    f = gs.stencil_plan(3, (64, 64, 64), "star", 1, "const", np.ones(7), "f32", "periodic")
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(f, family=gs.FAMILY_FUSED3D, block_x=32, block_y=4,
                                    vec_y=2, z_chunk=-1, fuse=2, tile_x=0, tile_y=0, stages=0)


def test_streaming_thread_caps():
    # 3D stars of radius >= 3 with one row per thread may take 8 warps of consumers, with two
    # rows per thread in f32 14 (one CTA per SM, taller tiles), every other streaming variant
    # 7; the CTA adds the producer warp
    p = gs.stencil_plan(3, (64, 64, 64), "star", 4, "const", np.ones(25), "f32", "periodic")
    gs.stencil_plan_set_variant(p, block_x=32, block_y=8, vec_y=1)
    for by, vy in ((9, 1), (15, 2), (8, 4)):
        with pytest.raises(gs.StencilError):
            gs.stencil_plan_set_variant(p, block_x=32, block_y=by, vec_y=vy)
    gs.stencil_plan_set_variant(p, block_x=32, block_y=14, vec_y=2)
    h = gs.stencil_plan(3, (64, 64, 64), "star", 4, "const", np.ones(25), "bf16", "periodic")
    gs.stencil_plan_set_variant(h, block_x=16, block_y=14, vec_y=2)
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(h, block_x=16, block_y=16, vec_y=2)
    b = gs.stencil_plan(3, (64, 64, 64), "box", 1, "const", np.ones(27), "bf16", "periodic")
    gs.stencil_plan_set_variant(b, block_x=16, block_y=14, vec_y=2)
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(b, block_x=16, block_y=16, vec_y=1)


def test_committed_dispatch_map_selects_its_entries():
    # the dispatch map shipped with the package loads, and a plan for each of its keys picks
    # the entry's variant (so the map still matches the library's keys and limits)
    path = os.path.join(ROOT, "paper_2609_06694_gb300", "dispatch_map.txt")
    gs.stencil_load_dispatch_map(path)
    shapes = {0: "star", 1: "box", 2: "diamond"}
    dtypes = {0: "f32", 1: "f16", 2: "bf16"}
    kinds = {0: "const", 1: "var", 2: "divkgrad"}
    names = ["family", "block_x", "block_y", "vec_y", "z_chunk", "fuse", "tile_x", "tile_y",
             "stages"]
    try:
        n = 0
        for line in open(path):
            line = line.split("#")[0].strip()
            if not line:
                continue
            key, val = line.split(":")
            if key.split()[0] == "batch":
                continue  # the batched launch's shape (read by stencil_batch_plan)
            fields = [int(t) for t in key.split()]
            ndim, shape, r, dt, bc, kind, cls = fields[:7]
            geo = fields[7] if len(fields) > 7 else 0
            want = dict(zip(names, (int(t) for t in val.split())))
            if geo == 1:  # z-slabs
                dims = (32, 1024, 1024) if cls == 3 else (16, 512, 512)
            else:
                dims = {3: (256, 256, 256), 2: (4096, 4096)}[ndim] if cls == 3 else \
                    {3: (128, 128, 128), 2: (1024, 1024)}[ndim] if cls == 2 else (512, 512)
            assert gs.stencil_geometry_class(ndim, dims) == geo, (line, dims)
            assert gs.stencil_size_class(int(np.prod(dims))) == cls, (line, dims)
            plan = _plan_for(ndim, dims, shapes[shape], r, dtypes[dt],
                             "periodic" if bc == 1 else "dirichlet", kinds[kind])
            got = gs.stencil_plan_get_variant(plan)
            assert all(got[k] == v for k, v in want.items()), (line, got)
            n += 1
        assert n >= 10
    finally:
        gs.stencil_load_dispatch_map(None)


def test_fused3d_variant_validation():
    f32 = dict(family=3, block_x=32, block_y=4, vec_y=2, z_chunk=16, fuse=2, tile_x=0,
               tile_y=0, stages=0)
    for shape, r, n in (("star", 1, 7), ("star", 2, 13), ("box", 1, 27), ("diamond", 2, 25)):
        p = gs.stencil_plan(3, (64, 64, 64), shape, r, "const", np.ones(n), "f32", "periodic")
        gs.stencil_plan_set_variant(p, **f32)
        assert gs.stencil_plan_get_variant(p)["family"] == 3
        for bad in (dict(fuse=3), dict(vec_y=1), dict(block_y=1), dict(block_y=8),
                    dict(block_x=16)):
            with pytest.raises(gs.StencilError):
                gs.stencil_plan_set_variant(p, **dict(f32, **bad))
    b = gs.stencil_plan(3, (64, 64, 64), "box", 1, "const", np.ones(27), "bf16", "dirichlet")
    gs.stencil_plan_set_variant(b, **dict(f32, block_x=16, block_y=8, vec_y=1))
    for shape, r, n in (("box", 2, 125), ("star", 3, 19)):
        p = gs.stencil_plan(3, (64, 64, 64), shape, r, "const", np.ones(n), "f32", "periodic")
        with pytest.raises(gs.StencilError) as e:
            gs.stencil_plan_set_variant(p, **f32)
        assert e.value.code == -2
    p2 = gs.stencil_plan(2, (64, 64), "box", 1, "const", np.ones(9), "f32", "periodic")
    with pytest.raises(gs.StencilError):
        gs.stencil_plan_set_variant(p2, **f32)


def test_tensor_variant_validation():
    # the tensor-core family runs the radius-2 box on 16-bit storage, zero Dirichlet, rows a
    # multiple of 8 cells; everything else is refused before any launch
    c125 = np.ones(125) / 125
    p = gs.stencil_plan(3, (8, 16, 16), "box", 2, "const", c125, "bf16", "dirichlet")
    gs.stencil_plan_set_variant(p, family=gs.FAMILY_TENSOR, tile_x=32, z_chunk=0, stages=0,
                                fuse=1, block_y=1, vec_y=2)  # two warps issue the MMAs
    assert gs.stencil_plan_get_variant(p)["family"] == gs.FAMILY_TENSOR
    p2 = gs.stencil_plan(2, (40, 24), "box", 2, "const", np.ones(25), "f16", "dirichlet")
    gs.stencil_plan_set_variant(p2, family=gs.FAMILY_TENSOR, tile_x=16, z_chunk=0, stages=0,
                                fuse=1, block_y=1, vec_y=0)
    for dtype, bc, dims, shape, r, n in (("f32", "dirichlet", (8, 16, 16), "box", 2, 125),
                                         ("bf16", "periodic", (8, 16, 16), "box", 2, 125),
                                         ("bf16", "dirichlet", (8, 16, 20), "box", 2, 125),
                                         ("bf16", "dirichlet", (8, 16, 16), "box", 1, 27),
                                         ("bf16", "dirichlet", (8, 16, 16), "star", 2, 13)):
        q = gs.stencil_plan(3, dims, shape, r, "const", np.ones(n), dtype, bc)
        with pytest.raises(gs.StencilError) as e:
            gs.stencil_plan_set_variant(q, family=gs.FAMILY_TENSOR, tile_x=16, z_chunk=0,
                                        stages=0, fuse=1, block_y=1, vec_y=1)
        assert e.value.code == -2
    gs.stencil_plan_set_variant(p, family=gs.FAMILY_TENSOR, tile_x=64, z_chunk=0, stages=0,
                                fuse=1, block_y=1, vec_y=4)  # four warps issue the MMAs
    for bad in (dict(tile_x=48), dict(tile_x=16, stages=4), dict(tile_x=16, stages=13),
                dict(tile_x=16, fuse=2), dict(tile_x=16, z_chunk=-1), dict(block_y=2),
                dict(vec_y=4), dict(vec_y=3, tile_x=64), dict(vec_y=8, tile_x=64),
                dict(vec_y=-1)):
        kw = dict(family=gs.FAMILY_TENSOR, tile_x=16, z_chunk=0, stages=0, fuse=1, block_y=1,
                  vec_y=1)
        kw.update(bad)
        with pytest.raises(gs.StencilError) as e:
            gs.stencil_plan_set_variant(p, **kw)
        assert e.value.code == -1


def test_every_map_line_is_a_recorded_autotuner_winner():
    # dispatch_map.txt holds no hand-set line: every line is the fastest candidate of its key in
    # dispatch_evidence.json (the autotuner's record), and every key carries the winner's ncu
    # DRAM counters
    import json
    pkg = os.path.join(ROOT, "paper_2609_06694_gb300")
    ev = json.load(open(os.path.join(pkg, "dispatch_evidence.json")))["keys"]
    names = ["family", "block_x", "block_y", "vec_y", "z_chunk", "fuse", "tile_x", "tile_y",
             "stages"]
    want = {}
    for e in ev:
        k, best = e["key"], e["fastest"][0]
        assert e.get("winner_ncu") and e["winner_ncu"]["dram_bytes_read"] > 0, k
        if "batch" in k:
            s = best["shape"]
            want[f"batch {api.DTYPES[k['batch']]}"] = [s["tile_y"], s["tile_x"], s["fuse"]]
        else:
            key = [k["ndim"], api.SHAPES[k["shape"]], k["radius"], api.DTYPES[k["dtype"]],
                   api.BOUNDARIES[k["boundary"]], api.KINDS[k["kind"]], k["size_class"],
                   k["geometry"]]
            want[" ".join(map(str, key))] = [best["variant"].get(n, 0) for n in names]
    lines = [ln.split("#")[0].strip() for ln in open(os.path.join(pkg, "dispatch_map.txt"))]
    lines = [ln for ln in lines if ln]
    assert len(lines) == len(want)
    for ln in lines:
        key, val = (part.strip() for part in ln.split(":"))
        assert key in want, ln
        assert [int(v) for v in val.split()] == want[key], ln

"""Benchmark of the stencil hot path on the 512^3 constant-coefficient workload.

Workload (one "step"): on a 512^3 f32 periodic grid with uniform[-1,1] input,
  (a) the 25-point radius-4 star with 8th-order Laplacian weights, 1 sweep and 8 sweeps;
  (b) the 27-point 3x3x3 box with seeded weights normalised to sum 1, 1 sweep and 8 sweeps;
18 sweeps = 18 * 512^3 cell updates.  Metric: Gcell-updates/s (higher is better).

Inputs are 512 MiB per array (larger than the 129 MB L2), so no L2 flush is needed between
timed iterations.  Timing: W untimed warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), measured with CUDA events on the launching stream; the maximum over
ranks is taken.  Several GPUs run independent replicas (weak scaling, no collective).

The same line carries `metric_ratios`: the adjoint against the forward sweep, div(k grad u)
per storage type, the batched launch against plain per-grid sweeps and the wave gradient
against its forward run, each with its own CUDA-event time (measured after the timed region).

--impl reference times the FP64 oracle (its OpenMP build, every host core) on the host on a
bounded sample of the same workload; that is this project's reference arm.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 512
CELLS = N ** 3
SWEEPS_PER_STEP = 1 + 8 + 1 + 8
ALG_BYTES_PER_CELL = 8  # f32: read one value, write one value per cell and sweep
METRIC = "Gcell-updates/s"
WORKLOAD = "3D const-coefficient sweeps 512^3 f32 periodic: 25-pt star r4 (8th-order " \
           "Laplacian) and 27-pt box (weights sum 1), 1 and 8 steps each"


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", str(r)))
    return r, w, lr


def reduce_over_ranks(value, op="max"):
    """MAX (or SUM) of a per-rank number over the ranks of the job (one process per GPU,
    replicas only); the number itself when the job has a single rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = (torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl"
           else torch.device("cpu"))
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(updates_per_rank, world, seconds):
    """Whole-job Gcell-updates/s: every rank's updates over the slowest rank's time."""
    return updates_per_rank * world / seconds / 1e9


NOMINAL_HBM_GBS = 8000.0  # GB/s, the nominal HBM3e rate of a GB300


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_workload(device, n=N):
    """Plans and device-resident inputs/outputs of the four sub-workloads."""
    import torch

    import paper_2609_06694_gb300 as gs
    from paper_2609_06694_gb300 import inputs

    dims = (n, n, n)
    star = gs.stencil_plan(3, dims, "star", 4, "const", np.ones(25), "f32", "periodic")
    offs_s = gs.stencil_offsets(star)
    c_star = inputs.laplacian_coeffs(offs_s, 4)
    star = gs.stencil_plan(3, dims, "star", 4, "const", c_star, "f32", "periodic")
    c_box, _ = inputs.normalised_sum_weights(2002, 27)
    box = gs.stencil_plan(3, dims, "box", 1, "const", c_box, "f32", "periodic")
    x_star = inputs.to_storage(inputs.uniform(2001, dims), "f32")
    x_box = inputs.to_storage(inputs.uniform(2003, dims), "f32")
    return {"star": star, "box": box, "x_star_host": x_star, "x_box_host": x_box,
            "x_star": x_star.to(device), "x_box": x_box.to(device),
            "y": torch.empty(dims, dtype=torch.float32, device=device),
            "c_star": c_star, "c_box": c_box, "offs_star": offs_s}


def run_step(gs, W, stream, ev=None, only=None):
    """The 18 sweeps; with ev, records events around each call: [(name, launches, s, e)]."""
    import torch
    calls = (("star", "x_star", 1), ("star", "x_star", 8), ("box", "x_box", 1),
             ("box", "x_box", 8))
    if only:
        calls = ((only, "x_" + only, 1),)
    for name, xin, steps in calls:
        if ev is not None:
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
        gs.stencil_apply(W[name], W[xin], W["y"], steps, stream=stream)
        if ev is not None:
            e.record(stream)
            ev.append((name, steps, s, e))


def kernel_source_sha():
    """sha256 prefix of the streaming kernel's sources (stream.cuh, then ring.cuh)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("stream.cuh", "ring.cuh"):
        with open(os.path.join(ROOT, "paper_2609_06694_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_tag):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    try:
        text = open(path).read()
        sha = kernel_source_sha()
        vals = {}
        for ln in text.splitlines():
            if ln.startswith("- ") and ":" in ln:
                k, v = ln[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
        if vals.get("kernel source sha256 prefix") != sha:
            return None
        return float(vals["dram bytes per launch"])
    except Exception:
        return None


def bench_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, lrank = rank_info()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(lrank)
    device = torch.device("cuda", lrank)
    from paper_2609_06694_gb300 import build
    build.build()
    import paper_2609_06694_gb300 as gs

    if args.only in ("divkgrad", "var", "wave", "batch", "fused3d", "reaction", "box2", "tensor"):
        profile_case(args)
        return
    W = build_workload(device, args.grid)
    stream = torch.cuda.current_stream(device)
    if args.only:
        # single-sweep profiling case (not a benchmark line)
        if args.variant:
            gs.stencil_plan_set_variant(W[args.only], **json.loads(args.variant))
        for _ in range(args.warmup + args.steps):
            run_step(gs, W, stream, only=args.only)
        torch.cuda.synchronize()
        rc = gs.stencil_sync_status(W[args.only])
        print(json.dumps({"profile_case": args.only, "grid": args.grid, "status": rc,
                          "variant": gs.stencil_plan_get_variant(W[args.only])}))
        if rc:
            raise SystemExit(1)
        return
    for _ in range(args.warmup):
        run_step(gs, W, stream)
    torch.cuda.synchronize()
    for name in ("star", "box"):
        rc = gs.stencil_sync_status(W[name])
        if rc != 0:
            raise RuntimeError(f"kernel error {rc}")

    sampler = ClockSampler(lrank)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = gs.stencil_launch_count()
    ev = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        run_step(gs, W, stream, ev)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = gs.stencil_launch_count() - launches0
    clocks = sampler.stop()
    ms_total = reduce_over_ranks(t0.elapsed_time(t1), "max")
    ms_per_step = ms_total / args.steps
    value = job_throughput(SWEEPS_PER_STEP * CELLS * args.steps, world, ms_total * 1e-3)

    # per-kernel timing from the events: star r4 sweep kernel is the dominant kernel
    per = {"star": [0.0, 0], "box": [0.0, 0]}
    for name, steps, s, e in ev:
        per[name][0] += s.elapsed_time(e)
        per[name][1] += steps
    dom = max(per, key=lambda k: per[k][0])
    ms_launch = per[dom][0] / per[dom][1]
    peak, peak_src = measured_peaks()
    achieved = ALG_BYTES_PER_CELL * CELLS / (ms_launch * 1e-3) / 1e9
    tag = "stream_sweep_star_r4_512" if dom == "star" else "stream_sweep_box_r1_512"
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic_from_profile(tag),
                "kernel": f"stream_sweep_kernel ({dom}), 1 sweep per launch",
                "peak_source": peak_src, "algorithmic_bytes_per_launch": ALG_BYTES_PER_CELL * CELLS,
                "ms_per_launch": round(ms_launch, 4),
                "per_kernel_ms_per_launch": {k: round(v[0] / v[1], 4) for k, v in per.items()},
                # the same against the nominal HBM3e rate the workload is quoted with
                "nominal_peak": NOMINAL_HBM_GBS,
                "frac_nominal": round(achieved / NOMINAL_HBM_GBS, 4)}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    xs = W["x_star_host"].pin_memory()
    xb = W["x_box_host"].pin_memory()
    yh = torch.empty((N, N, N), dtype=torch.float32).pin_memory()
    # host<->device copy times vary from call to call with the host's other memory traffic:
    # average over up to 10 steps
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 10))

    def e2e_step():
        gs.stencil_apply_host(W["star"], xs, yh, 1, stream=stream)
        gs.stencil_apply_host(W["star"], xs, yh, 8, stream=stream)
        gs.stencil_apply_host(W["box"], xb, yh, 1, stream=stream)
        gs.stencil_apply_host(W["box"], xb, yh, 8, stream=stream)

    e2e_val = None
    if e2e_steps:
        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        h0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = reduce_over_ranks(time.perf_counter() - h0, "max")
        e2e_val = round(job_throughput(SWEEPS_PER_STEP * CELLS * e2e_steps, world, e2e_s), 3)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(W)
    ratios = None
    if rank == 0 and not args.no_ratios:
        ratios = measure_metric_ratios(W)

    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gcell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N, N, N], "boundary": "periodic",
                       "sweeps_per_step": SWEEPS_PER_STEP, "l2": "inputs 512 MiB > L2, no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "Gcell-updates/s",
                    "h2d_bytes_per_step": 4 * CELLS * 4, "d2h_bytes_per_step": 4 * CELLS * 4,
                    "api": "stencil_apply_host (pinned host buffers)"},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "metric_ratios": ratios,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def tuned_variant(ndim, dims, shape, radius, dtype, bc, family=None):
    """The fastest variant the autotuner timed for this workload (of `family` if given, else
    of any family but the tensor cores), from the package's dispatch evidence; None if the
    key or such a variant is not there."""
    import paper_2609_06694_gb300 as gs
    path = os.path.join(os.path.dirname(gs.api.DISPATCH_MAP), "dispatch_evidence.json")
    try:
        with open(path) as f:
            keys = json.load(f)["keys"]
    except (OSError, ValueError, KeyError):
        return None
    for k in keys:
        kk = k["key"]
        if (kk.get("ndim") == ndim and tuple(kk.get("dims", ())) == tuple(dims) and
                kk.get("shape") == shape and kk.get("radius") == radius and
                kk.get("dtype") == dtype and kk.get("boundary") == bc):
            for e in k["fastest"]:
                fam = e["variant"]["family"]
                if (fam == family) if family is not None else (fam != gs.FAMILY_TENSOR):
                    return e["variant"]
    return None


def profile_case(args):
    """Single-kernel profiling cases of the other workloads (no JSON benchmark line)."""
    import torch

    import paper_2609_06694_gb300 as gs
    from paper_2609_06694_gb300 import inputs
    from paper_2609_06694_gb300 import wave as W
    if args.only == "tensor":
        # the 125-point box at 384^3 in bf16, zero Dirichlet, on the tensor cores (Toeplitz
        # packing; the dispatch map's variant, else 64 outputs per CTA along x, four warps
        # issuing the MMAs, one wave of z chunks)
        n = args.grid if args.grid != N else 384
        dims = (n, n, n)
        c, _ = inputs.normalised_sum_weights(2002, 125)
        x = inputs.to_storage(inputs.uniform(2003, dims), "bf16").cuda()
        y = torch.empty_like(x)
        plan = gs.stencil_plan(3, dims, "box", 2, "const", c, "bf16", "dirichlet")
        if gs.stencil_plan_get_variant(plan)["family"] != gs.FAMILY_TENSOR:
            gs.stencil_plan_set_variant(plan, family=gs.FAMILY_TENSOR, block_y=1, vec_y=4,
                                        tile_x=64, z_chunk=0, stages=0, fuse=1)
        for _ in range(args.warmup + args.steps):
            gs.stencil_apply(plan, x, y, 1)
        rc = gs.stencil_sync_status(plan)
    elif args.only in ("fused3d", "reaction", "box2"):
        # fused3d: two fused 7-point steps per launch at 512^3 (the dispatch map's choice for
        # this key); reaction: one Allen-Cahn step with the 7-point Laplacian at 512^3;
        # box2: one sweep of the 125-point box at 384^3 (the compute-bound corner)
        n = args.grid if args.grid != N else (384 if args.only == "box2" else 512)
        dims = (n, n, n)
        x = inputs.to_storage(inputs.uniform(2003, dims), "f32").cuda()
        y = torch.empty_like(x)
        if args.only == "box2":
            c = inputs.normalised_abs_weights(7, 125)
            plan = gs.stencil_plan(3, dims, "box", 2, "const", c, "f32", "periodic")
            fn = lambda: gs.stencil_apply(plan, x, y, 1)  # noqa: E731
        else:
            c7 = np.array([1.0, 1.0, 1.0, -6.0, 1.0, 1.0, 1.0]) / 6.0
            plan = gs.stencil_plan(3, dims, "star", 1, "const", c7, "f32", "periodic")
            if args.only == "fused3d":
                gs.stencil_plan_set_variant(plan, family=gs.FAMILY_FUSED3D, block_x=32,
                                            block_y=6, vec_y=2, z_chunk=64, fuse=2, tile_x=0,
                                            tile_y=0, stages=6)
                fn = lambda: gs.stencil_apply(plan, x, y, 2)  # noqa: E731
            else:
                fn = lambda: gs.stencil_apply_reaction(plan, x, y, 1, 0.1, 1.0, -1.0)  # noqa
        for _ in range(args.warmup + args.steps):
            fn()
        rc = gs.stencil_sync_status(plan)
    elif args.only == "divkgrad":
        n = args.grid if args.grid != N else 384
        dt = args.dtype
        plan = gs.stencil_plan(3, (n, n, n), "star", 1, "divkgrad", None, dt, "dirichlet")
        k = inputs.to_storage(inputs.lognormal_k(3002, (n, n, n)), dt).cuda()
        u = inputs.to_storage(inputs.uniform(3001, (n, n, n)), dt).cuda()
        y = torch.empty_like(u)
        for _ in range(args.warmup + args.steps):
            gs.stencil_apply_var(plan, u, [k], y, 1)
        rc = gs.stencil_sync_status(plan)
    elif args.only == "var":
        # general variable coefficients: 3D star r1, 7 coefficient arrays, forward sweep
        n = args.grid if args.grid != N else 384
        plan = gs.stencil_plan(3, (n, n, n), "star", 1, "var", None, "f32", "dirichlet")
        u = inputs.to_storage(inputs.uniform(3101, (n, n, n)), "f32").cuda()
        w = [inputs.to_storage(inputs.uniform(3110 + i, (n, n, n)), "f32").cuda()
             for i in range(7)]
        y = torch.empty_like(u)
        for _ in range(args.warmup + args.steps):
            gs.stencil_apply_var(plan, u, w, y, 1)
        rc = gs.stencil_sync_status(plan)
    elif args.only == "wave":
        n3 = (256, 256, 256)
        lp = gs.stencil_plan(3, n3, "star", 4, "const", np.ones(25), "f32", "dirichlet")
        lap = inputs.laplacian_coeffs(gs.stencil_offsets(lp), 4)
        dt = 0.4 * 10.0 / 4500.0
        steps = 20
        wp = W.wave_plan(n3, 4, lap, 10.0, dt, steps, (10, 128, 128),
                         inputs.ricker(15.0, dt, steps), 10, 25)
        v = torch.from_numpy(inputs.velocity_field(5001, n3).astype(np.float32)).cuda()
        tr = torch.empty(wp.trace_shape, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup + args.steps):
            W.wave_forward(wp, v, tr)
        torch.cuda.synchronize()
        rc = 0
    else:
        specs = inputs.batched_grid_specs()
        items = []
        for sp in specs:
            d = (sp["ny"], sp["nx"])
            npts = {"star": 4 * sp["radius"] + 1, "box": (2 * sp["radius"] + 1) ** 2}[sp["shape"]]
            c = inputs.normalised_abs_weights(sp["weight_seed"], npts)
            pl = gs.stencil_plan(2, d, sp["shape"], sp["radius"], "const", c, "f32", "dirichlet")
            xi = inputs.to_storage(inputs.uniform(sp["input_seed"], d), "f32").cuda()
            items.append((pl, xi, torch.empty_like(xi)))
        batch = gs.stencil_batch_plan(items, 20)
        for _ in range(args.warmup + args.steps):
            gs.stencil_batch_launch(batch)
        rc = gs.stencil_batch_status(batch)
    print(json.dumps({"profile_case": args.only, "status": rc}))
    if rc:
        raise SystemExit(1)


def _oracle_sample(seed_star=2001, seed_box=2003, nz=16):
    """One oracle sweep of each stencil on an nz x 512 x 512 periodic f64 grid; returns
    (cell updates, seconds, description)."""
    import oracle
    from paper_2609_06694_gb300 import inputs
    dims = (nz, N, N)
    offs_s = oracle.offsets(3, "star", 4)
    c_s = inputs.laplacian_coeffs(offs_s, 4)
    offs_b = oracle.offsets(3, "box", 1)
    c_b, _ = inputs.normalised_sum_weights(2002, 27)
    xs = inputs.stored_values(inputs.to_storage(inputs.uniform(seed_star, dims), "f32"))
    xb = inputs.stored_values(inputs.to_storage(inputs.uniform(seed_box, dims), "f32"))
    t0 = time.perf_counter()
    oracle.sweep_const(xs, offs_s, c_s, "periodic")
    oracle.sweep_const(xb, offs_b, c_b, "periodic")
    dt = time.perf_counter() - t0
    desc = (f"one FP64 oracle sweep of the 25-pt star and of the 27-pt box on a {nz}x512x512 "
            f"periodic grid (same per-cell work as the 512^3 sweeps), {oracle.threads()} "
            "host thread(s)")
    return 2 * nz * N * N, dt, desc


def cpu_baseline_sample(W=None):
    """The oracle on every host core (its OpenMP build: cell loops split over threads) over
    the whole 512^3 grid, one sweep of each stencil; the single-thread rate on a 64-plane slab
    is reported beside it."""
    import oracle
    oracle.use_threads(1)
    u1, t1, _ = _oracle_sample(nz=64)
    cores = oracle.use_threads(0)
    try:
        updates, dt, desc = _oracle_sample(nz=N)
    finally:
        oracle.use_threads(1)
    return {"value": round(updates / dt / 1e9, 6), "unit": "Gcell-updates/s", "cores": cores,
            "kind": "oracle", "sample": desc, "seconds": round(dt, 2),
            "single_thread_value": round(u1 / t1 / 1e9, 6)}


def bench_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on every host core (rank 0 only),
    each step one sweep of each stencil on a 64 x 512 x 512 periodic slab."""
    rank, world, _ = rank_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = oracle.use_threads(0)
    for _ in range(args.warmup):
        _oracle_sample(nz=16)
    total_u, total_t = 0, 0.0
    desc = None
    for _ in range(args.steps):
        u, dt, desc = _oracle_sample(nz=64)
        total_u += u
        total_t += dt
    oracle.use_threads(1)
    value = total_u / total_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6),
        "unit": "Gcell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_t / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N, N, N], "boundary": "periodic",
                   "sample": desc},
        "cpu_baseline": {"value": round(value, 6), "unit": "Gcell-updates/s", "cores": cores,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": round(value, 6), "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# --suite: the other workloads, one JSON line each (reported next to the bench line; not bench
# lines themselves).  Times are CUDA-event medians over `reps` runs after warm-up.
# ------------------------------------------------------------------------------------------
def _time(fn, reps=5, warm=2):
    import torch
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e))
    return float(np.median(ts))


def _frac(gbytes, ms, peak):
    gbs = gbytes / (ms * 1e-3)
    return round(gbs, 1), round(gbs / peak, 4)


def measure_metric_ratios(W3=None, wave=True):
    """The metric's other terms, measured on this GPU: the adjoint against the forward sweep
    (512^3 star r4 and box, the 384^3 variable-coefficient star), div(k grad u) per storage
    type, the batched launch against plain per-grid sweeps (256 grids x 20 steps, f32 and
    bf16) and the wave-equation gradient against its forward run.  Every entry carries its own
    CUDA-event median time and, where the bytes are fixed, its fraction of the measured HBM
    copy rate.  Returns {name: entry}."""
    import torch

    import paper_2609_06694_gb300 as gs
    from paper_2609_06694_gb300 import inputs
    from paper_2609_06694_gb300 import wave as WV

    peak, _ = measured_peaks()
    out = {}
    own = W3 is None
    if own:
        W3 = build_workload(torch.device("cuda", torch.cuda.current_device()))
    for name, xin in (("star", "x_star"), ("box", "x_box")):
        ms_f = _time(lambda: gs.stencil_apply(W3[name], W3[xin], W3["y"], 1))
        ms_a = _time(lambda: gs.stencil_apply_adjoint(W3[name], W3[xin], W3["y"], 1))
        gbs_f, fr_f = _frac(8 * CELLS / 1e9, ms_f, peak)
        gbs_a, fr_a = _frac(8 * CELLS / 1e9, ms_a, peak)
        out[f"adjoint_{name}_512"] = {
            "workload": f"512^3 f32 periodic {'25-pt star r4' if name == 'star' else '27-pt box'}, "
                        "1 sweep: adjoint (offset-flipped) vs forward",
            "ms_forward": round(ms_f, 4), "ms_adjoint": round(ms_a, 4),
            "adjoint_over_forward": round(ms_a / ms_f, 3),
            "frac_hbm_forward": fr_f, "frac_hbm_adjoint": fr_a}
        ms8 = _time(lambda: gs.stencil_apply(W3[name], W3[xin], W3["y"], 8), reps=3)
        out[f"steps8_{name}_512"] = {
            "workload": f"512^3 f32 periodic {name}, 8 steps", "ms": round(ms8, 4),
            "Gcell_updates_per_s": round(CELLS * 8 / ms8 / 1e6, 2),
            "frac_hbm": _frac(8 * 8 * CELLS / 1e9, ms8, peak)[1]}
    # temporal blocking in 3D: 8 steps as four fused pairs against eight single sweeps, and
    # the reaction-diffusion step (stencil + pointwise physics in one launch) against the plain
    # sweep of the same stencil
    dims = (N, N, N)
    c7 = np.array([1.0, 1.0, 1.0, -6.0, 1.0, 1.0, 1.0]) / 6.0
    c27, _ = inputs.normalised_sum_weights(2002, 27)
    for name, shape, c, by in (("star1", "star", c7, 7), ("box", "box", c27, 7)):
        plain = gs.stencil_plan(3, dims, shape, 1, "const", c, "f32", "periodic")
        if gs.stencil_plan_get_variant(plain)["family"] != gs.FAMILY_STREAM:
            # the map's entry for this key may be the fused kernel: single sweeps on the
            # fastest streaming variant the autotuner timed (else a tile tuned for the box)
            best = tuned_variant(3, dims, shape, 1, "f32", "periodic", gs.FAMILY_STREAM) or dict(
                family=gs.FAMILY_STREAM, block_x=32, block_y=4, vec_y=2, z_chunk=32, fuse=1,
                tile_x=0, tile_y=0, stages=0)
            gs.stencil_plan_set_variant(plain, **best)
        fused = gs.stencil_plan(3, dims, shape, 1, "const", c, "f32", "periodic")
        gs.stencil_plan_set_variant(fused, family=gs.FAMILY_FUSED3D, block_x=32, block_y=by,
                                    vec_y=2, z_chunk=64, fuse=2, tile_x=0, tile_y=0, stages=0)
        ms_p = _time(lambda: gs.stencil_apply(plain, W3["x_box"], W3["y"], 8), reps=3)
        ms_f = _time(lambda: gs.stencil_apply(fused, W3["x_box"], W3["y"], 8), reps=3)
        out[f"fused3d_{name}_512_8steps"] = {
            "workload": f"512^3 f32 periodic {shape} r1, 8 steps: four two-step fused launches "
                        "vs eight single sweeps",
            "ms_single_sweeps": round(ms_p, 4), "ms_fused_pairs": round(ms_f, 4),
            "fused_speedup": round(ms_p / ms_f, 3),
            "frac_hbm_single": _frac(8 * 8 * CELLS / 1e9, ms_p, peak)[1],
            "frac_hbm_fused_equivalent": _frac(8 * 8 * CELLS / 1e9, ms_f, peak)[1]}
        if name == "star1":
            ms_1 = _time(lambda: gs.stencil_apply(plain, W3["x_box"], W3["y"], 1))
            ms_r = _time(lambda: gs.stencil_apply_reaction(plain, W3["x_box"], W3["y"], 1, 0.1,
                                                           1.0, -1.0))
            out["reaction_star1_512"] = {
                "workload": "512^3 f32 periodic Allen-Cahn step u + dt (L u + u - u^3), 7-point "
                            "Laplacian, fused in one launch, vs the plain sweep",
                "ms_sweep": round(ms_1, 4), "ms_reaction_step": round(ms_r, 4),
                "reaction_over_sweep": round(ms_r / ms_1, 3),
                "frac_hbm_reaction": _frac(8 * CELLS / 1e9, ms_r, peak)[1]}
        del plain, fused
    if own:
        del W3
        torch.cuda.empty_cache()

    # the 125-point box in 16-bit storage: the CUDA-core streaming sweep against the tensor-core
    # Toeplitz kernel (the dispatch map's variant for the key when it picks the tensor family,
    # else 64 outputs per CTA, four MMA-issuing warps and one wave of z chunks)
    n = 384
    c125, _ = inputs.normalised_sum_weights(2002, 125)
    for dt in ("bf16", "f16"):
        dims = (n, n, n)
        x = inputs.to_storage(inputs.uniform(2003, dims), dt).cuda()
        y = torch.empty_like(x)
        core = gs.stencil_plan(3, dims, "box", 2, "const", c125, dt, "dirichlet")
        tens = gs.stencil_plan(3, dims, "box", 2, "const", c125, dt, "dirichlet")
        if gs.stencil_plan_get_variant(tens)["family"] != gs.FAMILY_TENSOR:
            gs.stencil_plan_set_variant(tens, family=gs.FAMILY_TENSOR, block_y=1, vec_y=4,
                                        tile_x=64, z_chunk=0, stages=0, fuse=1)
        # the CUDA-core side runs the fastest CUDA-core variant the autotuner timed for this
        # key (its evidence file), else the library default
        best = tuned_variant(3, dims, "box", 2, dt, "dirichlet")
        if best is not None:
            gs.stencil_plan_set_variant(core, **best)
        elif gs.stencil_plan_get_variant(core)["family"] == gs.FAMILY_TENSOR:
            gs.stencil_plan_set_variant(core, family=gs.FAMILY_STREAM, block_x=16, block_y=8,
                                        vec_y=2, z_chunk=64, fuse=1, tile_x=0, tile_y=0,
                                        stages=0)
        ms_c = _time(lambda: gs.stencil_apply(core, x, y, 1))
        ms_t = _time(lambda: gs.stencil_apply(tens, x, y, 1))
        useful = 2 * 125 * n ** 3  # FLOPs of the 125-point sweep
        out[f"box2_384_{dt}_tensor_cores"] = {
            "workload": f"384^3 {dt} zero-Dirichlet 125-point box, 1 sweep: tensor cores "
                        "(Toeplitz packing, tcgen05) vs the CUDA-core streaming sweep",
            "ms_cuda_cores": round(ms_c, 4), "ms_tensor_cores": round(ms_t, 4),
            "tensor_speedup": round(ms_c / ms_t, 3),
            "useful_TFLOPs_tensor": round(useful / ms_t / 1e9, 1),
            "tensor_variant": gs.stencil_plan_get_variant(tens),
            "cuda_core_variant": gs.stencil_plan_get_variant(core),
            "frac_hbm_tensor": _frac(4 * n ** 3 / 1e9, ms_t, peak)[1]}
        del core, tens, x, y

    n = 384
    for dt in ("f32", "bf16"):
        es = 4 if dt == "f32" else 2
        plan = gs.stencil_plan(3, (n, n, n), "star", 1, "var", None, dt, "dirichlet")
        u = inputs.to_storage(inputs.uniform(3101, (n, n, n)), dt).cuda()
        w = [inputs.to_storage(inputs.uniform(3110 + i, (n, n, n)), dt).cuda() for i in range(7)]
        y = torch.empty_like(u)
        ms_f = _time(lambda: gs.stencil_apply_var(plan, u, w, y, 1))
        ms_a = _time(lambda: gs.stencil_apply_adjoint_var(plan, u, w, y, 1))
        gb = 9 * es * n ** 3 / 1e9
        out[f"adjoint_var_star1_384_{dt}"] = {
            "workload": f"variable-coefficient star r1 384^3 {dt} Dirichlet (7 coefficient "
                        "arrays): adjoint (shifted gathers) vs forward",
            "ms_forward": round(ms_f, 4), "ms_adjoint": round(ms_a, 4),
            "adjoint_over_forward": round(ms_a / ms_f, 3),
            "frac_hbm_forward": _frac(gb, ms_f, peak)[1],
            "frac_hbm_adjoint": _frac(gb, ms_a, peak)[1]}
        del u, w, y
    torch.cuda.empty_cache()

    kk = inputs.lognormal_k(3002, (n, n, n))
    uu = inputs.uniform(3001, (n, n, n))
    for dt in ("f32", "f16", "bf16"):
        es = 4 if dt == "f32" else 2
        plan = gs.stencil_plan(3, (n, n, n), "star", 1, "divkgrad", None, dt, "dirichlet")
        k = inputs.to_storage(kk, dt).cuda()
        u = inputs.to_storage(uu, dt).cuda()
        y = torch.empty_like(u)
        ms = _time(lambda: gs.stencil_apply_var(plan, u, [k], y, 1))
        gbs, fr = _frac(3 * es * n ** 3 / 1e9, ms, peak)
        out[f"divkgrad_384_{dt}"] = {
            "workload": f"div(k grad u) 384^3 {dt} Dirichlet, 1 step", "ms": round(ms, 4),
            "Gcell_updates_per_s": round(n ** 3 / ms / 1e6, 2), "alg_GBps": gbs,
            "frac_hbm": fr}
        del k, u, y
    del kk, uu
    torch.cuda.empty_cache()

    specs = inputs.batched_grid_specs()
    for dt in ("f32", "bf16"):
        items = []
        cells = 0
        for sp in specs:
            d = (sp["ny"], sp["nx"])
            npts = {"star": 4 * sp["radius"] + 1, "box": (2 * sp["radius"] + 1) ** 2}[sp["shape"]]
            c = inputs.normalised_abs_weights(sp["weight_seed"], npts)
            pl = gs.stencil_plan(2, d, sp["shape"], sp["radius"], "const", c, dt, "dirichlet")
            xi = inputs.to_storage(inputs.uniform(sp["input_seed"], d), dt).cuda()
            items.append((pl, xi, torch.empty_like(xi)))
            cells += d[0] * d[1]
        batch = gs.stencil_batch_plan(items, 20)
        ms_b = _time(lambda: gs.stencil_batch_launch(batch), reps=5)

        def plain_single_steps():
            for pl, xi, yi in items:
                gs.stencil_apply(pl, xi, yi, 1)

        ms_1 = _time(plain_single_steps, reps=3, warm=1) * 20  # 256 x 20 single-step launches
        ms_20 = _time(lambda: [gs.stencil_apply(pl, xi, yi, 20) for pl, xi, yi in items],
                      reps=3, warm=1)
        es = 4 if dt == "f32" else 2
        gbs, fr = _frac(2 * es * cells * 20 / 1e9, ms_b, peak)
        out[f"batched_256x20_{dt}"] = {
            "workload": f"batched 2D, 256 grids (sides log-uniform 64-2048), 20 steps, {dt}, "
                        "one persistent launch in a CUDA graph",
            "cells_per_step": cells, "ms_batched": round(ms_b, 3),
            "ms_plain_256x20_launches": round(ms_1, 3),
            "ms_plain_256_calls_of_20_steps": round(ms_20, 3),
            "batched_speedup_vs_256x20": round(ms_1 / ms_b, 2),
            "batched_speedup_vs_256_calls": round(ms_20 / ms_b, 2),
            "Gcell_updates_per_s": round(cells * 20 / ms_b / 1e6, 2), "alg_GBps": gbs,
            "frac_hbm": fr, "batch": gs.stencil_batch_info(batch)}
        del batch, items
    torch.cuda.empty_cache()

    if wave:
        n3 = (256, 256, 256)
        lap_plan = gs.stencil_plan(3, n3, "star", 4, "const", np.ones(25), "f32", "dirichlet")
        lap = inputs.laplacian_coeffs(gs.stencil_offsets(lap_plan), 4)
        h, steps = 10.0, 500
        dtw = 0.4 * h / 4500.0
        wl = inputs.ricker(15.0, dtw, steps)
        v = inputs.velocity_field(5001, n3)
        vt = inputs.perturbed_velocity(v)
        wp = WV.wave_plan(n3, 4, lap, h, dtw, steps, (10, 128, 128), wl, 10, 25)
        v32 = torch.from_numpy(v.astype(np.float32)).cuda()
        vt32 = torch.from_numpy(vt.astype(np.float32)).cuda()
        obs = torch.empty(wp.trace_shape, dtype=torch.float32, device="cuda")
        WV.wave_forward(wp, vt32, obs)
        tr = torch.empty_like(obs)
        J = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.empty(n3, dtype=torch.float64, device="cuda")
        ms_f = _time(lambda: WV.wave_forward(wp, v32, tr), reps=3, warm=1)
        ms_g = _time(lambda: WV.wave_gradient(wp, v32, obs, tr, J, g), reps=3, warm=1)
        rc = WV.wave_sync_status(wp)
        cells = 256 ** 3
        out["wave_256_500"] = {
            "workload": "3D acoustic wave 256^3, r4 Laplacian, 500 leapfrog steps; gradient by "
                        "the adjoint with checkpoints every 25 steps (forward + recompute + "
                        "adjoint, FP64 accumulation)",
            "ms_forward": round(ms_f, 2), "ms_gradient": round(ms_g, 2),
            "gradient_over_forward": round(ms_g / ms_f, 2),
            "forward_Gcell_updates_per_s": round(cells * steps / ms_f / 1e6, 2),
            "forward_frac_hbm": _frac(16 * cells * steps / 1e9, ms_f, peak)[1],
            "status": rc}
        del wp, v32, vt32, obs, tr, g
        torch.cuda.empty_cache()
    return out


def suite():
    import torch

    from paper_2609_06694_gb300 import build
    build.build()
    import paper_2609_06694_gb300 as gs
    from paper_2609_06694_gb300 import inputs

    torch.cuda.set_device(0)
    # 2D 5-point Jacobi 512^2, 10 steps (L2-resident: latency-bound, reported formally vs HBM)
    dims = (512, 512)
    plan = gs.stencil_plan(2, dims, "star", 1, "const", np.full(5, 0.2), "f32", "dirichlet")
    x = inputs.to_storage(inputs.uniform(1001, dims), "f32").cuda()
    y = torch.empty_like(x)
    ms = _time(lambda: gs.stencil_apply(plan, x, y, 10), reps=20)
    print(json.dumps({"workload": "2D Jacobi 512^2 f32 Dirichlet, 10 steps", "ms": round(ms, 4),
                      "Gcell_updates_per_s": round(512 * 512 * 10 / ms / 1e6, 2),
                      "variant": gs.stencil_plan_get_variant(plan),
                      "note": "1 MiB grid stays in L2: latency-bound, not HBM-bound"}),
          flush=True)
    for name, row in measure_metric_ratios().items():
        print(json.dumps(dict(row, key=name)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ratios", action="store_true",
                    help="skip the adjoint / batched / div(k grad u) / wave measurements that "
                         "the bench line carries under metric_ratios")
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default="f32",
                    help="storage type of the div(k grad u) profiling case")
    ap.add_argument("--only", choices=["star", "box", "divkgrad", "var", "wave", "batch", "tensor",
                                       "fused3d", "reaction", "box2"],
                    default=None,
                    help="profiling case: only the 1-sweep call of one stencil, no JSON line")
    ap.add_argument("--grid", type=int, default=N, help="cube side (profiling cases only)")
    ap.add_argument("--suite", action="store_true",
                    help="measure the other workloads (one JSON line each) instead")
    ap.add_argument("--variant", default=None,
                    help="profiling case: JSON dict of stencil_variant fields to force")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: at least 3 warm-up steps are required; using 3", file=sys.stderr)
        args.warmup = 3
    if args.suite:
        suite()
        return
    if args.only is None:
        args.grid = N  # the benchmark line is always the 512^3 workload
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()

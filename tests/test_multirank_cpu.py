"""The multi-GPU path of the benchmark is replicas only: one process per GPU, each running the
whole workload, no collective on the data path; the job's time is the slowest rank's and its
value is every rank's updates over that time.  These checks run that host logic as two gloo
ranks on the CPU (the same reduction code the NCCL ranks run on GPUs)."""
import contextlib
import io
import os
import socket
import types

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.rank_info()
        ms_max = bench.reduce_over_ranks(10.0 + 5.0 * rank, "max")   # per-rank step time
        total = bench.reduce_over_ranks(100.0 * (rank + 1), "sum")
        value = bench.job_throughput(1e9, w, ms_max * 1e-3)
        q.put((rank, r, w, lr, ms_max, total, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_benchmark():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seen = set()
    for rank, r, w, lr, ms_max, total, value in results:
        seen.add(rank)
        assert (r, w, lr) == (rank, world, rank)
        assert ms_max == 15.0                       # the slowest rank's time, on every rank
        assert total == 300.0
        assert value == pytest.approx(2 * 1e9 / 15e-3 / 1e9)   # both ranks' updates / slowest time
    assert seen == {0, 1}


def test_single_rank_needs_no_process_group():
    assert bench.reduce_over_ranks(3.5, "max") == 3.5
    assert bench.job_throughput(2e9, 1, 0.5) == pytest.approx(4.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    # under torchrun every rank but 0 leaves at once, printing nothing
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.bench_reference(types.SimpleNamespace(steps=1, warmup=1, gpus=2))
    assert out.getvalue() == ""


def test_committed_profile_matches_the_kernel_sources():
    # the bench line's roofline.traffic comes from the committed ncu summary of its dominant
    # kernel only while stream.cuh and ring.cuh hash as they did when it was captured: a change
    # to either file needs a new capture, not an edited hash
    assert bench.traffic_from_profile("stream_sweep_star_r4_512") is not None

"""bench.py's multi-rank host logic on CPU ranks (gloo, world size 2): the
max-over-ranks timing, the barrier, the whole-job throughput, and the
reference arm under a two-rank launch (rank 0 alone runs and prints).  The
step itself has no exchange (replicas only), so this is all of the N > 1
path that does not need GPUs."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        bench.barrier(w)
        elapsed = 1.0 + rank  # rank 1 is the slower one
        emax = bench.max_over_ranks(elapsed, w)
        value = bench.job_mlups(w, 1000, 10, emax)
        bench.barrier(w)
        out.put((r, local, emax, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_job_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1] and [loc for _, loc, *_ in res] == [0, 1]
    for _, _, emax, value in res:
        assert emax == 2.0
        assert value == pytest.approx(2 * 1000 * 10 / 2.0 / 1e6)


def test_reference_arm_under_two_ranks():
    env = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "3"]
    r1 = subprocess.run(cmd, env=dict(env, RANK="1", LOCAL_RANK="1"), capture_output=True, text=True,
                        timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = subprocess.run(cmd, env=dict(env, RANK="0", LOCAL_RANK="0"), capture_output=True, text=True,
                        timeout=300)
    assert r0.returncode == 0
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["unit"] == "MLUPS"
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    # the same workload config the GPU arm prints (one helper builds both)
    sys.path.insert(0, ROOT)
    import bench
    assert line["config"] == bench.workload_config(2)
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True

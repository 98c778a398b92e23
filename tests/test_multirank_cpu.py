"""N > 1 host logic on CPU (gloo, world size 2): the benchmark's replica aggregation
(slowest rank's time, sum of all ranks' units) and the reference arm under torchrun
(rank 0 prints one JSON line, the other ranks exit 0 without work)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, units = bench.aggregate_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1))
    out.put((rank, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in res:
        assert ms == 15.0          # max over ranks
        assert units == 3000.0     # sum over ranks


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(29700 + os.getpid() % 200),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1",
           "--cpu-cores", "2"]
    import time
    t0 = time.perf_counter()
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "DOF-updates/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    # the printed time per step is measured on the sample that ran: K steps of it fit in the run
    assert d["cpu_baseline"]["cores"] == 2
    assert 0 < d["ms_per_step"] * d["steps"] / 1e3 < wall
    assert abs(d["value"] - 2 * d["config"]["sample_dofs"] / (d["ms_per_step"] / 1e3)) <= 1e-9 * d["value"]

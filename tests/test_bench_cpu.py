"""bench.py on the CPU: the reference arm (the oracle on the host cores)
keeps the JSON contract of the benchmark line, and the multi-rank timing
(max over ranks, work summed over ranks) holds on two gloo ranks."""
import json
import os
import subprocess
import sys

from conftest import ROOT


def _bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=600, env=e, cwd=ROOT)
    return r


def test_reference_arm_prints_one_contract_line():
    r = _bench("--impl", "reference", "--workload", "cfg2", "--steps", "1", "--warmup", "3", "--cpu-rows", "400")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "TFLOP/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("cfg2") and d["config"]["sample_rows"] == 400
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_warmup_floor_and_unavailable_workloads():
    # the default workload is the bf16 65536 x 16384 matrix (row-sampled here)
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--cpu-rows", "300", "--cpu-cols", "300")
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["warmup"] == 3                                                 # at least 3 warm-up steps
    assert d["config"]["workload"].startswith("cfg3")
    assert d["config"]["sample_rows"] == 300 and d["config"]["sample_cols"] == 300
    r = _bench("--impl", "reference", "--workload", "cfg4")
    assert r.returncode == 0
    d = json.loads(r.stdout.strip())
    assert d["impl"] == "reference" and "unavailable" in d


def test_reference_arm_prints_on_rank_zero_only():
    r = _bench("--impl", "reference", "--workload", "cfg2", "--steps", "1", "--warmup", "3", "--cpu-rows", "300",
               env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def _replica_rank(rank, world, port, root, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(1.0 + rank, world, "cpu")     # rank r took 1 + r ms
        q.put((rank, ms, bench.job_tflops(3e9, world, ms)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_work():
    # the N > 1 path: one independent problem per rank, no data-path
    # collective; the step time is the slowest rank's, the work is summed
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    procs = [ctx.Process(target=_replica_rank, args=(r, world, port, ROOT, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, ms, tf in got:
        assert ms == 2.0                                        # max over ranks
        assert abs(tf - 3e9 * world / 2e-3 / 1e12) < 1e-12       # both ranks' work / slowest time

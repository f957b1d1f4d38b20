"""Host-side logic of bench.py on the CPU.

The multi-GPU form of the benchmark runs independent replicas (one tensor per
rank, no collective on the data path); only its timing needs the ranks: a
step's time is the maximum over ranks and the value is every rank's bytes over
that time.  Those two pieces run here under a world-size-2 gloo group.  The
reference arm (the FP64 oracle on the host cores) needs no GPU at all: rank 0
prints the contract's JSON line, the other ranks exit 0 without output.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench._DIST["on"] = True
        ms = bench.max_over_ranks(100.0 + 25.0 * rank, torch.device("cpu"))   # rank 1 is the slow one
        bench.dist_barrier()
        q.put((rank, ms, bench.whole_job_gbps(world, 6.4e9, 5, ms)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_all_ranks_bytes():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        r, ms, v = q.get(timeout=120)
        out[r] = (ms, v)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's 125 ms; 2 ranks x 5 steps x 6.4 GB / 0.125 s
    assert out[0] == out[1]
    assert out[0][0] == 125.0
    assert out[0][1] == pytest.approx(2 * 6.4 * 5 / 0.125)


def test_single_process_value_and_time():
    import bench
    bench._DIST["on"] = False
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_gbps(1, 6.4e9, 5, 100.0) == pytest.approx(320.0)


def _bench(args, **env):
    e = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        e.pop(k, None)
    e.update(env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_other_ranks_exit_quietly():
    r = _bench(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
               RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "GB/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    import bench
    assert d["metric"] == bench.METRIC


def test_pipeline_bytes_accounting():
    """The roofline's algorithmic bytes of the sketch-and-projection phase:
    two reads of X (strict) or one per projected mode plus one (per-mode
    accounting), plus each chain intermediate written and read once and P
    written.  200^4 with K = 25 gives the 14.6 GB and 33.8 GB of the scope
    table; the small case is counted by hand (mode 1 kept whole)."""
    import bench
    assert bench.pipeline_bytes((200,) * 4, (25,) * 4, [0, 1, 2, 3]) == (14626562500, 33826562500)
    assert bench.pipeline_bytes((200,) * 4, (25,) * 4, [3, 1, 2, 0]) == (14626562500, 33826562500)
    # (10, 20, 30), K = (5, 20, 6), order 2, 0, 1: intermediates 1200 and 600
    # elements written and read, P = 600 elements written: 16800 B
    assert bench.pipeline_bytes((10, 20, 30), (5, 20, 6), [2, 0, 1]) == (2 * 6000 * 4 + 16800, 3 * 6000 * 4 + 16800)

"""Host-side logic of bench.py on the CPU.

- The reference arm: the FP64 oracle timed on the host cores, printed as one
  JSON line with impl = "reference"; ranks other than 0 exit without work.
- Replicas over several ranks: the job's step time is the maximum over the
  ranks' timed totals and the value counts every rank's units, checked with
  two gloo ranks on 127.0.0.1 (the same reduction bench.py runs over NCCL).
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, rank="0"):
    env = dict(os.environ, RANK=rank)
    return subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=900)


def test_reference_arm_line():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "projections/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "projections/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "1"], rank="1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms = bench.max_over_ranks(dist, 100.0 + 50.0 * rank, "cpu")
    q.put((rank, ms, bench.whole_job_rate(9, world, ms)))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replicas_take_the_slowest_rank_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    for rank, ms, rate in res:
        assert ms == 150.0
        assert abs(rate - 9 * 2 / 0.150) < 1e-9


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 123.5, "cpu") == 123.5
    assert abs(bench.whole_job_rate(9, 1, 900.0) - 10.0) < 1e-12

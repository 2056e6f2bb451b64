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


def test_kernel_rooflines_pick_the_bounding_unit():
    """The bench line's roofline arithmetic: kernels ordered by summed event
    time; achieved = algorithmic work / time against the peak of the unit
    that bounds each kernel (HBM for the split-BF16 product, the split
    product's FP64-equivalent tensor peak, FP64 or FP32 CUDA cores, none for
    latency-bound kernels without a work count)."""
    sys.path.insert(0, ROOT)
    import bench
    pk = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1680.0}
    named = {
        "k_trid_eig": {"ms": 5.0, "timed": 2, "flops": 0.0, "bytes": 0.0},
        "k_tc_wprod": {"ms": 2.0, "timed": 4, "flops": 0.0, "bytes": 6.0e9},           # 6 GB in 2 ms
        "oz_gemm": {"ms": 40.0, "timed": 8, "flops": 8.0e11, "bytes": 0.0},             # 0.8 TFLOP in 40 ms
        "k_latrd_coop": {"ms": 10.0, "timed": 1, "flops": 6.0e9, "bytes": 0.0},         # FP64 CUDA cores
        "k_gemm<NN,f32>": {"ms": 1.0, "timed": 1, "flops": 2.0e10, "bytes": 0.0},       # FP32 CUDA cores
        "k_idle": {"ms": 0.0, "timed": 0, "flops": 1.0, "bytes": 1.0},                  # never timed: left out
    }
    out = bench.kernel_rooflines(named, pk, total_ms=100.0)
    assert [r["kernel"] for r in out] == ["oz_gemm", "k_latrd_coop", "k_trid_eig", "k_tc_wprod", "k_gemm<NN,f32>"]
    by = {r["kernel"]: r for r in out}
    w = by["k_tc_wprod"]
    assert w["bound"] == "hbm" and w["unit"] == "GB/s" and abs(w["achieved"] - 3000.0) < 1e-9
    assert abs(w["frac"] - 0.5) < 1e-12 and abs(w["avg_launch_ms"] - 0.5) < 1e-12
    o = by["oz_gemm"]
    assert o["bound"] == "tensor" and abs(o["achieved"] - 20.0) < 1e-9       # TFLOP/s FP64-equivalent
    assert abs(o["peak"] - 80.0) < 1e-9 and abs(o["frac"] - 0.25) < 1e-12    # sustained bf16 / 21
    assert abs(o["executed_bf16_tflops"] - 420.0) < 1e-9
    lt = by["k_latrd_coop"]
    assert lt["bound"] == "alu" and abs(lt["achieved"] - 0.6) < 1e-12
    assert lt["peak"] == bench.FP64_PEAK_TFLOPS_NOMINAL and abs(lt["share_of_step"] - 0.1) < 1e-12
    g = by["k_gemm<NN,f32>"]
    assert g["peak"] == bench.FP32_PEAK_TFLOPS_DERIVED and abs(g["achieved"] - 20.0) < 1e-9
    e = by["k_trid_eig"]
    assert e["bound"] == "latency" and e["achieved"] is None and e["frac"] is None

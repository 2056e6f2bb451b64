"""Benchmark: PSD projections/s of the warm-started LOBPCG projection (the
hot path of approximate ADMM, Algorithm 3 + Eq. 2) on the projection-sweep
workload: W = Q Lambda Q^T with Haar Q, n in {256, 1024, 4096}, k/n in
{1%, 5%, 25%}, positive eigenvalues U[0.1, 1], negative U[-1, -0.1], warm
start = the k positive eigenvectors perturbed by 1e-3.

One step = one projection of every matrix of the sweep from its fixed warm
start (the same work every step).  Inputs are resident in HBM; L2 is flushed
between steps by writing a 256 MiB buffer.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|bf16x3]
  python bench.py --impl reference      # the FP64 CPU oracle (Jacobi), timed
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

from paper_1912_02767_gb300 import instances as gen  # noqa: E402

FP64_PEAK_TFLOPS_NOMINAL = 1.25  # GB300 FP64 (CUDA cores); 1.20 measured by an FMA loop on this machine


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "bf16x3"])
    ap.add_argument("--sizes", default="256,1024,4096")
    ap.add_argument("--fracs", default="0.01,0.05,0.25")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def sweep(args):
    ns = [int(x) for x in args.sizes.split(",") if x]
    fs = [float(x) for x in args.fracs.split(",") if x]
    return [(n, f) for n in ns for f in fs]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(mats, budget_s=12.0):
    """The FP64 CPU oracle (cyclic Jacobi projection) on a bounded sample:
    the sweep's n = 256 matrices, repeated until about budget_s seconds."""
    import importlib
    importlib.import_module("oracle.build").build()
    import oracle
    sample = [m for m in mats if m["n"] == 256] or sorted(mats, key=lambda m: m["n"])[:1]
    done, t0 = 0, time.perf_counter()
    while True:
        for m in sample:
            oracle.psd_project(m["W"])
            done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "projections/s", "cores": 1, "kind": "oracle",
            "sample": "%d Jacobi projections of the sweep's n=%d matrices (%d distinct), %.1f s, 1 thread"
                      % (done, sample[0]["n"], len(sample), dt)}


def make_mats(args):
    mats = []
    for n, f in sweep(args):
        sp = gen.workload_projection(n, f)
        mats.append({"n": n, "f": f, "k": sp["k"], "W": sp["W"], "X0": sp["X0"], "Q": sp["Q"], "lam": sp["lam"]})
    return mats


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    mats = make_mats(args)
    import importlib
    importlib.import_module("oracle.build").build()
    import oracle
    sample = [m for m in mats if m["n"] == 256] or mats[:1]
    for _ in range(args.warmup):
        oracle.psd_project(sample[0]["W"])
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        for m in sample:
            oracle.psd_project(m["W"])
            done += 1
    dt = time.perf_counter() - t0
    v = done / dt
    line = {"impl": "reference", "metric": "PSD projections/s (warm-started LOBPCG, k/n sweep)", "value": v,
            "unit": "projections/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "psd_projection_sweep", "sample": "n=256 matrices of the sweep",
                       "matrices_per_step": len(sample)},
            "cpu_baseline": {"value": v, "unit": "projections/s", "cores": 1, "kind": "oracle",
                             "sample": "%d Jacobi projections of the sweep's n=256 matrices per step" % len(sample)},
            "e2e": {"value": v, "unit": "projections/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1912_02767_gb300 import build_lib, sdpgpu
    build_lib.build()
    sdpgpu.load()
    prec = sdpgpu.PREC_FP64 if args.prec == "fp64" else sdpgpu.PREC_BF16X3
    stream = torch.cuda.current_stream()
    ctx = sdpgpu.Context(stream=stream, precision=prec)
    mats = make_mats(args)
    dev = []
    for m in mats:
        n = m["n"]
        Wd = torch.from_numpy(np.ascontiguousarray(m["W"])).cuda()
        X0 = torch.zeros((n, n), dtype=torch.float64, device="cuda")  # column-major n x mcap(=n) buffer
        X0[: m["k"]] = torch.from_numpy(np.ascontiguousarray(m["X0"].T)).cuda()
        V = torch.zeros_like(X0)
        out = torch.empty((n, n), dtype=torch.float64, device="cuda")
        dev.append((m, Wd, X0, V, out))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    nbytes_W = sum(m["n"] * m["n"] * 8 for m in mats)

    tol_scale = 0.5e-6 if args.prec == "fp64" else 1e-5
    tols = [tol_scale * float(np.linalg.norm(m["W"])) / np.sqrt(2.0 * m["k"]) for m in mats]
    per_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in mats]

    def step(timed=False):
        infos = []
        for q, (m, Wd, X0, V, out) in enumerate(dev):
            V.copy_(X0)
            if timed:
                per_ev[q][0].record(stream)
            info = ctx.project_raw(m["n"], Wd.data_ptr(), out.data_ptr(), V.data_ptr(), m["k"], m["n"], tols[q], True)
            if timed:
                per_ev[q][1].record(stream)
            infos.append(info)
        return infos

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    sdpgpu.prof_reset()
    # correctness of the measured path on every matrix (closed form)
    errs = []
    for (m, Wd, X0, V, out) in dev:
        P = out.cpu().numpy()
        ref = (m["Q"] * np.maximum(m["lam"], 0)) @ m["Q"].T
        errs.append(float(np.linalg.norm(P - ref) / np.linalg.norm(m["W"])))
    clocks = ClockSampler(local)
    sdpgpu.prof_reset()
    sdpgpu.prof_enable(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    per_ms = [0.0] * len(mats)
    last_infos = None
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        last_infos = step(timed=True)
        ev[s][1].record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev[s][0].elapsed_time(ev[s][1]))
        for q in range(len(mats)):
            per_ms[q] += per_ev[q][0].elapsed_time(per_ev[q][1]) / args.steps
    torch.cuda.synchronize()
    ck = clocks.stop()
    sdpgpu.prof_enable(False)
    prof = sdpgpu.prof_get()
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    per_rank = len(mats) * args.steps
    value = per_rank * world / (total_ms / 1000.0)
    launches = sum(v["launches"] for v in prof.values())
    # roofline of the dominant kernel family (largest summed event time)
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    pk = peaks()
    prod = prof["product"]
    ach = prod["flops"] / (prod["ms"] / 1000.0) / 1e12 if prod["ms"] > 0 else 0.0
    if args.prec == "fp64":
        roof = {"kernel": "k_gemm<NN,double> (W times block, FP64 CUDA cores)", "bound": "alu",
                "achieved": ach, "peak": FP64_PEAK_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS_NOMINAL, "traffic": None,
                "peak_source": "nominal FP64 of GB300 (1.25 TFLOP/s; 1.20 measured by an FMA loop)",
                "launches": prod["launches"], "avg_launch_ms": prod["ms"] / max(prod["timed"], 1)}
    else:
        gbs = prod["bytes"] / (prod["ms"] / 1000.0) / 1e9 if prod["ms"] > 0 else 0.0
        peak = pk.get("hbm_gbs", 6800.0)
        roof = {"kernel": "tcgen05 split-BF16x3 product", "bound": "hbm", "achieved": gbs, "peak": peak,
                "unit": "GB/s", "frac": gbs / peak, "traffic": None, "launches": prod["launches"],
                "avg_launch_ms": prod["ms"] / max(prod["timed"], 1)}
    roof["share_of_step"] = {k: round(v["ms"] / max(total_ms, 1e-9), 4) for k, v in prof.items() if v["ms"] > 0}
    roof["dominant_family"] = dom[0]
    # end to end through the C ABI with host buffers (H2D W + V, D2H result + V)
    e2e = None
    if not args.no_e2e and rank == 0:
        h2d = d2h = 0
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            for m, _, _, _, _ in dev:
                P, Vout, info = ctx.project_psd(m["W"], m["X0"], tol=0.0, mcap=m["n"])
                h2d += m["n"] * m["n"] * 8 + m["X0"].size * 8
                d2h += m["n"] * m["n"] * 8 + Vout.size * 8
        dt = time.perf_counter() - t0
        steps = max(1, args.steps)
        e2e = {"value": len(mats) * steps / dt, "unit": "projections/s", "h2d_bytes_per_step": h2d // steps,
               "d2h_bytes_per_step": d2h // steps}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_rate(mats)
    if rank == 0:
        line = {"metric": "PSD projections/s (warm-started LOBPCG, k/n sweep)", "value": value,
                "unit": "projections/s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
                "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "bf16x3+f32+f64",
                "data": "synthetic",
                "config": {"workload": "psd_projection_sweep",
                           "matrices": ["n=%d k/n=%g" % (m["n"], m["f"]) for m in mats],
                           "precision": args.prec, "l2": "flushed between steps (256 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": ck, "max_rel_err_vs_closed_form": max(errs),
                "per_matrix": [{"n": m["n"], "k": m["k"], "ms": round(per_ms[q], 3), "rel_err": errs[q],
                                "rr_steps": last_infos[q]["steps"], "m": last_infos[q]["m"],
                                "jacobi_sweeps": last_infos[q]["jacobi_sweeps"],
                                "converged": last_infos[q]["converged"]} for q, m in enumerate(mats)]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

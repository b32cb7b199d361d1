"""Throughput benchmark of the fused axisymmetric thermal LBM-LES step.

Default workload: the 4096 x 1024 synthetic hot jet (nozzle radius 128,
u = 0.08 (1 - (r/R)^2), T ratio 10, Smagorinsky Cs = 0.17, 256-entry
nu(T) table), FP32 population storage.  One "step" is one time step of the
whole lattice (one fused kernel launch).  The two population buffers
(436 MB in FP32) are larger than the 129 MB L2, so no flush is needed
between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BYTES_PER_VALUE = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}
POPS = 13  # 9 D2Q9 + 4 D2Q4 populations, each read once and written once per update
METRIC = "MLUPS & HBM-roofline % (D2Q9+D2Q4 LES); serving p50/p99 latency vs plain"
KERNEL_SRC = os.path.join(ROOT, "paper_1002_3028_gb300", "csrc", "lbm_kernels.cuh")


def workload_by_name(name: str):
    from paper_1002_3028_gb300 import inputs as I

    m = re.fullmatch(r"jet(\d+)x(\d+)", name)
    if m:
        return I.jet_workload(nx=int(m.group(1)), nr=int(m.group(2)))
    if name == "pipe":
        return I.pipe_workload()
    raise SystemExit(f"unknown workload {name}")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash() -> str:
    with open(KERNEL_SRC, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def ncu_traffic(storage: str, workload: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None if there is none for this storage/workload or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", f"step_kernel_{storage}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    b = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not h or not b or h.group(1) != kernel_hash():
        return None
    return float(b.group(1))


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def __enter__(self):
        def run():
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                         timeout=5).stdout.strip()
                    if out:
                        self.samples.append([v.strip() for v in out.split(",")])
                except Exception:
                    return
                self._stop.wait(0.2)

        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 3 + k and s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(w, budget_s: float):
    """The FP64 oracle on the host cores, on a bounded sample of the same lattice."""
    from oracle import oracle

    cores = os.cpu_count() or 1
    o = oracle.Oracle.from_workload(w, nthreads=cores)
    o.step(1)  # warm-up
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    o.close()
    return {"value": w.nodes * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n} time steps of the {w.cfg.nx}x{w.cfg.nr} lattice (FP64, after 1 warm-up step)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workload_by_name(args.workload)
    from oracle import oracle

    cores = os.cpu_count() or 1
    o = oracle.Oracle.from_workload(w, nthreads=cores)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    mlups = w.nodes * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"jet {w.cfg.nx}x{w.cfg.nr}", "storage": "f64 (oracle)"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full time steps of the {w.cfg.nx}x{w.cfg.nr} lattice"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)

    from paper_1002_3028_gb300 import lbm

    w = workload_by_name(args.workload)
    lat = lbm.Lattice.from_workload(w, args.storage, device=device)
    if args.band or args.warps:
        lat.set_launch(max(args.band, 0), args.warps)
    stream = torch.cuda.current_stream(device)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(device)

    # warm-up, then the device-timed region: K launches bracketed by events on the launching stream
    lat.step(args.warmup)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    if ws > 1:
        t = torch.tensor([ms], device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    nodes = w.nodes
    mlups = nodes * args.steps * ws / (ms * 1e-3) / 1e6
    per_launch_s = ms * 1e-3 / args.steps
    bpl = POPS * 2 * BYTES_PER_VALUE[args.storage]
    achieved = bpl * nodes / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()

    finite = bool(torch.isfinite(lat.fields(dtype=torch.float32)).all().item())

    # end to end through the public API: the job's initial state from pinned host memory,
    # K steps, the job's result fields back to pinned host memory, all inside the timed region
    nx, nr = w.cfg.nx, w.cfg.nr
    f_h = torch.empty((9, nr, nx), dtype=torch.float64).pin_memory()
    g_h = torch.empty((4, nr, nx), dtype=torch.float64).pin_memory()
    fd, gd = lat.get_state()
    f_h.copy_(fd)
    g_h.copy_(gd)
    del fd, gd
    out_h = torch.empty((4, nr, nx), dtype=torch.float32).pin_memory()
    f_d = torch.empty_like(f_h, device=device)
    g_d = torch.empty_like(g_h, device=device)
    out_d = torch.empty((4, nr, nx), dtype=torch.float32, device=device)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    f_d.copy_(f_h, non_blocking=True)
    g_d.copy_(g_h, non_blocking=True)
    lat.set_state(f_d, g_d, lat.step_count, stream=stream)
    lat.step(args.steps)
    lat.fields(out=out_d)
    out_h.copy_(out_d, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([e2e_ms], device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    h2d = (f_h.numel() + g_h.numel()) * 8
    d2h = out_h.numel() * 4
    e2e = {"value": nodes * args.steps * ws / (e2e_ms * 1e-3) / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "note": "initial state uploaded, K steps, fields downloaded; copies amortised over K"}

    if rank != 0:
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)
    traffic = ncu_traffic(args.storage, args.workload)
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage != "f64" else "f64",
        "data": "synthetic",
        "config": {"workload": f"jet {nx}x{nr}", "storage": args.storage, "nodes": nodes,
                   "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2": "no flush: inputs larger than L2 (two population buffers of "
                         f"{2 * POPS * BYTES_PER_VALUE[args.storage] * nodes / 1e6:.0f} MB)",
                   "bytes_per_lup": bpl,
                   "launch": dict(zip(("band_rows", "warps_per_cta", "ctas"), lat.launch()))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "fields_finite": finite,
    }
    print(json.dumps(line), flush=True)
    lat.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="jet4096x1024")
    ap.add_argument("--storage", default="f32", choices=sorted(BYTES_PER_VALUE))
    ap.add_argument("--band", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

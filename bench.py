"""Throughput benchmark of the fused axisymmetric thermal LBM-LES step.

Default workload: the 4096 x 1024 synthetic hot jet (nozzle radius 128,
u = 0.08 (1 - (r/R)^2), T ratio 10, Smagorinsky Cs = 0.17, 256-entry
nu(T) table), FP32 population storage.  One "step" is one time step of the
whole lattice; the K timed steps run in one persistent launch of the fused
kernel (tiles of step t + 1 start as soon as their neighbours finished
step t).  The two population buffers
(436 MB in FP32) are larger than the 129 MB L2, so no flush is needed
between steps.  ``--workload ensemble`` steps 256 ragged jets as one batch
(persistent multi-step launches, CUDA-graph replay); ``--workload jetNXxNR`` any size;
``--workload serving`` the continuous-batching service alone; ``--workload sweep`` the
precision sweep (every storage type against an FP64 GPU run of the same steps).

Prints one JSON line (rank 0).  The default line also carries the ensemble (FP16
moment-split and rest-deviation storage) and the 2000-request serving run against the
one-at-a-time FP32 path (``--no-extras`` leaves them out).  ``--impl reference`` times the
FP64 CPU oracle on the host cores on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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

BYTES_PER_VALUE = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "f16s": 2, "bf16s": 2}
POPS = 13  # 9 D2Q9 + 4 D2Q4 populations, each read once and written once per update
SPLIT_MOMENT_BYTES = 3 * 4  # moment-split storage: j_x, j_r, T - T0 in FP32 per node


def bytes_per_node(storage: str) -> int:
    """Bytes of one node's stored state: 13 populations, plus the FP32 moments of moment-split storage."""
    return POPS * BYTES_PER_VALUE[storage] + (SPLIT_MOMENT_BYTES if storage.endswith("s") else 0)


def bytes_per_lup(storage: str) -> int:
    """Algorithmic DRAM bytes per lattice update, either pattern: every node's stored state read
    once and written once (the AA pattern's edge moments are a few per cent more and are
    not counted)."""
    return 2 * bytes_per_node(storage)


def resident_mb(storage: str, pattern: str, nodes: int) -> float:
    """Population storage of the lattices (one buffer for the AA pattern, two otherwise), in MB."""
    return bytes_per_node(storage) * (1 if pattern == "aa" else 2) * nodes / 1e6
METRIC = "MLUPS & HBM-roofline % (D2Q9+D2Q4 LES); serving p50/p99 latency vs plain"
HOLD_CYCLES = 4_000_000  # device-side hold before a timed region: about 2 ms at 2 GHz
KERNEL_SRC = os.path.join(ROOT, "paper_1002_3028_gb300", "csrc", "lbm_kernels.cuh")
AA_SRC = os.path.join(ROOT, "paper_1002_3028_gb300", "csrc", "lbm_aa.cuh")


def workloads_by_name(name: str):
    """The lattices of a named workload: one jet, the pipe, or the ragged ensemble."""
    from paper_1002_3028_gb300 import inputs as I

    m = re.fullmatch(r"jet(\d+)x(\d+)", name)
    if m:
        return [I.jet_workload(nx=int(m.group(1)), nr=int(m.group(2)))]
    if name == "pipe":
        return [I.pipe_workload()]
    m = re.fullmatch(r"ensemble(\d*)", name)
    if m:
        return I.ensemble_workloads(int(m.group(1) or 256), seed=7)
    raise SystemExit(f"unknown workload {name}")


def workload_label(name: str, ws) -> str:
    if len(ws) == 1:
        return f"jet {ws[0].cfg.nx}x{ws[0].cfg.nr}" if name.startswith("jet") else name
    return f"ensemble of {len(ws)} ragged jets ({sum(w.nodes for w in ws)} nodes)"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash(pattern: str = "ab") -> str:
    """First 16 hex digits of the SHA-256 of the kernel source's code: every line cut at `//`,
    trailing blanks and empty lines dropped, so that comment edits keep the hash.  The AA
    pattern's kernel also covers its own source file."""
    code = []
    for path in (KERNEL_SRC, AA_SRC) if pattern == "aa" else (KERNEL_SRC,):
        with open(path) as fh:
            lines = (ln.split("//", 1)[0].rstrip() for ln in fh.read().splitlines())
        code.extend(ln for ln in lines if ln)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def ncu_traffic(storage: str, workload: str, pattern: str = "ab", kernel: str = "step"):
    """DRAM bytes per step of the step kernel (or, with kernel="batch", of the batch kernel;
    a launch holds K steps; per step, like `achieved`) from the committed ncu summary, or None
    if there is none for this storage/workload/pattern or the kernel source changed since."""
    if kernel == "batch":
        name = f"batch_kernel_{storage}_{workload}.md"
    else:
        name = f"step_kernel_{storage}_{workload}.md" if pattern == "ab" else f"aa_step_kernel_{storage}_{workload}.md"
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = re.search(r"kernel_code_sha256_16:\s*([0-9a-f]+)", text)
    b = re.search(r"dram_bytes_per_step_full_size:\s*([0-9.eE+]+)", text)
    if not h or not b or h.group(1) != kernel_hash(pattern):
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
    from paper_1002_3028_gb300 import replicas

    return replicas.world()


def cpu_baseline(ws, budget_s: float, label: str):
    """The FP64 oracle on the host cores, on a bounded sample of the same workload.

    One lattice: as many whole time steps as fit in about budget_s.  An
    ensemble: one timed step (after a warm-up step) of each lattice in turn
    until about budget_s has passed.
    """
    from oracle import oracle

    cores = os.cpu_count() or 1
    if len(ws) == 1:
        w = ws[0]
        o = oracle.Oracle.from_workload(w, nthreads=cores)
        o.step(1)
        t0 = time.perf_counter()
        steps = 0
        while True:
            o.step(1)
            steps += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        dt = time.perf_counter() - t0
        o.close()
        return {"value": w.nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                "sample": f"{steps} time steps of the {w.cfg.nx}x{w.cfg.nr} lattice (FP64, after 1 warm-up step)"}
    total_nodes, total_s, used = 0, 0.0, 0
    t_start = time.perf_counter()
    for w in ws:
        o = oracle.Oracle.from_workload(w, nthreads=cores)
        o.step(1)
        t1 = time.perf_counter()
        o.step(1)
        total_s += time.perf_counter() - t1
        total_nodes += w.nodes
        used += 1
        o.close()
        if time.perf_counter() - t_start >= budget_s:
            break
    return {"value": total_nodes / total_s / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"one timed step (after a warm-up step) of each of the first {used} lattices of {label}"}


def reference_sample(works, per_step_s: float, cores: int):
    """A bounded sample of a workload that the oracle steps in about per_step_s: the first rows
    of a single lattice (same inlet, boundaries and tables; the nozzle is at the axis), or the
    first lattices of an ensemble.  The per-node cost comes from one step of a 32-row probe."""
    import dataclasses

    from oracle import oracle

    w0 = works[0]
    rows = min(32, w0.cfg.nr)
    probe = dataclasses.replace(w0, cfg=dataclasses.replace(w0.cfg, nr=rows), u_in=w0.u_in[:rows],
                                T_in=w0.T_in[:rows])
    o = oracle.Oracle.from_workload(probe, nthreads=cores)
    o.step(1)
    t0 = time.perf_counter()
    o.step(2)
    per_node = (time.perf_counter() - t0) / (2 * probe.nodes)
    o.close()
    budget_nodes = max(1, int(per_step_s / per_node))
    if len(works) == 1:
        nr = max(1, min(w0.cfg.nr, budget_nodes // w0.cfg.nx))
        w = dataclasses.replace(w0, cfg=dataclasses.replace(w0.cfg, nr=nr), u_in=w0.u_in[:nr], T_in=w0.T_in[:nr])
        return [w], f"the first {nr} of {w0.cfg.nr} rows of the {w0.cfg.nx}x{w0.cfg.nr} lattice"
    picked, nodes = [], 0
    for w in works:
        if picked and nodes + w.nodes > budget_nodes:
            break
        picked.append(w)
        nodes += w.nodes
    return picked, f"the first {len(picked)} of {len(works)} lattices"


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (the paper ships no code to install).
    Each step is one time step of a bounded sample of the workload, sized so that the whole
    run takes about two minutes; the metric is per lattice node."""
    nranks, rank, _ = dist_env()
    if rank != 0:
        return 0
    works = workloads_by_name(args.workload)
    label = workload_label(args.workload, works)
    from oracle import oracle

    cores = os.cpu_count() or 1
    sample, desc = reference_sample(works, 120.0 / (args.steps + args.warmup), cores)
    orcs = [oracle.Oracle.from_workload(w, nthreads=cores) for w in sample]
    for _ in range(args.warmup):
        for o in orcs:
            o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for o in orcs:
            o.step(1)
    dt = time.perf_counter() - t0
    nodes = sum(w.nodes for w in sample)
    mlups = nodes * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": nranks,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": label, "storage": "f64 (oracle)"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{desc}, one time step each of {args.steps} timed steps"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    for o in orcs:
        o.close()
    print(json.dumps(line), flush=True)
    return 0


def error_vs_f64(works, storage: str, device, steps: int = 1000, sample: int = 4, pattern: str = "ab"):
    """Field errors of the measured storage type against the FP64 GPU path (which the parity
    tests hold to the oracle within 1e-12 per step): up to `sample` lattices of the workload
    run `steps` steps from the same start in both, and the largest relative errors of rho,
    u (against the maximum speed) and T are reported."""
    if storage == "f64":
        return {"vs": "FP64 oracle (parity tests)", "bound_per_step": 1e-12}
    from paper_1002_3028_gb300 import lbm

    picks = list(range(0, len(works), max(1, len(works) // sample)))[:sample]
    worst = {"rho": 0.0, "u": 0.0, "T": 0.0}
    for k in picks:
        a = lbm.Lattice.from_workload(works[k], storage, device=device, pattern=pattern)
        b = lbm.Lattice.from_workload(works[k], "f64", device=device)
        a.step(steps)
        b.step(steps)
        Fa, Fb = a.fields(), b.fields()
        speed = float(Fb[1:3].abs().max())
        worst["rho"] = max(worst["rho"], float((Fa[0] - Fb[0]).abs().max() / Fb[0].abs().max()))
        worst["u"] = max(worst["u"], float((Fa[1:3] - Fb[1:3]).abs().max()) / max(speed, 1e-30))
        worst["T"] = max(worst["T"], float((Fa[3] - Fb[3]).abs().max() / Fb[3].abs().max()))
        a.close()
        b.close()
    return {"vs": "FP64 GPU path (held to the oracle within 1e-12 per step by the parity tests)",
            "steps": steps, "lattices": len(picks), **worst}


def step_launches(lats, storage: str, launch, steps: int, strip: int = 0) -> int:
    """Kernels launched by `steps` steps.  One lattice runs its steps in persistent launches
    of up to 2^31 / (2 x warp tiles) steps each (either pattern).  A batch replays a
    captured launch of 64 steps and runs the rest in one launch; each launch is followed
    by the parameter advance."""
    strip = strip or (32 if storage == "f64" else 64)
    band = launch[0]
    ntiles = sum(-(-lat.nx // strip) * -(-lat.nr // band) for lat in lats)
    per_launch = max(1, (1 << 31) // (2 * ntiles))
    if len(lats) == 1:
        return -(-steps // per_launch)
    graph = min(64, per_launch)
    return 2 * (steps // graph + (1 if steps % graph else 0))


def run_gpu(args):
    import torch

    from paper_1002_3028_gb300 import autotune, lbm, replicas

    ws, rank, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    replicas.init("nccl", device)  # replicas only: no collective on the data path

    works = workloads_by_name(args.workload)
    label = workload_label(args.workload, works)
    lats = [lbm.Lattice.from_workload(w, args.storage, device=device, pattern=args.pattern) for w in works]
    nodes = sum(w.nodes for w in works)
    stream = torch.cuda.current_stream(device)
    if len(lats) == 1:
        target = lats[0]
        step = target.step
    else:  # an ensemble: one batch, persistent multi-step launches, graph replay
        target = lbm.Batch(args.storage)
        for lat in lats:
            target.add(lat)

        def step(n, stream=None):
            target.step(n, graph=True, stream=stream)
    if args.autotune:  # outside the timed region; the lattices advance while tuning
        autotune.tune(target)
    else:
        if args.strip:
            target.set_strip_width(args.strip)
        if args.band or args.warps:
            target.set_launch(max(args.band, 0), args.warps)
    if args.group > 0 and len(lats) == 1:
        target.set_item_group(args.group)

    def barrier():
        replicas.barrier()
        torch.cuda.synchronize(device)

    # The error check against the FP64 path runs before the timed region: it is untimed work
    # that also brings the GPU to its working clocks before the region starts.
    errors = error_vs_f64(works, args.storage, device, pattern=args.pattern)

    # The clock sampler runs from before the warm-up to after the timed region, so that its
    # first nvidia-smi process is not started inside the timed region.  Warm-up, then the
    # device-timed region: K steps bracketed by events on the launching stream.  Before the
    # start event the stream is held on the device for about 2 ms (a sleep kernel, outside the
    # region), so the start event and the steps are already enqueued when the GPU reaches
    # them: the region holds the device work of the K steps, not the host's launch latency.
    clk = ClockSampler(local).__enter__()
    step(args.warmup)
    barrier()
    time.sleep(0.3)  # the sampler's first reading lands before the region
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda._sleep(HOLD_CYCLES)
    ev0.record(stream)
    step(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    clk.__exit__(None, None, None)
    barrier()
    ms, units = replicas.combine(ev0.elapsed_time(ev1), nodes * args.steps, device)
    mlups = units / (ms * 1e-3) / 1e6
    per_step_s = ms * 1e-3 / args.steps
    bpl = bytes_per_lup(args.storage)
    achieved = bpl * nodes / per_step_s / 1e9  # algorithmic bytes of the launch(es) / their duration
    peak, peak_kind = measured_peaks()
    finite = all(bool(torch.isfinite(lat.fields(dtype=torch.float32)).all().item()) for lat in lats)
    flags = max(lat.check() for lat in lats)

    # end to end through the public API: every lattice's initial state (its checkpoint in the
    # storage type, lbm_save's layout) from pinned host memory through lbm_restore, K steps,
    # every lattice's fields back to pinned host memory, all timed
    host_states, dev_states, outs = [], [], []
    for lat in lats:
        planes, _ = lat.save()
        ph = torch.empty(planes.shape, dtype=planes.dtype).pin_memory()
        ph.copy_(planes)
        host_states.append(ph)
        dev_states.append(torch.empty_like(planes))
        outs.append((torch.empty((4, lat.nr, lat.nx), dtype=torch.float32, device=device),
                     torch.empty((4, lat.nr, lat.nx), dtype=torch.float32).pin_memory()))
        del planes
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for lat, ph, pd in zip(lats, host_states, dev_states):
        pd.copy_(ph, non_blocking=True)
        lat.restore_async(pd, lat.step_count, stream=stream)
    step(args.steps, stream=stream)
    for lat, (od, oh) in zip(lats, outs):
        lat.fields(out=od, stream=stream)
        oh.copy_(od, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    barrier()
    e2e_ms, e2e_units = replicas.combine(e0.elapsed_time(e1), nodes * args.steps, device)
    h2d = sum(ph.numel() * ph.element_size() for ph in host_states)
    d2h = sum(oh.numel() * 4 for _, oh in outs)
    e2e = {"value": e2e_units / (e2e_ms * 1e-3) / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "note": "initial states (storage-type checkpoints) uploaded and restored, K steps, fields "
                   "downloaded; copies amortised over K"}

    if rank != 0:
        replicas.finish()
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(works, args.cpu_seconds, label)
    traffic = ncu_traffic(args.storage, args.workload, args.pattern)
    launch = target.launch()
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage != "f64" else "f64",
        "data": "synthetic",
        "config": {"workload": label, "storage": args.storage, "pattern": args.pattern, "nodes": nodes,
                   "lattices": len(lats), "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2": "no flush: inputs larger than L2 ("
                         + ("one population buffer" if args.pattern == "aa"
                            else "two population buffers")
                         + f" of {resident_mb(args.storage, args.pattern, nodes):.0f} MB)",
                   "bytes_per_lup": bpl,
                   "launch": {**dict(zip(("band_rows", "warps_per_cta", "ctas" if len(lats) == 1 else "tiles"),
                                         launch)), "strip_columns": target.strip_width}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "per": "step (the timed steps run in persistent launches of many steps)"},
        "cpu_baseline": cpu,
        "error": errors,
        "e2e": e2e,
        "gpu_launches": step_launches(lats, args.storage, launch, args.steps, target.strip_width),
        "clocks": clk.summary(),
        "fields_finite": finite,
        "device_flags": flags,
    }
    if ws == 1 and not args.no_extras and len(lats) == 1:
        # the metric's other halves: the batched ensemble and the serving loop (after the headline
        # measurement, so they do not touch it)
        for lat in lats:
            lat.close()
        torch.cuda.empty_cache()
        line["ensemble"] = {st: ensemble_object(device, st) for st in ("f16s", "f16")}
        line["serving"] = serving_object(device, args.requests, args.rate, args.budget_gb, args.chunk,
                                         storage=args.serve_storage)
    print(json.dumps(line), flush=True)
    replicas.finish()
    return 0


def field_errors(Fa, Fb) -> dict:
    """Largest relative differences of fields Fa from Fb ((4, nr, nx): rho, u_x, u_r, T): rho and T
    against their own maxima, u against the maximum speed."""
    speed = float(Fb[1:3].abs().max())
    return {"rho": float((Fa[0] - Fb[0]).abs().max() / Fb[0].abs().max()),
            "u": float((Fa[1:3] - Fb[1:3]).abs().max()) / max(speed, 1e-30),
            "T": float((Fa[3] - Fb[3]).abs().max() / Fb[3].abs().max())}


def storage_errors(w, storage: str, steps: int, device) -> dict:
    """Errors of a storage type against the FP64 path on one workload (untimed):

    - ``per_step``: after `steps` steps in `storage`, its state is copied exactly (as FP64) into
      an FP64 lattice and both take one more step; the fields are compared.  This is the bound
      that holds at any time, turbulent or not;
    - ``after_steps``: `storage`, FP32 and FP64 run `steps` steps from rest; the `storage` and
      FP32 fields are compared with the FP64 ones.  On a turbulent jet the trajectories diverge
      whatever the precision, which the FP32 column shows.
    """
    from paper_1002_3028_gb300 import lbm

    a = lbm.Lattice.from_workload(w, storage, device=device)
    b = lbm.Lattice.from_workload(w, "f64", device=device)
    a.step(steps)
    b.step(steps)
    out = {"steps": steps, "after_steps": {storage: field_errors(a.fields(), b.fields())}}
    if storage != "f32":
        c = lbm.Lattice.from_workload(w, "f32", device=device)
        c.step(steps)
        out["after_steps"]["f32"] = field_errors(c.fields(), b.fields())
        c.close()
    f, g = a.get_state()
    b.set_state(f, g, a.step_count)
    a.step(1)
    b.step(1)
    out["per_step"] = field_errors(a.fields(), b.fields())
    a.close()
    b.close()
    return out


def worst(errs, key) -> dict:
    """Component-wise maximum of the `key` error dicts of a list of storage_errors results."""
    out = {}
    for e in errs:
        d = e
        for k in key.split("."):
            d = d[k]
        for c, v in d.items():
            out[c] = max(out.get(c, 0.0), v)
    return out


def ensemble_object(device, storage: str = "f16s", steps: int = 5000, warm: int = 64, count: int = 256) -> dict:
    """The ragged ensemble (256 jets, 2-byte storage, one batch, persistent launches from a captured
    CUDA graph), timed over `steps` steps of every member, with its roofline and errors."""
    import torch

    from paper_1002_3028_gb300 import inputs as I
    from paper_1002_3028_gb300 import lbm

    works = I.ensemble_workloads(count, seed=7)
    nodes = sum(w.nodes for w in works)
    lats = [lbm.Lattice.from_workload(w, storage, device=device) for w in works]
    batch = lbm.Batch(storage)
    for lat in lats:
        batch.add(lat)
    stream = torch.cuda.current_stream(device)
    batch.step(warm, graph=True, stream=stream)
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda._sleep(HOLD_CYCLES)
    e0.record(stream)
    batch.step(steps, graph=True, stream=stream)
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    launch = batch.launch()
    flags = max(lat.check() for lat in lats)
    batch.close()
    for lat in lats:
        lat.close()
    del lats
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_lup(storage) * nodes * steps / sec / 1e9
    picks = [works[k] for k in range(0, count, count // 4)][:4]
    errs = [storage_errors(w, storage, 1000, device) for w in picks]
    return {"workload": f"{count} ragged jets, seed 7 ({nodes} nodes)", "storage": storage, "steps": steps,
            "glups": nodes * steps / sec / 1e9, "ms_per_step": sec * 1e3 / steps,
            "launch": dict(zip(("band_rows", "warps_per_cta", "tiles"), launch)),
            "graph": "one captured launch of 64 steps, replayed",
            "roofline": {"bound": "hbm", "bytes_per_lup": bytes_per_lup(storage), "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": ncu_traffic(storage, f"ensemble{count}", kernel="batch") if count == 256 else None},
            "error_vs_f64": {"lattices": len(picks), "per_step": worst(errs, "per_step"),
                             "after_1000_steps": {k: worst(errs, "after_steps." + k)
                                                  for k in errs[0]["after_steps"]}},
            "device_flags": flags}


def plain_service_times(reqs, storage: str, device, n1: int = 100, n2: int = 500):
    """Service time of every request on the plain path (one lattice alone, created, stepped in
    one persistent launch, fields read back), measured request by request: creation and read-back
    with the host clock, and the launch time for the request's step count from two timed launches
    of n1 and n2 steps (a persistent launch costs a + b n; both launches are measured)."""
    import torch

    from paper_1002_3028_gb300 import lbm

    out = []
    for req in reqs:
        w = req.workload
        t0 = time.perf_counter()
        lat = lbm.Lattice.from_workload(w, storage, device=device)
        torch.cuda.synchronize(device)
        t_create = time.perf_counter() - t0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        lat.step(n1)
        ev[1].record()
        lat.step(n2)
        ev[2].record()
        ev[2].synchronize()
        ta, tb = ev[0].elapsed_time(ev[1]) * 1e-3, ev[1].elapsed_time(ev[2]) * 1e-3
        slope = (tb - ta) / (n2 - n1)
        icpt = ta - slope * n1
        t0 = time.perf_counter()
        lat.fields(dtype=torch.float32).cpu()
        t_fields = time.perf_counter() - t0
        lat.close()
        out.append(t_create + icpt + slope * w.steps + t_fields)
    return out


def fifo_replay(reqs, service):
    """One server, first come first served: finish_i = max(arrival_i, finish_(i-1)) + service_i."""
    from paper_1002_3028_gb300.serve import Result, ServeStats

    t = 0.0
    results = []
    for req, s in zip(sorted(reqs, key=lambda r: r.arrival_s), service):
        start = max(req.arrival_s, t)
        t = start + s
        results.append(Result(req.rid, req.arrival_s, start, t, req.workload.steps, req.workload.nodes))
    return ServeStats(results, t, float(sum(r.workload.nodes * r.workload.steps for r in reqs)))


def serving_object(device, count: int = 2000, rate: float = 40.0, budget_gb: float = 120.0, chunk: int = 256,
                   pattern: str = "ab", validate: int = 30, storage: str = "f16s") -> dict:
    """The serving workload: `count` Poisson requests at `rate`/s, jets drawn like the ensemble with
    1000-20000 steps, admitted by an HBM budget into one batch of 2-byte storage (FP16 moment-split
    by default: within 1e-3 of FP64 over whole requests; continuous batching), against the plain
    FP32 path that runs one request at a time."""
    import torch

    from paper_1002_3028_gb300 import inputs as I
    from paper_1002_3028_gb300.serve import GpuBatchEngine, serve, serve_plain

    reqs = I.request_stream(count=count, rate_per_s=rate, seed=11)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    batched = serve(reqs, GpuBatchEngine(storage, device=device, pattern=pattern), budget_gb * 1e9, chunk=chunk)
    torch.cuda.synchronize(device)
    batched_wall = time.perf_counter() - t0
    # the plain path: every request's service time measured alone, then queued first come first
    # served; the first `validate` requests are also served for real to check the replay
    service = plain_service_times(reqs, "f32", device)
    plain = fifo_replay(reqs, service)
    sub = sorted(reqs, key=lambda r: r.arrival_s)[:validate]
    real = serve_plain(sub, "f32", device=device)
    model = fifo_replay(sub, service[:validate])
    picks = [reqs[r.rid].workload for r in batched.results[:: max(1, len(reqs) // 4)][:4]]
    errs = [storage_errors(w, storage, w.steps, device) for w in picks]
    b, p_ = batched.summary(), plain.summary()
    return {"workload": f"{count} Poisson requests at {rate}/s, jets drawn like the ensemble, "
                        f"steps U{{1000..20000}}, seed 11", "budget_gb": budget_gb, "chunk_steps": chunk,
            "batched": {**b, "storage": storage, "wall_s": batched_wall, "pattern": pattern},
            "plain_f32_one_at_a_time": {**p_, "how": "each request's service time measured alone (creation, "
                                        "launches of 100 and 500 steps, fields read back), queued first come "
                                        "first served",
                                        "replay_check": {"requests": validate, "real_makespan_s": real.makespan_s,
                                                         "replayed_makespan_s": model.makespan_s}},
            "mlups_ratio_batched_over_plain": b["mlups"] / p_["mlups"],
            "error_vs_f64_sample": {"requests": [w.name for w in picks], "storage": storage,
                                        "per_step": worst(errs, "per_step"),
                                        "after_request_steps": {k: worst(errs, "after_steps." + k)
                                                                for k in errs[0]["after_steps"]}}}


def l2_errors(Fa, Fb) -> dict:
    """Relative L2 differences of fields Fa from Fb: ||a - b|| / ||b|| over the lattice, for rho, for
    the velocity vector (u_x, u_r) and for T."""
    def rel(a, b):
        return float(((a - b) ** 2).sum().sqrt() / (b ** 2).sum().sqrt())

    return {"rho": rel(Fa[0], Fb[0]), "u": rel(Fa[1:3], Fb[1:3]), "T": rel(Fa[3], Fb[3])}


def run_sweep(args):
    """The precision sweep: the 4096 x 1024 jet stored in FP32, FP16 and BF16 against an FP64 GPU
    run of the same steps (relative L2 and max errors of rho, u, T), with the MLUPS of each storage
    type (K timed steps in one persistent launch after W warm-up steps)."""
    import torch

    from paper_1002_3028_gb300 import lbm

    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    device = torch.device("cuda", 0)
    w = workloads_by_name(args.workload if args.workload != "sweep" else "jet4096x1024")[0]
    ref = lbm.Lattice.from_workload(w, "f64", device=device)
    ref.step(args.sweep_steps)
    Fr = ref.fields()
    ref.close()
    rows = {}
    for storage in ("f32", "f16s", "bf16s", "f16", "bf16"):
        a = lbm.Lattice.from_workload(w, storage, device=device)
        a.step(args.sweep_steps)
        Fa = a.fields()
        rows[storage] = {"l2": l2_errors(Fa, Fr), "max": field_errors(Fa, Fr)}
        del Fa
        a.step(args.warmup)
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(HOLD_CYCLES)
        e0.record()
        a.step(args.steps)
        e1.record()
        e1.synchronize()
        rows[storage]["mlups"] = w.nodes * args.steps / (e0.elapsed_time(e1) * 1e-3) / 1e6
        rows[storage]["bytes_per_lup"] = bytes_per_lup(storage)
        a.close()
    line = {"metric": METRIC, "value": rows["f16s"]["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"precision sweep: jet {w.cfg.nx}x{w.cfg.nr}, {args.sweep_steps} steps from "
                                   "rest against the FP64 GPU path",
                       "storage": "f32; f16s, bf16s (moment-split); f16, bf16 (rest deviations)"},
            "sweep": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """The serving workload alone (one JSON line)."""
    import torch

    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    device = torch.device("cuda", 0)
    with ClockSampler(0) as clk:
        srv = serving_object(device, args.requests, args.rate, args.budget_gb, args.chunk, args.pattern,
                             storage=args.serve_storage)
    b = srv["batched"]
    line = {
        "metric": METRIC, "value": b["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": None, "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": "serving: " + srv["workload"],
                                        "storage": srv["batched"]["storage"] + " (batched), f32 (plain)"},
        "serving": srv, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="jet4096x1024")
    ap.add_argument("--storage", default="f32", choices=sorted(BYTES_PER_VALUE))
    ap.add_argument("--pattern", default="ab", choices=["ab", "aa"],
                    help="memory layout: two population buffers, or one updated in place (AA)")
    ap.add_argument("--band", type=int, default=0)
    ap.add_argument("--strip", type=int, default=0, help="tile width in columns: 32 or 64 (0 = default)")
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--group", type=int, default=0,
                    help="one lattice: warp tiles per work item of the persistent launch (0 = automatic)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="tune the launch shape before timing")
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of requests")
    ap.add_argument("--sweep-steps", type=int, default=1000,
                    help="precision sweep (--workload sweep): steps from rest compared with FP64")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ensemble and serving objects of the default line")
    ap.add_argument("--rate", type=float, default=40.0, help="serving: arrivals per second")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serving: device memory budget")
    ap.add_argument("--chunk", type=int, default=256, help="serving: most steps per batch launch sequence")
    ap.add_argument("--serve-storage", default="f16s", choices=["f16s", "bf16s", "f16", "bf16", "f32"],
                    help="serving: storage type of the batched lattices")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "sweep":
        return run_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

"""Continuous-batching service for independent jet simulations.

Requests (a lattice, its inlet and tables, a step count) arrive over time.
The scheduler admits them first-in first-out as long as their device memory
fits the HBM budget, keeps every admitted lattice resident on the GPU, and
advances all active lattices together as one batch (one persistent launch
for many steps of all of them), in chunks that end where the next active request completes.
A finished request leaves the batch at once; its fields are copied to pinned
host memory asynchronously and its memory is released when that copy has
landed, so requests that arrive while others run are admitted as soon as
memory frees up and their work overlaps on the device.

The scheduling logic (``serve``) only talks to an engine and a clock, so it
runs against the GPU engine here and against a fake engine in the CPU tests.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass
from typing import Callable, Dict, List

import numpy as np

from .inputs import Request


@dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    steps: int
    nodes: int
    fields: object = None  # host (4, nr, nx) float32 tensor when kept

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


@dataclass
class ServeStats:
    results: List[Result]
    makespan_s: float
    lups: float

    @property
    def mlups(self) -> float:
        return self.lups / self.makespan_s / 1e6

    def percentile(self, q: float) -> float:
        return float(np.percentile([r.latency_s for r in self.results], q))

    def summary(self) -> dict:
        return {"requests": len(self.results), "p50_s": self.percentile(50), "p95_s": self.percentile(95),
                "p99_s": self.percentile(99), "mlups": self.mlups, "makespan_s": self.makespan_s}


class Engine:
    """What the scheduler needs from a device back end."""

    def bytes_needed(self, req: Request) -> int:
        raise NotImplementedError

    def admit(self, req: Request):
        """Create the request's lattice (resident) and add it to the batch; return a handle."""
        raise NotImplementedError

    def step(self, n: int) -> None:
        """Advance every admitted, unfinished lattice by n steps (asynchronous)."""
        raise NotImplementedError

    def retire(self, handle):
        """Take a finished lattice out of the batch and start copying its fields out; return a token."""
        raise NotImplementedError

    def done(self, token) -> bool:
        """True once the retired lattice's fields have landed (then its memory is released)."""
        raise NotImplementedError

    def fields(self, token):
        return None

    def fence(self):
        """A marker of the work enqueued so far (None when steps run synchronously)."""
        return None

    def wait(self, fence) -> None:
        """Block until the work before `fence` has run."""


def serve(requests: List[Request], engine: Engine, budget_bytes: float, chunk: int = 256,
          clock: Callable[[], float] = time.perf_counter, sleep: Callable[[float], None] = time.sleep,
          keep_fields: bool = False, ahead: int = 2) -> ServeStats:
    """Run a request stream to completion; arrival times are relative to the start.

    The host runs at most `ahead` chunks ahead of the device: before enqueuing
    another chunk it waits for the chunk `ahead` back, so arrivals are admitted
    at device time, not behind a long queue of enqueued steps.
    """
    t0 = clock()
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
    waiting: collections.deque = collections.deque()
    active: Dict[int, list] = {}  # rid -> [handle, remaining, request, admitted_s, bytes]
    retiring: Dict[int, list] = {}  # rid -> [token, request, admitted_s, bytes]
    results: List[Result] = []
    fences: collections.deque = collections.deque()
    used = 0.0
    lups = 0.0
    for r in requests:
        if engine.bytes_needed(r) > budget_bytes:
            raise ValueError(f"request {r.rid} alone exceeds the memory budget")

    while pending or waiting or active or retiring:
        now = clock() - t0
        while pending and pending[0].arrival_s <= now:
            waiting.append(pending.popleft())
        # finished copies free their memory
        for rid in [rid for rid, (tok, _, _, _) in retiring.items() if engine.done(tok)]:
            tok, req, adm, nbytes = retiring.pop(rid)
            used -= nbytes
            results.append(Result(req.rid, req.arrival_s, adm, clock() - t0, req.workload.steps,
                                  req.workload.nodes, engine.fields(tok) if keep_fields else None))
        # first-in first-out admission within the budget
        while waiting and used + engine.bytes_needed(waiting[0]) <= budget_bytes:
            req = waiting.popleft()
            nbytes = engine.bytes_needed(req)
            active[req.rid] = [engine.admit(req), req.workload.steps, req, clock() - t0, nbytes]
            used += nbytes
        if active:
            n = min(chunk, min(a[1] for a in active.values()))
            engine.step(n)
            fences.append(engine.fence())
            while len(fences) > ahead:
                engine.wait(fences.popleft())
            lups += n * sum(a[2].workload.nodes for a in active.values())
            for rid in list(active):
                a = active[rid]
                a[1] -= n
                if a[1] == 0:
                    handle, _, req, adm, nbytes = active.pop(rid)
                    retiring[rid] = [engine.retire(handle), req, adm, nbytes]
        elif retiring:
            sleep(0.0002)
        elif pending and not waiting:
            sleep(max(0.0, min(0.001, pending[0].arrival_s - (clock() - t0))))
    results.sort(key=lambda r: r.rid)
    return ServeStats(results, clock() - t0, lups)


class GpuBatchEngine(Engine):
    """All active lattices in one liblbm batch (persistent multi-step launches, graph replay).

    The default storage is FP16 moment-split ("f16s"), the 2-byte type that stays within
    1e-3 of FP64 on u and T over whole runs.  ``pattern="aa"`` keeps every lattice in one
    population buffer updated in place, so the same memory budget admits more lattices
    (rest-deviation FP16: about 32 instead of 52 bytes per node; moment-split storage has no
    AA form).
    """

    def __init__(self, storage: str = "f16s", device=None, graph: bool = True, pattern: str = "ab"):
        import torch

        from . import lbm

        self.lbm = lbm
        self.storage = storage
        self.pattern = pattern
        self.device = torch.device(device if device is not None else "cuda")
        self.batch = lbm.Batch(storage)
        self.graph = graph
        self.stream = torch.cuda.current_stream(self.device)

    def bytes_needed(self, req: Request) -> int:
        w = req.workload
        return self.lbm.required_bytes(w.cfg, self.storage, self.pattern) + 4 * 4 * w.nodes

    def admit(self, req: Request):
        lat = self.lbm.Lattice.from_workload(req.workload, self.storage, device=self.device, pattern=self.pattern)
        self.batch.add(lat)
        return lat

    def step(self, n: int) -> None:
        self.batch.step(n, graph=self.graph, stream=self.stream)

    def retire(self, lat):
        import torch

        self.batch.remove(lat)
        out_d = lat.fields(dtype=torch.float32, stream=self.stream)
        out_h = torch.empty(out_d.shape, dtype=torch.float32).pin_memory()
        out_h.copy_(out_d, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        return [ev, lat, out_d, out_h]

    def done(self, token) -> bool:
        if token[0].query():
            if token[1] is not None:
                token[1].close()  # the lattice's memory goes back to the caching allocator
                token[1] = None
                token[2] = None
            return True
        return False

    def fields(self, token):
        return token[3]

    def fence(self):
        import torch

        ev = torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def wait(self, fence) -> None:
        fence.synchronize()


def serve_plain(requests: List[Request], storage: str = "f32", device=None,
                clock: Callable[[], float] = time.perf_counter, sleep: Callable[[float], None] = time.sleep,
                keep_fields: bool = False) -> ServeStats:
    """The plain baseline: one request at a time, in arrival order, each lattice alone."""
    import torch

    from . import lbm

    dev = torch.device(device if device is not None else "cuda")
    t0 = clock()
    results: List[Result] = []
    lups = 0.0
    for req in sorted(requests, key=lambda r: r.arrival_s):
        while clock() - t0 < req.arrival_s:
            sleep(max(0.0, min(0.001, req.arrival_s - (clock() - t0))))
        adm = clock() - t0
        lat = lbm.Lattice.from_workload(req.workload, storage, device=dev)
        lat.step(req.workload.steps)
        out = lat.fields(dtype=torch.float32).cpu()
        lat.close()
        lups += req.workload.nodes * req.workload.steps
        results.append(Result(req.rid, req.arrival_s, adm, clock() - t0, req.workload.steps, req.workload.nodes,
                              out if keep_fields else None))
    return ServeStats(results, clock() - t0, lups)

"""Autotuner of the step kernel's launch shape (band height x warps per CTA).

Times each candidate shape on the live lattice or batch with CUDA events on
its stream (after a warm-up), keeps the fastest, and remembers it in a small
JSON cache keyed by the GPU name, the storage type and the lattice shape(s),
so a later lattice of the same kind starts from the tuned shape.  Tuning
steps the lattice: tune before setting the initial state, or save and
restore it (``Lattice.get_state`` / ``set_state``).
"""
from __future__ import annotations

import hashlib
import json
import os
import threading
from typing import Iterable, List, Optional, Sequence, Tuple

from . import build as _build

CACHE = os.path.join(_build.BUILD, "autotune.json")
# (band rows, warps per CTA).  One lattice: short bands keep many tiles between dependent
# steps of the persistent launch; one-warp CTAs measured fastest.  A batch spreads each
# step over many lattices and profits from longer bands.
LATTICE_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (1, 1), (2, 1), (3, 1), (4, 1), (5, 1), (6, 1), (7, 1), (8, 1), (6, 2),
)
BATCH_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (4, 1), (6, 1), (8, 1), (12, 1), (16, 1), (16, 2),
)
_lock = threading.Lock()


def _gpu_name() -> str:
    import torch

    return torch.cuda.get_device_name(torch.cuda.current_device())


def _load() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(key: str, value) -> None:
    with _lock:
        data = _load()
        data[key] = value
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)


def lattice_key(storage: str, shapes: Iterable[Tuple[int, int]]) -> str:
    shapes = sorted(shapes)
    digest = hashlib.sha1(repr(shapes).encode()).hexdigest()[:12]
    return f"{_gpu_name()}|{storage}|{len(shapes)}|{digest}"


def _time(step_fn, steps: int, warmup: int) -> float:
    import torch

    step_fn(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    step_fn(steps)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def tune(target, candidates: Optional[Sequence[Tuple[int, int]]] = None, steps: int = 400, warmup: int = 20,
         use_cache: bool = True) -> Tuple[int, int]:
    """Pick and set the fastest (band rows, warps per CTA) for a Lattice or Batch.

    Returns the chosen shape.  With use_cache, a shape tuned earlier for the
    same GPU, storage and lattice shapes is applied without timing.  Each
    candidate runs `steps` steps in one persistent launch (enough that the
    launch's ramp and tail do not decide the ranking), twice.
    """
    from .lbm import Batch

    is_batch = isinstance(target, Batch)
    shapes = [(m.nx, m.nr) for m in target.members] if is_batch else [(target.nx, target.nr)]
    key = lattice_key(target.storage, shapes)
    if use_cache:
        hit = _load().get(key)
        if hit:
            target.set_launch(int(hit["band"]), int(hit["warps"]))
            return int(hit["band"]), int(hit["warps"])
    if is_batch:
        def run(n):
            target.step(n, graph=False)
    else:
        run = target.step
    cands = list(candidates or (BATCH_CANDIDATES if is_batch else LATTICE_CANDIDATES))
    # bring the GPU to its working clocks first, then time every candidate twice, in
    # opposite orders, and keep each one's best: a fixed order would favour whichever
    # candidate runs last on a warming GPU
    run(max(warmup, steps))
    best = {}
    for order in (cands, cands[::-1]):
        for band, warps in order:
            target.set_launch(band, warps)
            ms = _time(run, steps, warmup)
            best[(band, warps)] = min(ms, best.get((band, warps), ms))
    results: List[Tuple[float, int, int]] = sorted((ms, b, w) for (b, w), ms in best.items())
    ms, band, warps = results[0]
    target.set_launch(band, warps)
    _store(key, {"band": band, "warps": warps, "ms_per_step": ms,
                 "timings": [[b, w, t] for t, b, w in results]})
    return band, warps

"""Autotuner of the step kernel's launch and tile shape (strip width x band height x warps per CTA).

Times each candidate shape on the live lattice or batch with CUDA events on
its stream (after a warm-up), three runs each, keeps the one whose slowest
run is fastest, and remembers it in a small
JSON cache keyed by the GPU name, the storage type and the lattice shape(s),
so a later lattice of the same kind starts from the tuned shape.  The key
also holds the memory pattern: the in-place (AA) kernel takes other strip
widths and bands than the two-buffer one.  The tile
is the warp's strip of 32 or 64 columns (one or two nodes per lane) by the
band height; results are bit for bit the same for every shape.  Tuning steps
the lattice: tune before setting the initial state, or save and restore it
(``Lattice.save`` / ``restore``).
"""
from __future__ import annotations

import hashlib
import json
import os
import threading
from typing import Iterable, List, Optional, Sequence, Tuple

from . import build as _build

CACHE = os.path.join(_build.BUILD, "autotune.json")
# (strip columns, band rows, warps per CTA).  One lattice: short bands keep many tiles between
# dependent steps of the persistent launch; one-warp CTAs measured fastest; 32-column strips
# double the tiles of small lattices.  A batch spreads each step over many lattices and
# profits from longer bands.
LATTICE_CANDIDATES: Tuple[Tuple[int, int, int], ...] = (
    (64, 1, 1), (64, 2, 1), (64, 3, 1), (64, 4, 1), (64, 5, 1), (64, 6, 1), (64, 7, 1), (64, 8, 1), (64, 9, 1),
    (64, 10, 1), (64, 6, 2), (32, 1, 1), (32, 2, 1), (32, 4, 1), (32, 6, 1), (32, 8, 1),
)
BATCH_CANDIDATES: Tuple[Tuple[int, int, int], ...] = (
    (64, 4, 1), (64, 8, 1), (64, 12, 1), (64, 16, 1), (64, 16, 2), (64, 32, 1),
    (32, 8, 1), (32, 16, 1), (32, 32, 1), (32, 64, 1),
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


def lattice_key(storage: str, shapes: Iterable[Tuple[int, int]], pattern: str = "ab") -> str:
    shapes = sorted(shapes)
    digest = hashlib.sha1(repr(shapes).encode()).hexdigest()[:12]
    return f"{_gpu_name()}|{storage}|{pattern}|{len(shapes)}|{digest}"


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


def _widths(storage: str, pattern: str) -> Tuple[int, ...]:
    """Strip widths a lattice of this storage type and pattern accepts."""
    if pattern == "aa":
        return (32,) if storage == "f64" else (64,)
    return (32,) if storage == "f64" else (64, 32)


def _apply(target, cols: int, band: int, warps: int) -> None:
    target.set_strip_width(cols)
    target.set_launch(band, warps)


def tune(target, candidates: Optional[Sequence[Tuple[int, int, int]]] = None, steps: int = 400,
         warmup: int = 20, use_cache: bool = True) -> Tuple[int, int, int]:
    """Pick and set the fastest (strip columns, band rows, warps per CTA) for a Lattice or Batch.

    Returns the chosen shape.  With use_cache, a shape tuned earlier for the
    same GPU, storage type, memory pattern and lattice shapes is applied
    without timing.  Each
    candidate runs `steps` steps in one persistent launch (enough that the
    launch's ramp and tail do not decide the ranking), three times, and is
    ranked by its slowest run.  Candidates with a strip width the lattice
    does not accept are skipped.
    """
    from .lbm import Batch

    is_batch = isinstance(target, Batch)
    members = target.members if is_batch else [target]
    shapes = [(m.nx, m.nr) for m in members]
    pattern = members[0].pattern if members else "ab"
    key = lattice_key(target.storage, shapes, pattern)
    if use_cache:
        hit = _load().get(key)
        if hit:
            shape = (int(hit.get("strip", 0)), int(hit["band"]), int(hit["warps"]))
            _apply(target, *shape)
            return shape
    if is_batch:
        def run(n):
            target.step(n, graph=False)
    else:
        run = target.step
    widths = _widths(target.storage, pattern)
    cands = [c for c in (candidates or (BATCH_CANDIDATES if is_batch else LATTICE_CANDIDATES)) if c[0] in widths]
    if not cands:
        raise ValueError(f"no candidate strip width among {widths} for {target.storage}/{pattern}")
    # bring the GPU to its working clocks first, then time every candidate three times, in
    # alternating orders (a fixed order would favour whichever candidate runs last on a
    # warming GPU), and rank each by its slowest run: a shape whose launches fall into a
    # slower schedule part of the time (FP32 band 6 on the 4096 x 1024 jet runs a launch
    # at either 79 or 87 us per step) must not win on its fast launches
    run(max(warmup, steps))
    worst = {}
    for order in (cands, cands[::-1], cands):
        for shape in order:
            _apply(target, *shape)
            ms = _time(run, steps, warmup)
            worst[shape] = max(ms, worst.get(shape, ms))
    results: List[Tuple[float, Tuple[int, int, int]]] = sorted((ms, sh) for sh, ms in worst.items())
    ms, shape = results[0]
    _apply(target, *shape)
    _store(key, {"strip": shape[0], "band": shape[1], "warps": shape[2], "ms_per_step": ms,
                 "timings": [[*sh, t] for t, sh in results]})
    return shape

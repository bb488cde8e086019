"""Autotuner of the radix-sort variant (digit width, threads and keys per
thread of a tile).

It times every compiled variant (tb_sort_variant) on the caller's particles
with CUDA events around whole builds and keeps the fastest, cached per GPU
name and size class (log2 of the particle count) in _build/autotune.json.
`build()` of the binding uses the cached choice when the caller names no
variant.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import _lib

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(n: int) -> str:
    return f"{torch.cuda.get_device_name()}|{max(0, int(math.log2(max(1, n))))}"


def _load() -> dict:
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def cached(n: int):
    """Cached (radix_bits, threads, items) for n particles on this GPU, or None."""
    v = _load().get(_key(n))
    return tuple(v["cfg"]) if v else None


def tune(pos: torch.Tensor, mass: torch.Tensor | None = None, n_crit: int = 16, reps: int = 3,
         save: bool = True):
    """Time every compiled variant on these particles; return (best cfg, {cfg: ms})."""
    times = {}
    tree = None
    for cfg in _lib.sort_variants():
        tree = _lib.build(pos, mass, n_crit=n_crit, sort_cfg=cfg, tree=tree)
        cap = tree.n_cells
        _lib.build(pos, mass, n_crit=n_crit, sort_cfg=cfg, cell_capacity=cap, tree=tree)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            _lib.build(pos, mass, n_crit=n_crit, sort_cfg=cfg, cell_capacity=cap, tree=tree)
        e1.record()
        torch.cuda.synchronize()
        if tree.sync() != 0:
            continue
        times[cfg] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    if save:
        d = _load()
        d[_key(pos.shape[0])] = {"cfg": list(best), "ms": {",".join(map(str, k)): v
                                                          for k, v in times.items()}}
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(d, f, indent=1)
    return best, times

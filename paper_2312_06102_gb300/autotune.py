"""Autotuners of the build's compiled shapes.

tune() times every compiled radix-sort variant (digit width, threads and
keys per thread of a tile; tb_sort_variant) on the caller's particles with
CUDA events around whole builds and keeps the fastest, cached per GPU name
and size class (log2 of the particle count) in _build/autotune.json.
`build()` of the binding uses the cached choice when the caller names no
variant.

tune_batched() does the same for the batched build's block size (512 or
1024 threads per set: two sets per SM at a time, or one), keyed by GPU name,
the number of sets and the size class of the mean set;
`build_batched()` uses the cached choice when the caller names none.
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


_MEM = {"mtime": None, "data": {}}


def _load() -> dict:
    """The cache file's contents, re-read only when the file has changed."""
    try:
        mt = os.path.getmtime(_CACHE)
    except OSError:
        return {}
    if _MEM["mtime"] != mt:
        try:
            with open(_CACHE) as f:
                _MEM["data"] = json.load(f)
            _MEM["mtime"] = mt
        except Exception:
            return {}
    return _MEM["data"]


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
        d = dict(_load())
        d[_key(pos.shape[0])] = {"cfg": list(best), "ms": {",".join(map(str, k)): v
                                                          for k, v in times.items()}}
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(d, f, indent=1)
    return best, times


BATCH_THREADS = (512, 1024)


def _bkey(n_sets: int, n_total: int) -> str:
    mean = max(1, n_total // max(1, n_sets))
    return f"batched|{torch.cuda.get_device_name()}|{n_sets}|{max(0, int(math.log2(mean)))}"


def cached_batched(n_sets: int, n_total: int):
    """Cached batch_threads for this many sets and particles on this GPU, or None."""
    v = _load().get(_bkey(n_sets, n_total))
    return int(v["threads"]) if v else None


def tune_batched(pos: torch.Tensor, mass: torch.Tensor | None, set_offsets: torch.Tensor,
                 n_crit: int = 16, reps: int = 3, save: bool = True):
    """Time the batched build at every block size; return (best threads, {threads: ms})."""
    times = {}
    tree = None
    for th in BATCH_THREADS:
        tree = _lib.build_batched(pos, mass, set_offsets, n_crit=n_crit, batch_threads=th,
                                  tree=tree)
        cap = tree.n_cells
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            _lib.build_batched(pos, mass, set_offsets, n_crit=n_crit, batch_threads=th,
                               cell_capacity=cap, tree=tree)
        e1.record()
        torch.cuda.synchronize()
        if tree.sync() != 0:
            continue
        times[th] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    if save:
        d = dict(_load())
        d[_bkey(set_offsets.shape[0] - 1, pos.shape[0])] = {
            "threads": best, "ms": {str(k): v for k, v in times.items()}}
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(d, f, indent=1)
    return best, times

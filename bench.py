#!/usr/bin/env python3
"""Tree-build throughput on one GB300 (or N replicas).

A step is one full build of the hashed oct-tree -- root cell, keys, radix
sort, leaves, cells with links, moments (tb_build + tb_moments) -- over one
batch of synthetic particles already resident in HBM.  The default workload
is the 2^27-particle clustered-halo set (n_crit = 16).  Prints one JSON line
(rank 0):

  value        Mparticles/s over the K timed steps (device events, max over
               ranks, all ranks' particles)
  roofline     the dominant kernel (one radix-sort pass): algorithmic bytes
               per launch / its mean event-timed duration, against the
               measured HBM copy bandwidth
  cpu_baseline the FP64 oracle, single thread, on a bounded sample
  e2e          the same metric through the C ABI from pinned host buffers,
               host<->device copies inside the timed region
  batched      (when built) batched vs plain per-set builds, same GB300

--impl reference times the oracle instead (the reference arm of the
comparison): host cores, bounded sample, same metric and unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import WORKLOADS, batched_plummer, workload  # noqa: E402

# DRAM bytes per launch of the dominant kernel from one ncu capture, keyed by
# the digest of the kernel source it was taken on; reported only while the
# source is unchanged (see profiles/).
NCU_TRAFFIC = {
    # onesweep pass <8, 512, 8>, N = 2^25 clustered, passes 2, 3 and 4 of a
    # timed build: dram__bytes_read.sum + dram__bytes_write.sum, their mean
    "639068564be370b2": {"bytes": 770.47e6, "n": 1 << 25, "variant": (8, 512, 8)},
}

METRIC = "tree-build Mparticles/s + HBM roofline %; batched vs plain on same GB300"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clustered_2p27", choices=sorted(
        k for k, v in WORKLOADS.items() if v["kind"] != "batched"))
    ap.add_argument("--n", type=int, default=0, help="override particle count")
    ap.add_argument("--n-crit", type=int, default=0)
    ap.add_argument("--radix-bits", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--sort-variant", default="", help="bits,threads,items of a compiled variant")
    ap.add_argument("--cpu-sample", type=int, default=1 << 24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-reorder", action="store_true", help="skip the key-ordered-input build")
    ap.add_argument("--no-walk", action="store_true", help="skip the tree-walk timing")
    ap.add_argument("--precision-workload", default="stress_2p26", choices=sorted(WORKLOADS),
                    help="workload of the --precision report")
    ap.add_argument("--keys", default="morton", choices=["morton", "hilbert"],
                    help="particle key order of the timed builds")
    ap.add_argument("--batched-steps", type=int, default=100)
    ap.add_argument("--batch-threads", type=int, default=0, choices=[0, 512, 1024],
                    help="threads per set of the batched build (default: tuned)")
    ap.add_argument("--batched-sets", type=int, default=0,
                    help="number of sets of the batched workload (default: its 4,096)")
    ap.add_argument("--precision", action="store_true",
                    help="print the per-level moment error of the three modes against the oracle")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_digest():
    h = hashlib.sha256()
    for f in ("tb_sort.cu", "tb_device.cuh"):
        with open(os.path.join(ROOT, "paper_2312_06102_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi samples (every 50 ms), kept when they fall inside the timed
    region (host wall clock), else all of them with a note."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def wait_first(self, timeout=5.0):
        """Block until the sampler has written its first line."""
        t_end = time.time() + timeout
        while self.proc and time.time() < t_end:
            if self.path and os.path.getsize(self.path) > 0:
                return
            time.sleep(0.02)

    def stop(self, window=None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]),
                             {nm for nm, v in zip(names, parts[6:10]) if v.lower().startswith("active")}))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = rows
        note = None
        if window is not None:
            inside = [r for r in rows if window[0] - 0.06 <= r[0] <= window[1] + 0.06]
            if not inside:
                inside, note = rows, "no sample inside the timed region; all samples of the run"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [r[1] for r in inside]
        reasons = set().union(*[r[3] for r in inside])
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        out = {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(r[2] for r in inside)),
               "reasons": sorted(reasons), "samples": len(inside)}
        if note:
            out["note"] = note
        return out


def gen(wl: str, n_override: int):
    spec = dict(WORKLOADS[wl])
    n = n_override or spec["n"]
    t0 = time.perf_counter()
    pos, mass = workload(spec["kind"], n, spec["seed"])
    log(f"[bench] generated {wl} n={n} in {time.perf_counter() - t0:.1f}s")
    return pos, mass, spec, n


def oracle_rate(pos, mass, n_crit, sample):
    """FP64 oracle (single thread): full build + direct-sum moments of the
    first `sample` particles; returns (Mparticles/s, seconds, particles)."""
    import oracle
    m = min(sample, pos.shape[0])
    p, w = np.ascontiguousarray(pos[:m]), np.ascontiguousarray(mass[:m])
    t0 = time.perf_counter()
    t = oracle.build_tree(p, n_crit)
    oracle.moments(t, p, w)
    dt = time.perf_counter() - t0
    return m / dt / 1e6, dt, m


def whole_job_rate(n_per_rank, steps, world, ms, device="cuda"):
    """The slowest rank's time for `steps` builds (max over ranks) and the
    whole-job rate: the particles all ranks built / that time, Mparticles/s.
    Each rank builds its own replica; nothing but this maximum is exchanged."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, n_per_rank * steps * world / (ms / 1e3) / 1e6


def per_step_ms(stages, steps):
    """Median, min and max step time from the (name, ms) stage intervals of
    the timed steps; None when they do not split into `steps` steps.

    tb_stage_times names each interval after the event that closes it, and
    every step records a "start" event first.  The first step's "start"
    closes no interval, so the intervals up to the first one named "start"
    belong to step 1, and each later "start" interval (the gap between two
    steps) opens the next step."""
    if not stages or steps <= 0:
        return None
    per_step = [0.0]
    for i, (name, v) in enumerate(stages):
        if name == "start" and i > 0:
            per_step.append(0.0)
        per_step[-1] += v
    if len(per_step) != steps:
        return None
    return {"median": round(float(np.median(per_step)), 4), "min": round(min(per_step), 4),
            "max": round(max(per_step), 4), "from": "stage events of each timed step"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pos, mass, spec, n = gen(a.workload, a.n)
    n_crit = a.n_crit or spec["n_crit"]
    import oracle
    oracle.build()
    # the per-step sample shrinks as the step count grows, so that the whole
    # run stays near ten full samples of oracle work (a few minutes)
    m = min(a.cpu_sample, n, max(1 << 20, (10 * a.cpu_sample) // max(1, a.steps)))
    for _ in range(max(0, min(a.warmup, 1))):
        oracle_rate(pos, mass, n_crit, min(m, 1 << 16))
    times = []
    for _ in range(a.steps):
        r, dt, _ = oracle_rate(pos, mass, n_crit, m)
        times.append(dt)
    tot = sum(times)
    value = m * len(times) / tot / 1e6
    sample = f"first {m} of the {n} particles of {a.workload}, full FP64 build + direct-sum moments"
    out = {"metric": METRIC, "value": round(value, 4), "unit": "Mparticles/s",
           "impl": "reference", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": round(1e3 * tot / len(times), 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": a.workload, "n_particles": n, "n_crit": n_crit},
           "cpu_baseline": {"value": round(value, 4), "unit": "Mparticles/s", "cores": 1,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": "Mparticles/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(a):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import paper_2312_06102_gb300 as tb
    tb.lib()

    pos, mass, spec, n = gen(a.workload, a.n)
    n_crit = a.n_crit or spec["n_crit"]
    hpos = torch.from_numpy(pos).pin_memory()
    hmass = torch.from_numpy(mass).pin_memory()
    p = hpos.cuda()
    w = hmass.cuda()
    stream = torch.cuda.current_stream()

    ko = 1 if a.keys == "hilbert" else 0
    # pick the radix-sort variant on this workload (untimed), unless one is named
    cfg = None
    tune_ms = None
    if a.sort_variant:
        cfg = tuple(int(v) for v in a.sort_variant.split(","))
    elif a.radix_bits:
        cfg = next(v for v in tb.sort_variants() if v[0] == a.radix_bits)
    elif not a.no_autotune:
        from paper_2312_06102_gb300 import autotune
        cfg, tune_ms = autotune.tune(p, w, n_crit=n_crit)
        log(f"[bench] autotune: {cfg} " + " ".join(f"{k}:{v:.3f}" for k, v in tune_ms.items()))
    # first build sizes the cell arrays; later builds use that capacity and
    # need no host synchronisation
    torch.cuda.synchronize()
    t_first = time.perf_counter()
    tree = tb.build(p, w, n_crit=n_crit, sort_cfg=cfg, key_order=ko)
    C = tree.n_cells
    tb.moments(tree, p, w)
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t_first) * 1e3
    for _ in range(a.warmup):
        tb.build(p, w, n_crit=n_crit, cell_capacity=C, sort_cfg=cfg, tree=tree, key_order=ko)
        tb.moments(tree, p, w)
    torch.cuda.synchronize()
    st = tree.sync()
    if st != 0:
        raise SystemExit(f"warm-up build failed: {tb.STATUS[st]}")

    tree.profile(True)
    tree.stage_times()   # drop anything recorded so far
    clocks = Clocks(local)
    clocks.start()
    clocks.wait_first()
    barrier()
    torch.cuda.synchronize()
    w_begin = time.time()
    l0 = tb.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")   # lets a profiler keep to the timed steps
    e0.record(stream)
    for _ in range(a.steps):
        tb.build(p, w, n_crit=n_crit, cell_capacity=C, sort_cfg=cfg, tree=tree, key_order=ko)
        tb.moments(tree, p, w)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    w_end = time.time()
    barrier()
    ck = clocks.stop((w_begin, w_end))
    launches = tb.kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    stages = tree.stage_times()
    tree.profile(False)
    st = tree.sync()
    if st != 0:
        raise SystemExit(f"timed build failed: {tb.STATUS[st]}")
    ms, value = whole_job_rate(n, a.steps, world, ms)

    # per-step times from the stage marks: the median over the K steps beside
    # the K-step mean of `ms_per_step`
    try:
        step_ms = per_step_ms(stages, a.steps)
    except Exception:
        step_ms = None

    # per-stage totals over the timed region
    agg = {}
    for name, v in stages:
        agg.setdefault(name, [0.0, 0])
        agg[name][0] += v
        agg[name][1] += 1
    sort_ms, sort_launches = agg.get("sort_pass", [0.0, 0])
    passes = max(1, sort_launches // max(1, a.steps))
    bytes_per_launch = (20 + 24 * (passes - 1)) / passes * n
    peak, peak_kind = peaks()
    avg_launch_s = sort_ms / max(1, sort_launches) / 1e3
    achieved = bytes_per_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    dig = kernel_digest()
    rec = NCU_TRAFFIC.get(dig)
    # scaled by the keys per launch (the capture's inputs are 3x L2 already)
    traffic = None
    if rec is not None and cfg is not None and tuple(cfg) == rec["variant"]:
        traffic = rec["bytes"] * n / rec["n"]
    roofline = {"bound": "hbm", "kernel": "onesweep radix pass", "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_kind": peak_kind,
                "traffic": None if traffic is None else round(traffic),
                "algorithmic_bytes_per_launch": round(bytes_per_launch),
                "mean_launch_ms": round(avg_launch_s * 1e3, 4)}
    # whole-build ideal bytes B* = 40 N + 90 C: positions read for the root
    # cell (12 B), positions and masses read once more (16 B), sorted keys and
    # permutation written once (12 B), and a 90-byte cell record (26 B of
    # structure, 64 B of moments)
    strict = 40 * n + 90 * C
    # sort-adjusted: B* plus what this sort moves beyond one sorted write --
    # the unsorted key write (8 B), the first pass's key read and write
    # (20 B), 24 B for each further pass, the run step's key read (8 B):
    # (24 P + 12) N in all, P the global passes, less the 12 N in B*
    sort_adj = strict + 24 * passes * n
    build_s = ms / a.steps / 1e3
    stage_ms = {k: round(v[0] / a.steps, 4) for k, v in agg.items()}

    out = {"metric": METRIC, "value": round(value, 2),
           "unit": "Mparticles/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": round(ms / a.steps, 4), "step_ms": step_ms,
           "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+u64",
           "data": "synthetic (seeded generator, same draw on every rank)",
           "config": {"workload": a.workload, "n_particles": n, "n_crit": n_crit,
                      "n_cells": C, "sort_variant": list(cfg) if cfg else "library default",
                      "autotune_ms": ({",".join(map(str, k)): round(v, 3) for k, v in tune_ms.items()}
                                      if tune_ms else None),
                      "parallelism": f"replicas{world}",
                      "l2": "inputs larger than L2 (1.6 GB positions vs 129 MB), no flush",
                      "mom_mode": "fp32_compensated", "keys": a.keys},
           "roofline": roofline,
           "build_roofline": {"strict_bytes": int(strict),
                              "achieved_gbs": round(strict / build_s / 1e9, 1),
                              "frac": round(strict / build_s / 1e9 / peak, 4),
                              "sort_adjusted_bytes": int(sort_adj),
                              "sort_adjusted_frac": round(sort_adj / build_s / 1e9 / peak, 4)},
           "stage_ms": stage_ms,
           "gpu_launches": int(launches),
           "clocks": ck,
           "first_call": {"ms": round(first_ms, 3),
                          "what": "first tb_build + tb_moments on a new tree, wall clock: "
                                  "allocation, the one cell-count read and the build"}}

    # end to end through the C ABI from pinned host buffers: every step copies
    # its positions and masses in and reads its root moments back; the copy of
    # step t + 1 runs on a second stream while step t builds (two input buffers)
    if not a.no_e2e:
        res = torch.empty(10, dtype=torch.float32).pin_memory()
        p2, w2 = torch.empty_like(p), torch.empty_like(w)
        bufs = [(p, w), (p2, w2)]
        cstream = torch.cuda.Stream()
        with torch.cuda.stream(cstream):     # touch the second buffer once
            p2.copy_(hpos, non_blocking=True)
            w2.copy_(hmass, non_blocking=True)
        tb.build(p, w, n_crit=n_crit, cell_capacity=C, sort_cfg=cfg, tree=tree, key_order=ko)
        # the result read once before timing: its first device allocation
        # would otherwise hold the host until the first step's work is done
        res.copy_(torch.cat([tree.mass[:1], tree.com[0], tree.quad[0]]), non_blocking=True)
        torch.cuda.synchronize()
        barrier()
        # every in-loop copy is bracketed by its own events on the copy stream
        cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(a.steps)]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        used = [torch.cuda.Event(), torch.cuda.Event()]
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        cstream.wait_event(f0)

        def copy_in(b_, t_):
            cev[t_][0].record(cstream)
            with torch.cuda.stream(cstream):
                bufs[b_][0].copy_(hpos, non_blocking=True)
                bufs[b_][1].copy_(hmass, non_blocking=True)
            cev[t_][1].record(cstream)
            copied[b_].record(cstream)

        tree.profile(True)
        tree.stage_times()
        copy_in(0, 0)
        for t_ in range(a.steps):
            b_ = t_ % 2
            stream.wait_event(copied[b_])
            pb, wb = bufs[b_]
            tb.build(pb, wb, n_crit=n_crit, cell_capacity=C, sort_cfg=cfg, tree=tree, key_order=ko)
            # the build reads the inputs only for the root cell and the keys;
            # the moments sum the snapshot the key pass took, so the buffer
            # is free for the next copy once the build's work is done
            used[b_].record(stream)
            tb.moments(tree, pb, wb)
            root = torch.cat([tree.mass[:1], tree.com[0], tree.quad[0]])
            res.copy_(root, non_blocking=True)
            if t_ + 1 < a.steps:
                if t_ >= 1:
                    cstream.wait_event(used[1 - b_])   # step t - 1's build is done with it
                copy_in(1 - b_, t_ + 1)
        f1.record(stream)
        torch.cuda.synchronize()
        e_stages = {}
        for name_, v_ in tree.stage_times():
            e_stages[name_] = e_stages.get(name_, 0.0) + v_ / a.steps
        tree.profile(False)
        ems = f0.elapsed_time(f1)
        ems, evalue = whole_job_rate(n, a.steps, world, ems)
        copy_ms = [c0.elapsed_time(c1) for c0, c1 in cev]
        h2d_bytes = int(p.numel() * p.element_size() + w.numel() * w.element_size())
        out["e2e"] = {"value": round(evalue, 2),
                      "unit": "Mparticles/s", "h2d_bytes_per_step": h2d_bytes,
                      "d2h_bytes_per_step": int(res.numel() * res.element_size()),
                      "ms_per_step": round(ems / a.steps, 4),
                      "h2d_ms_median": round(float(np.median(copy_ms)), 3),
                      "h2d_gbs_median": round(h2d_bytes / (float(np.median(copy_ms)) / 1e3) / 1e9, 1),
                      "pipelining": "step t+1's H2D copy overlaps step t's build (two input "
                                    "buffers); copy times from events around each in-loop copy "
                                    "on the copy stream",
                      "stage_ms": {k: round(v, 4) for k, v in e_stages.items()}}
        del p2, w2

    # key-ordered input: what a simulation sees when it reorders its particle
    # arrays every few steps (tb_reorder), so the build's gather is local
    if not a.no_reorder:
        tb.build(p, w, n_crit=n_crit, cell_capacity=C, sort_cfg=cfg, tree=tree, key_order=ko)
        torch.cuda.synchronize()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        pr = tb.reorder(tree, p)
        wr = tb.reorder(tree, w)
        r1.record(stream)
        torch.cuda.synchronize()
        reorder_ms = r0.elapsed_time(r1)
        tree2 = tb.build(pr, wr, n_crit=n_crit, cell_capacity=C, sort_cfg=cfg, key_order=ko)
        tb.moments(tree2, pr, wr)
        torch.cuda.synchronize()
        for _ in range(a.warmup):
            tb.build(pr, wr, n_crit=n_crit, cell_capacity=C, sort_cfg=cfg, tree=tree2, key_order=ko)
            tb.moments(tree2, pr, wr)
        torch.cuda.synchronize()
        r0.record(stream)
        for _ in range(a.steps):
            tb.build(pr, wr, n_crit=n_crit, cell_capacity=C, sort_cfg=cfg, tree=tree2, key_order=ko)
            tb.moments(tree2, pr, wr)
        r1.record(stream)
        torch.cuda.synchronize()
        kms = r0.elapsed_time(r1) / a.steps
        ok = tree2.sync() == 0 and tree2.n_cells == C
        out["key_ordered_input"] = {
            "reorder_ms_pos_and_mass": round(reorder_ms, 4),
            "build_ms": round(kms, 4),
            "mparticles_s": round(n / (kms / 1e3) / 1e6, 2),
            "same_cell_count": bool(ok),
            "note": "positions and masses reordered into key order by tb_reorder, then "
                    "built again (the same tree, identity permutation)"}
        tree2.free()
        del pr, wr

    if not a.no_walk and world == 1:
        try:
            out["walk"] = run_walk(a, tb, torch)
        except Exception as ex:  # reported, never hides the main line
            out["walk"] = {"error": str(ex)[:200]}

    if not a.no_batched and world == 1:
        try:
            out["batched"] = run_batched(a, tb, torch)
        except Exception as ex:  # reported, never hides the main line
            out["batched"] = {"error": str(ex)[:200]}

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        r, dt, m = oracle_rate(pos, mass, n_crit, a.cpu_sample)
        out["cpu_baseline"] = {"value": round(r, 4), "unit": "Mparticles/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"first {m} particles of the same draw: full FP64 build "
                                         f"+ direct-sum moments, {dt:.1f} s single-threaded"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


_MASK64 = (1 << 64) - 1


def _u64(v):
    """A uint64 constant as the int64 with the same bits."""
    v &= _MASK64
    return v - (1 << 64) if v >= 1 << 63 else v


def _srl(x, k):
    """Logical right shift of int64 tensors holding uint64 bits."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _splitmix(x):
    """SplitMix64 finaliser on int64 tensors (two's-complement wraparound)."""
    z = x + _u64(0x9E3779B97F4A7C15)
    z = (z ^ _srl(z, 30)) * _u64(0xBF58476D1CE4E5B9)
    z = (z ^ _srl(z, 27)) * _u64(0x94D049BB133111EB)
    return z ^ _srl(z, 31)


class Jitter:
    """Per-step positions x_t = fp32(x_0 + j_t) of the batched workload, made on
    the GPU with the same counter-based definition as synth.jitter_offsets."""

    def __init__(self, torch, b, seed, dev="cuda"):
        sizes = np.diff(b.offsets)
        self.dev = dev
        self.torch = torch
        self.base = torch.from_numpy(b.pos).to(dev)
        self.set_id = torch.from_numpy(np.repeat(np.arange(len(sizes), dtype=np.int64), sizes)).to(dev)
        self.local = torch.from_numpy((np.arange(int(b.offsets[-1]), dtype=np.int64)
                                       - np.repeat(b.offsets[:-1], sizes))).to(dev)
        self.amp = torch.from_numpy(np.repeat((1e-4 * b.scale).astype(np.float32), sizes)).to(dev)
        self.h0 = int(_splitmix(torch.tensor([seed], dtype=torch.int64))[0])

    def fill(self, step, out):
        t = self.torch
        h1 = _splitmix(t.tensor([self.h0 ^ step], dtype=t.int64, device=self.dev))
        h2 = _splitmix(h1 ^ self.set_id)
        for ax in range(3):
            h3 = _splitmix(h2 ^ ((self.local << 2) | ax))
            u = _srl(h3, 40).to(t.float32) * (2.0 ** -24)
            out[:, ax] = self.base[:, ax] + (2.0 * u - 1.0) * self.amp


def run_walk(a, tb, torch):
    """Gravity from the tree (tb_walk) on a Plummer sphere of 2^22 particles:
    theta 0.75 and n_crit 10 as in the paper's runs, groups of up to 128
    particles (the fastest of 8 .. 256 here; the paper's group bound is 512),
    quadrupoles on, softening 1e-3 of the root side."""
    n = 1 << 22
    pos, mass = workload("plummer", n, 7)
    p = torch.from_numpy(pos).cuda()
    w = torch.from_numpy(mass).cuda()
    t = tb.build(p, w, n_crit=10)
    tb.moments(t, p, w)
    eps = 1e-3 * t.side
    acc = tb.walk(t, 0.75, eps, n_group=128)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        tb.walk(t, 0.75, eps, n_group=128, out=acc)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ok = t.sync() == 0 and bool(torch.isfinite(acc).all())
    # one more walk, untimed, with profiling on: it counts its interactions
    t.profile(True)
    tb.walk(t, 0.75, eps, n_group=128, out=acc)
    cells, pairs = tb.walk_counts(t)
    t.profile(False)
    t.free()
    # FP32 operations per interaction as the walk evaluates them (an FMA is 2,
    # rsqrt / sqrt / reciprocal 1): a particle pair 19 (offset 3, softened
    # point mass 16), a cell with its quadrupole 66 (double-float offset 6,
    # point mass 16, quadrupole term 44).  Peak: 152 SMs x 128 FP32 lanes x
    # 2 x 2.07 GHz = 80.5 TFLOP/s.
    flops = 19 * pairs + 66 * cells
    peak_tf = 152 * 128 * 2 * 2.07e9 / 1e12
    tf = flops / (ms / 1e3) / 1e12
    return {"workload": "plummer n=2^22 (seed 7)", "theta": 0.75, "n_crit": 10, "n_group": 128,
            "quadrupole": True, "ms": round(ms, 3), "mparticles_s": round(n / (ms / 1e3) / 1e6, 2),
            "finite": ok,
            "interactions": {"cell": cells, "particle": pairs,
                             "per_particle": round((cells + pairs) / n, 1),
                             "g_per_s": round((cells + pairs) / (ms / 1e3) / 1e9, 1)},
            "roofline": {"bound": "alu", "achieved": round(tf, 2), "peak": round(peak_tf, 1),
                         "unit": "TFLOP/s", "frac": round(tf / peak_tf, 4),
                         "flops_per_interaction": {"particle": 19, "cell_quadrupole": 66}}}


def run_batched(a, tb, torch):
    """4096 independent Plummer sets: one tb_build_batched per step, captured in
    a CUDA graph and replayed on jittered positions, against the plain loop of
    one tb_build + tb_moments per set, both timed with CUDA events."""
    spec = WORKLOADS["batched_4096"]
    t0 = time.perf_counter()
    b = batched_plummer(n_sets=a.batched_sets or spec["n_sets"], seed=spec["seed"])
    log(f"[bench] generated batched_4096 ({int(b.offsets[-1])} particles) in {time.perf_counter() - t0:.1f}s")
    n = int(b.offsets[-1])
    S = len(b.offsets) - 1
    n_crit = spec["n_crit"]
    p = torch.from_numpy(b.pos).cuda()
    w = torch.from_numpy(b.mass).cuda()
    off = torch.from_numpy(b.offsets).cuda()
    jit = Jitter(torch, b, spec["seed"])
    # the block size per set (512 or 1024 threads), tuned untimed unless named
    bt, bt_ms = 0, None
    if a.batch_threads:
        bt = a.batch_threads
    elif not a.no_autotune:
        from paper_2312_06102_gb300 import autotune
        bt, bt_ms = autotune.tune_batched(p, w, off, n_crit=n_crit)
        log(f"[bench] batched autotune: {bt} " + " ".join(f"{k}:{v:.3f}" for k, v in bt_ms.items()))
    tree = tb.build_batched(p, w, off, n_crit=n_crit, batch_threads=bt)
    cap = int(tree.n_cells * 1.1) + 1024
    stream = torch.cuda.Stream()
    g_build = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        tb.build_batched(p, w, off, n_crit=n_crit, cell_capacity=cap, tree=tree, stream=stream,
                         batch_threads=bt)
        jit.fill(0, p)
        stream.synchronize()
        l0 = tb.kernel_launches()
        with torch.cuda.graph(g_build, stream=stream):
            tb.build_batched(p, w, off, n_crit=n_crit, cell_capacity=cap, tree=tree, stream=stream,
                             batch_threads=bt)
        per_build = tb.kernel_launches() - l0
    steps = a.batched_steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            g_build.replay()
        for t_ in range(steps):
            jit.fill(t_ + 1, p)
            evs[t_][0].record(stream)
            g_build.replay()
            evs[t_][1].record(stream)
        stream.synchronize()
    st = tree.sync(stream)
    if st != 0:
        raise RuntimeError(f"batched replay failed: {tb.STATUS[st]}")
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    batched_ms = float(np.median(ms))
    # the same build as one cooperative launch (tb_params.batch_one_launch),
    # captured and replayed the same way, for the record
    g_one = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        tb.build_batched(p, w, off, n_crit=n_crit, cell_capacity=cap, tree=tree, stream=stream,
                         batch_threads=bt, one_launch=True)
        stream.synchronize()
        with torch.cuda.graph(g_one, stream=stream):
            tb.build_batched(p, w, off, n_crit=n_crit, cell_capacity=cap, tree=tree, stream=stream,
                             batch_threads=bt, one_launch=True)
        for _ in range(3):
            g_one.replay()
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for _ in range(20):
            g_one.replay()
        o1.record(stream)
        stream.synchronize()
    one_ms = o0.elapsed_time(o1) / 20
    if tree.sync(stream) != 0:
        raise RuntimeError("one-launch batched replay failed")
    # stage times of a few builds outside the graph (events at stage ends)
    tree.profile(True)
    tree.stage_times(stream)
    with torch.cuda.stream(stream):
        for _ in range(3):
            tb.build_batched(p, w, off, n_crit=n_crit, cell_capacity=cap, tree=tree, stream=stream,
                             batch_threads=bt)
    st_ = tree.stage_times(stream)
    tree.profile(False)
    stages = {}
    for name, v in st_:
        if name != "start":
            stages[name] = stages.get(name, 0.0) + v / 3

    # plain loop: one tb_build + tb_moments per set, one tree rebuilt in place
    sizes = np.diff(b.offsets)
    plain = tb.build(p[: int(sizes[0])], w[: int(sizes[0])], n_crit=n_crit)
    caps = 0
    for s_ in range(S):
        lo_, hi_ = int(b.offsets[s_]), int(b.offsets[s_ + 1])
        caps = max(caps, 2 * (hi_ - lo_) + 64)
    loops = 2
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    tw = time.perf_counter()
    e0.record()
    for _ in range(loops):
        for s_ in range(S):
            lo_, hi_ = int(b.offsets[s_]), int(b.offsets[s_ + 1])
            ps, ws_ = p[lo_:hi_], w[lo_:hi_]
            tb.build(ps, ws_, n_crit=n_crit, cell_capacity=caps, tree=plain)
            tb.moments(plain, ps, ws_)
    e1.record()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - tw) / loops * 1e3
    plain_ms = e0.elapsed_time(e1) / loops
    if plain.sync() != 0:
        raise RuntimeError("plain loop failed")
    return {"workload": "batched_4096" if S == spec["n_sets"] else f"batched_{S}",
            "sets": S, "particles": n, "n_crit": n_crit,
            "graph_replays": steps, "cell_capacity": cap,
            "batched_ms_per_build": round(batched_ms, 4),
            "batched_mparticles_s": round(n / batched_ms / 1e3, 1),
            "plain_loop_ms_per_build": round(plain_ms, 3),
            "plain_loop_wall_ms": round(wall, 1),
            "plain_loop_mparticles_s": round(n / plain_ms / 1e3, 2),
            "speedup_vs_plain": round(plain_ms / batched_ms, 1),
            "kernels_per_batched_build": int(per_build),
            "batch_threads": int(bt) if bt else 512,
            "one_launch_ms_per_build": round(one_ms, 4),
            "batch_threads_autotune_ms": ({str(k): round(v, 3) for k, v in bt_ms.items()}
                                          if bt_ms else None),
            "stage_ms": {k: round(v, 4) for k, v in stages.items()},
            "timing": "CUDA events around each graph replay (jitter kernel outside); plain loop: "
                      "events around the whole loop of per-set calls, no host sync inside"}


def run_precision_batched(a):
    """The batched workload's moment error per level, three modes, against the
    oracle's FP64 direct sums over every cell of 64 sets spread over the size
    range (each set is its own tree)."""
    import torch
    import oracle
    import paper_2312_06102_gb300 as tb
    spec = WORKLOADS["batched_4096"]
    b = batched_plummer(n_sets=spec["n_sets"], seed=spec["seed"])
    n_crit = a.n_crit or spec["n_crit"]
    sizes = np.diff(b.offsets)
    order = np.argsort(sizes, kind="stable")
    pick = order[np.linspace(0, len(order) - 1, 64).astype(np.int64)]
    p = torch.from_numpy(b.pos).cuda()
    w = torch.from_numpy(b.mass).cuda()
    off = torch.from_numpy(b.offsets).cuda()
    ref = {}
    for s_ in pick:
        lo_, hi_ = int(b.offsets[s_]), int(b.offsets[s_ + 1])
        o = oracle.build_tree(b.pos[lo_:hi_], n_crit)
        M, com, quad, _ = oracle.moments(o, b.pos[lo_:hi_], b.mass[lo_:hi_])
        ref[int(s_)] = (o.level.astype(np.int64), o.side, M, com, quad)
    report = {"workload": "batched_4096", "sets_compared": len(pick),
              "particles_compared": int(sizes[pick].sum()), "n_crit": n_crit, "levels": {}}
    for mode, name in ((0, "fp32_comp"), (1, "fp32_plain"), (2, "fp64")):
        t = tb.build_batched(p, w, off, n_crit=n_crit, mom_mode=mode)
        torch.cuda.synchronize()
        co = t.set_cell_offset.cpu().numpy()
        gm_all = (t.mass64 if mode == 2 else t.mass).cpu().numpy()
        gc_all = t.com64.cpu().numpy() if mode == 2 else (
            t.com.cpu().numpy().astype(np.float64) + t.com_lo.cpu().numpy().astype(np.float64))
        gq_all = (t.quad64 if mode == 2 else t.quad).cpu().numpy().astype(np.float64)
        for s_, (lv, side, M, com, quad) in ref.items():
            a0, a1 = int(co[s_]), int(co[s_ + 1])
            assert a1 - a0 == len(lv)
            sc = side / np.exp2(lv)
            em = np.abs(gm_all[a0:a1].astype(np.float64) / M - 1)
            ec = np.abs(gc_all[a0:a1] - com).max(1) / sc
            eq = np.abs(gq_all[a0:a1] - quad).max(1) / (M * sc * sc)
            for d in np.unique(lv):
                k = lv == d
                r = report["levels"].setdefault(int(d), {"cells": 0})
                if mode == 0:
                    r["cells"] += int(k.sum())
                cur = r.setdefault(name, {"mass_rel": 0.0, "com_per_side": 0.0, "quad_per_Ms2": 0.0})
                cur["mass_rel"] = max(cur["mass_rel"], float(em[k].max()))
                cur["com_per_side"] = max(cur["com_per_side"], float(ec[k].max()))
                cur["quad_per_Ms2"] = max(cur["quad_per_Ms2"], float(eq[k].max()))
        t.free()
    print(json.dumps(report), flush=True)
    return 0


def run_precision(a):
    """Largest moment error per level for FP32-compensated, FP32-plain and FP64
    moments against direct FP64 sums of the oracle (sampled cells)."""
    import torch
    import oracle
    import paper_2312_06102_gb300 as tb
    wl = a.precision_workload
    if WORKLOADS[wl]["kind"] == "batched":
        return run_precision_batched(a)
    pos, mass, spec, n = gen(wl, a.n)
    n_crit = a.n_crit or spec["n_crit"]
    idx = oracle.PrefixIndex(pos)
    p = torch.from_numpy(pos).cuda()
    w = torch.from_numpy(mass).cuda()
    rng = np.random.default_rng(0)
    report = {"workload": wl, "n_particles": n, "n_crit": n_crit, "levels": {}}
    cells = lv = None
    for mode, name in ((0, "fp32_comp"), (1, "fp32_plain"), (2, "fp64")):
        t = tb.build(p, w, n_crit=n_crit, mom_mode=mode)
        tb.moments(t, p, w)
        torch.cuda.synchronize()
        if cells is None:
            lv_all = t.level.cpu().numpy()
            sel = []
            for d in range(22):
                ids = np.nonzero(lv_all == d)[0]
                if len(ids):
                    sel.append(ids if len(ids) <= 400 else rng.choice(ids, 400, replace=False))
            cells = np.unique(np.concatenate(sel))
            lv = lv_all[cells].astype(np.int64)
            M, com, quad, aabb, cnt = idx.moments(mass, lv, t.ckey.cpu().numpy()[cells])
        gm = t.mass.cpu().numpy()[cells].astype(np.float64)
        gc = t.com.cpu().numpy()[cells].astype(np.float64) + t.com_lo.cpu().numpy()[cells].astype(np.float64)
        gq = t.quad.cpu().numpy()[cells].astype(np.float64)
        if mode == 2:
            gm, gc, gq = (t.mass64.cpu().numpy()[cells], t.com64.cpu().numpy()[cells],
                          t.quad64.cpu().numpy()[cells])
        s = t.side / np.exp2(lv)
        em = np.abs(gm / M - 1)
        ec = np.abs(gc - com).max(1) / s
        eq = np.abs(gq - quad).max(1) / (M * s * s)
        for d in np.unique(lv):
            r = report["levels"].setdefault(int(d), {"cells_sampled": int((lv == d).sum())})
            k = lv == d
            r[name] = {"mass_rel": float(em[k].max()), "com_per_side": float(ec[k].max()),
                       "quad_per_Ms2": float(eq[k].max())}
        t.free()
    print(json.dumps(report), flush=True)
    return 0


def main():
    a = args_()
    if a.impl == "reference":
        return run_reference(a)
    if a.precision:
        return run_precision(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())

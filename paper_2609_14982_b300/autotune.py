"""Autotuner for the traversal launch settings of a built tangent.

The structure of a tangent is fixed at build time; how it is traversed is not.  This
module times one J p and one J^T y (CUDA events on the current stream) for each
candidate run-time setting and applies the fastest with tangent_tune, caching the choice
per (grid size, sources, levels, R, dtype) in a JSON file.  The knobs:
  schedule           persistent item queue, cluster (one cluster per source, a hardware
                     barrier per level), level-synchronous (one cooperative launch, a
                     grid-wide barrier per global step) or graph-replayed per-level launches;
  rhs_chunk          right-hand-side columns per traversal pass;
  threads per level  cluster schedule: cluster_size CTAs x cluster_threads threads work on
                     one source's level; persistent schedule: CTAs per SM (ctas_per_sm);
  lane groups        pass_units: right-hand-side vectors a thread carries per position
                     (level-synchronous schedule: rows a thread has in flight, 1, 2 or 4);
  block tiling       block_lu_min: SCC blocks of at least this size are solved by
                     column-parallel substitution with the LU factors instead of the
                     explicit inverse;
  waits              per-item dependencies or whole previous level (persistent);
  concurrency        split_dirs: J p and J^T y on two streams at once, each with about
                     half the CTAs (the pair is timed that way);
  items in flight    item_slots: work items a CTA of the persistent schedule holds at once.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import eik

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "eik_autotune.json")


# every knob at its default: a candidate names only what it changes
DEFAULTS = {"schedule": eik.SCHED_PERSISTENT, "rhs_chunk": 0, "ctas_per_sm": 0, "item_deps": 1, "pass_units": 0,
            "cluster_size": 0, "cluster_threads": 0, "block_lu_min": 0, "split_dirs": 0, "item_slots": 0}


def _key(tan, R: int, dtype) -> str:
    st = tan.stats(0)
    lv = max(tan.stats(a)["levels"] for a in range(tan.S))
    return f"N{tan.N}-S{tan.S}-L{lv}-R{R}-{str(dtype).split('.')[-1]}-E{st['edges']}"


def candidates(R: int, dtype) -> list:
    """The full search space (used by autotune when no candidates are given)."""
    unit = 4 if dtype == torch.float32 else 2
    chunks = [0] + [c for c in (R // 2, R // 4) if c >= unit and c % unit == 0 and c < R]
    out = []
    for ch in chunks:
        out.append({"schedule": eik.SCHED_LEVELS, "ctas_per_sm": 0, "rhs_chunk": ch})
        out.append({"schedule": eik.SCHED_STAGED, "ctas_per_sm": 0, "rhs_chunk": ch})
        for per_sm in (0, 1, 2):
            for deps in (1, 0):
                for pu in (1, 2):
                    out.append({"schedule": eik.SCHED_PERSISTENT, "ctas_per_sm": per_sm, "rhs_chunk": ch,
                                "item_deps": deps, "pass_units": pu})
        for cs in (0, 4, 8, 16):
            for ct in (128, 256):
                for pu in (2, 4):
                    out.append({"schedule": eik.SCHED_CLUSTER, "rhs_chunk": ch, "cluster_size": cs,
                                "cluster_threads": ct, "pass_units": pu})
        for pu in (0, 2, 4):
            out.append({"schedule": eik.SCHED_SYNC, "rhs_chunk": ch, "pass_units": pu})
        for blk in (0, 64):
            out.append({"schedule": eik.SCHED_PERSISTENT, "rhs_chunk": ch, "block_lu_min": blk})
        for per_sm in (1, 2):
            out.append({"schedule": eik.SCHED_PERSISTENT, "rhs_chunk": ch, "split_dirs": 1, "ctas_per_sm": per_sm})
        for slots in (2, 3):
            out.append({"schedule": eik.SCHED_PERSISTENT, "rhs_chunk": ch, "item_slots": slots})
            out.append({"schedule": eik.SCHED_PERSISTENT, "rhs_chunk": ch, "item_slots": slots, "split_dirs": 1,
                        "ctas_per_sm": 2})
    return out


def quick_candidates(R: int, dtype) -> list:
    """A short list for callers that tune on every run (the benchmark): the defaults of
    each schedule, the cluster schedule at two sizes, and the lane-group and
    block-tiling variants of the persistent schedule."""
    base = {"rhs_chunk": 0, "ctas_per_sm": 0, "item_deps": 1, "pass_units": 0, "cluster_size": 0,
            "cluster_threads": 0, "block_lu_min": 0, "split_dirs": 0, "item_slots": 0}
    out = [dict(base, schedule=eik.SCHED_PERSISTENT),
           dict(base, schedule=eik.SCHED_PERSISTENT, split_dirs=1, ctas_per_sm=2),
           dict(base, schedule=eik.SCHED_PERSISTENT, split_dirs=1, ctas_per_sm=2, item_slots=2),
           dict(base, schedule=eik.SCHED_PERSISTENT, item_slots=2),
           dict(base, schedule=eik.SCHED_PERSISTENT, pass_units=2),
           dict(base, schedule=eik.SCHED_PERSISTENT, block_lu_min=64),
           dict(base, schedule=eik.SCHED_CLUSTER),
           dict(base, schedule=eik.SCHED_CLUSTER, cluster_size=8, pass_units=2),
           dict(base, schedule=eik.SCHED_SYNC, pass_units=4),
           dict(base, schedule=eik.SCHED_LEVELS)]
    return out


def run_pair(tan, p, y, d_rec=None, g=None, streams=None):
    """One J p + J^T y pair on the current stream: in order, or (split_dirs with two
    streams given) J p on streams[0] and J^T y on streams[1] at once, joined back."""
    if streams is None or not tan.opts.split_dirs:
        tan.apply(p, shared_model=True, d_rec=d_rec)
        tan.apply_T(y, sum_sources=True, g=g)
        return
    cur = torch.cuda.current_stream()
    ev = torch.cuda.Event()
    ev.record(cur)
    for st in streams:
        st.wait_event(ev)
    with torch.cuda.stream(streams[0]):
        tan.apply(p, shared_model=True, d_rec=d_rec)
    with torch.cuda.stream(streams[1]):
        tan.apply_T(y, sum_sources=True, g=g)
    for st in streams:
        done = torch.cuda.Event()
        done.record(st)
        cur.wait_event(done)


def time_setting(tan, p, y, reps: int = 3) -> float:
    """Mean milliseconds of one J p + J^T y pair (after one untimed call)."""
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    run_pair(tan, p, y, streams=streams)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        run_pair(tan, p, y, streams=streams)
    e1.record(stream)
    torch.cuda.synchronize()
    tan.status()
    return e0.elapsed_time(e1) / reps


def autotune(tan, R: int, dtype=torch.float32, reps: int = 3, cache_path: str | None = DEFAULT_CACHE,
             cands: list | None = None, seed: int = 0) -> dict:
    """Pick the fastest setting for this tangent and R, apply it, return the record."""
    key = _key(tan, R, dtype)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache and cands is None:
        best = cache[key]["setting"]
        tan.tune(**{**DEFAULTS, **best})
        return dict(cache[key], cached=True)
    gen = torch.Generator("cuda").manual_seed(seed)
    p = torch.randn((tan.N, R), device="cuda", dtype=dtype, generator=gen)
    y = torch.randn((tan.S, max(tan.n_rec, 1), R), device="cuda", dtype=dtype, generator=gen)
    results = []
    t0 = time.time()
    for c in (cands or candidates(R, dtype)):
        tan.tune(**{**DEFAULTS, **c})
        results.append((time_setting(tan, p, y, reps), c))
    results.sort(key=lambda r: r[0])
    best_ms, best = results[0]
    tan.tune(**{**DEFAULTS, **best})
    rec = {"setting": best, "ms": best_ms, "tried": [{"ms": ms, **c} for ms, c in results],
           "tune_s": time.time() - t0}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache[key] = rec
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(rec, cached=False)

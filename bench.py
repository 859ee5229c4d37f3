"""Benchmark: paired J p + J^T y node-updates/s of the frozen full-metric tangent.

Workload (3-D tomography-scale apply): 101 x 101 x 51 curvilinear grid over
20 x 20 x 8 km, Gaussian-hill topography on a seeded smooth random surface,
v = 2.0 + 0.5 z km/s with a +-5% 2 km checkerboard, 25 surface sources, a block of
R = 64 model-space right-hand sides shared by all sources, 441 surface receivers.
One step = the whole hot path once: J p (M, C, forward block traversal, P sampling)
and J^T y (P^T, reverse traversal with U^T/L^T/P^T blocks, C^T M^T, sum over sources),
FP32 substitution with FP64 SCC blocks.  Node-updates per step = 2 N S R.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own 25 sources (weak scaling); J^T's
source sum ends in one NCCL all-reduce of g [N][R].
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "J·v+Jᵀ·w node-updates/s per B300 vs GPU sweeping; % HBM roofline"
UNIT = "node-updates/s"
WORKLOAD = "3d-101x101x51-S25-R64 (config: 3-D tomography-scale apply)"
KRYLOV_CHUNK = 256      # item size of the tangents of the one-right-hand-side Krylov workloads
KRYLOV_SLOTS = 2        # items held per CTA in those Krylov loops (measured: 22.7 against 25.0 ms per LSQR iteration)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (read-only queries)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


KERNEL_SOURCES = ("eik_apply.cu", "eik_trav.h", "eik_vec.cuh")   # the files that define the traversal kernels


def kernel_source_digest() -> str:
    """SHA-256 over the traversal kernels' source files (those present), in a fixed order."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        path = os.path.join(ROOT, "paper_2609_14982_b300", "csrc", name)
        if os.path.exists(path):
            h.update(open(path, "rb").read())
    return h.hexdigest()


def measured_traffic(direction: str, kernel: str) -> float | None:
    """DRAM bytes per node-update of the traversal kernel from the committed ncu summary
    (profiles/traffic.txt: one line per kernel and direction with the SHA-256 of the
    kernel sources it was captured from, kernel_source_digest); None once the kernel
    source has changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        digest = kernel_source_digest()
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            kv = dict(tok.split("=", 1) for tok in line.split())
            if kv.get("direction") == direction and kv.get("kernel") == kernel and kv.get("source_sha256") == digest:
                return float(kv["bytes_per_update"])
    except (OSError, ValueError, KeyError):
        return None
    return None


def algorithmic_bytes(st_list, R: int, esz: int, S: int, N: int, n_rec: int) -> dict:
    """Bytes each call must move (per call, all sources), counted at the method's own
    minimum for this layout:
      structure, per (source, node): perm 4 + row offset 4 + C*M esz + receiver slot 4 and,
        per upstream edge, index 4 + weight esz; read once per call and shared by the R
        right-hand sides;
      J p: the shared model p [N][R] once (every source reads it, but it is one array),
        dT written for every node-update (downstream levels read it back from L2), d_rec;
      J^T y: y (receivers), lam written for every node-update, g [N][R] written once.
    The re-reads of p by the 25 sources and the source-sum kernel's read of lam are not
    counted (they are what a perfect cache would absorb).  For comparison, the per-update
    figure 2 esz + 36/R (FP32) that reads the input once per source is also returned."""
    edges = sum(s["edges"] for s in st_list)
    struct = S * N * (12 + esz) + edges * (4 + esz)
    upd = S * N * R
    fwd = N * R * esz + upd * esz + struct + n_rec * S * R * esz
    bwd = n_rec * S * R * esz + upd * esz + struct + N * R * esz
    per_source_input = upd * esz * 2 + struct + n_rec * S * R * esz
    return {"fwd": fwd, "bwd": bwd, "struct_per_node": struct / (S * N), "updates": upd,
            "fwd_per_update": fwd / upd, "bwd_per_update": bwd / upd,
            "fwd_per_update_input_per_source": per_source_input / upd}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2609_14982_b300 import eik
    from paper_2609_14982_b300 import workloads as W
    from paper_2609_14982_b300.sharding import reduce_model_gradient

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = W.config3()
    g = wl.grid
    src = wl.src.copy()
    if rank > 0:   # each rank owns its own 25 sources: shift the lattice by `rank` nodes in x
        src = np.array([g.index(10 + 20 * (a // 5) + rank % 10, 10 + 20 * (a % 5), 0) for a in range(len(src))],
                       dtype=np.int32)
    if args.sources > 0:
        src = src[:args.sources]
    S, N, R, n_rec = len(src), g.N, wl.R, len(wl.rec)
    workload = WORKLOAD if S == 25 else WORKLOAD.replace("S25", f"S{S}")
    dg = eik.DeviceGrid(g, device=dev)
    s = torch.tensor(wl.s, device=dev)
    t0 = time.time()
    cache = args.state_cache
    if cache and os.path.exists(cache):
        # states written by an earlier run of this command (profiling runs skip the state solve)
        T = torch.tensor(np.load(cache), device=dev)
        assert tuple(T.shape) == (S, N)
        cyc = -1
    else:
        T, cyc = eik.eik_forward(dg, s, src)
        if cache:
            np.save(cache, T.cpu().numpy())
    torch.cuda.synchronize()
    t_state = time.time() - t0
    sched = {"persistent": eik.SCHED_PERSISTENT, "levels": eik.SCHED_LEVELS, "staged": eik.SCHED_STAGED,
             "cluster": eik.SCHED_CLUSTER, "sync": eik.SCHED_SYNC}[args.schedule]
    opts = eik.default_opts(schedule=sched, item_deps=0 if args.level_waits else 1, ctas_per_sm=args.ctas_per_sm,
                            cluster_size=args.cluster_size, cluster_threads=args.cluster_threads,
                            pass_units=args.pass_units, split_dirs=int(args.split_dirs), item_slots=args.item_slots)
    if args.split_dirs and not args.ctas_per_sm:
        opts.ctas_per_sm = 2
    if args.chunk:
        opts.chunk = args.chunk
    t0 = time.time()
    tan = eik.Tangent(dg, T, s, src, rec=wl.rec, opts=opts)
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    st = [tan.stats(a) for a in range(S)]

    dtype = torch.float32
    schedule, pass_units, tuned, item_slots = args.schedule, args.pass_units, None, args.item_slots
    if args.autotune:
        # time each schedule's default and a few variants on this tangent (one J p + J^T y
        # pair each, CUDA events) and keep the fastest for the timed region
        from paper_2609_14982_b300.autotune import autotune, quick_candidates
        rec = autotune(tan, R, dtype, reps=3, cache_path=None, cands=quick_candidates(R, dtype), seed=rank)
        tuned = {"setting": rec["setting"], "ms": round(rec["ms"], 3), "tune_s": round(rec["tune_s"], 2),
                 "tried": [{k: v for k, v in c.items() if k in ("ms", "schedule", "pass_units", "block_lu_min",
                                                                 "cluster_size", "split_dirs", "ctas_per_sm",
                                                                 "item_slots")}
                           for c in rec["tried"]]}
        for c in tuned["tried"]:
            c["ms"] = round(c["ms"], 3)
        names = {eik.SCHED_PERSISTENT: "persistent", eik.SCHED_LEVELS: "levels", eik.SCHED_STAGED: "staged",
                 eik.SCHED_CLUSTER: "cluster", eik.SCHED_SYNC: "sync"}
        schedule = names[rec["setting"]["schedule"]]
        pass_units = rec["setting"].get("pass_units", 0)
        item_slots = rec["setting"].get("item_slots", 0)
    gen = torch.Generator(dev).manual_seed(20263 + rank)
    p = torch.randn((N, R), device=dev, dtype=dtype, generator=gen)
    y = torch.randn((S, n_rec, R), device=dev, dtype=dtype, generator=gen)
    d_rec = torch.empty((S, n_rec, R), device=dev, dtype=dtype)
    gvec = torch.empty((N, R), device=dev, dtype=dtype)
    stream = torch.cuda.current_stream(dev)
    # with split_dirs (chosen by the autotuner) J p and J^T y of a step run at once on two
    # streams; the kernel times are then taken on those streams
    concurrent = bool(tan.opts.split_dirs)
    pair_streams = (torch.cuda.Stream(dev), torch.cuda.Stream(dev))

    def pair(pv, yv, ev=None):
        if not concurrent:
            if ev: ev[0].record(stream)
            tan.apply(pv, shared_model=True, d_rec=d_rec)
            if ev: ev[1].record(stream)
            tan.apply_T(yv, sum_sources=True, g=gvec)
            if ev: ev[2].record(stream)
            return
        fork = torch.cuda.Event()
        fork.record(stream)
        sa, sb = pair_streams
        sa.wait_event(fork)
        sb.wait_event(fork)
        with torch.cuda.stream(sa):
            if ev: ev[0].record(sa)
            tan.apply(pv, shared_model=True, d_rec=d_rec)
            if ev: ev[1].record(sa)
        with torch.cuda.stream(sb):
            if ev: ev[2].record(sb)
            tan.apply_T(yv, sum_sources=True, g=gvec)
            if ev: ev[3].record(sb)
        for st_ in pair_streams:
            join = torch.cuda.Event()
            join.record(st_)
            stream.wait_event(join)

    def step():
        pair(p, y)
        reduce_model_gradient(gvec)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tan.status()

    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(args.steps)]
    clk = Clocks(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        pair(p, y, evs[k])
        reduce_model_gradient(gvec)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    tan.status()
    ms = start.elapsed_time(end) / args.steps
    t_fwd = [e[0].elapsed_time(e[1]) for e in evs]
    t_bwd = [e[2].elapsed_time(e[3]) if concurrent else e[1].elapsed_time(e[2]) for e in evs]
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt)
    upd_step = 2.0 * N * S * R * world
    value = upd_step / (ms / 1e3)

    # ---- end to end through the public API: pinned host inputs in, results out.  Every
    # step copies its inputs (p, y) from pinned host memory and its results (d_rec, g) back;
    # the copies run on two copy streams into double-buffered device arrays, so the input
    # copy of step k + 1 and the result copy of step k - 1 overlap the traversals of step k.
    p_h = torch.empty((N, R), dtype=dtype, pin_memory=True).copy_(p.cpu())
    y_h = torch.empty((S, n_rec, R), dtype=dtype, pin_memory=True).copy_(y.cpu())
    drec_h = torch.empty((S, n_rec, R), dtype=dtype, pin_memory=True)
    g_h = torch.empty((N, R), dtype=dtype, pin_memory=True)
    nbuf = 2
    p_ds = [torch.empty_like(p) for _ in range(nbuf)]
    y_ds = [torch.empty_like(y) for _ in range(nbuf)]
    drec_ds = [torch.empty_like(d_rec) for _ in range(nbuf)]
    g_ds = [torch.empty_like(gvec) for _ in range(nbuf)]
    c_in, c_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_run(nsteps):
        """nsteps pipelined steps, all issued on the streams; returns when issued."""
        in_ready = [None] * nbuf      # input copy of the step using buffer b landed
        used = [None] * nbuf          # traversals of the step that used buffer b finished
        out_done = [None] * nbuf      # result copy of the step that used buffer b finished
        start_ev = torch.cuda.Event()
        start_ev.record(stream)
        for st_ in (c_in, c_out, *pair_streams):
            st_.wait_event(start_ev)

        def issue_in(k):
            b = k % nbuf
            if used[b] is not None:
                c_in.wait_event(used[b])
            with torch.cuda.stream(c_in):
                p_ds[b].copy_(p_h, non_blocking=True)
                y_ds[b].copy_(y_h, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(c_in)
            in_ready[b] = ev

        issue_in(0)
        for k in range(nsteps):
            b = k % nbuf
            if k + 1 < nsteps:
                issue_in(k + 1)
            sa, sb = pair_streams if concurrent else (pair_streams[0], pair_streams[0])
            for st_ in {sa, sb}:
                st_.wait_event(in_ready[b])
                if out_done[b] is not None:
                    st_.wait_event(out_done[b])
            with torch.cuda.stream(sa):
                tan.apply(p_ds[b], shared_model=True, d_rec=drec_ds[b])
            with torch.cuda.stream(sb):
                tan.apply_T(y_ds[b], sum_sources=True, g=g_ds[b])
                reduce_model_gradient(g_ds[b])
            ev = torch.cuda.Event()
            for st_ in {sa, sb}:
                e_ = torch.cuda.Event()
                e_.record(st_)
                c_out.wait_event(e_)
            ev.record(c_out)
            used[b] = ev
            with torch.cuda.stream(c_out):
                drec_h.copy_(drec_ds[b], non_blocking=True)
                g_h.copy_(g_ds[b], non_blocking=True)
                ev2 = torch.cuda.Event()
                ev2.record(c_out)
            out_done[b] = ev2
        for st_ in (c_in, c_out, *pair_streams):
            j = torch.cuda.Event()
            j.record(st_)
            stream.wait_event(j)

    e2e_run(max(1, args.warmup))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        tt = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt)
    # the last step's results arrived on the host: they match the device-resident pair
    assert torch.equal(g_h, g_ds[(args.steps - 1) % nbuf].cpu()) and torch.equal(drec_h, drec_ds[(args.steps - 1) % nbuf].cpu())
    h2d = (p_h.numel() + y_h.numel()) * 4
    d2h = (drec_h.numel() + g_h.numel()) * 4

    if rank != 0:
        tan.free()
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (forward or reverse traversal)
    peak, peak_kind = _peaks()
    ab = algorithmic_bytes(st, R, 4, S, N, n_rec)
    mf, mb = statistics.mean(t_fwd), statistics.mean(t_bwd)
    # The dominant kernel is the J traversal: J p is that one launch, while the timed J^T y
    # call is the reverse traversal plus the separate source-sum kernel, and the launch
    # list of this step gives the J traversal the largest share of any single kernel.
    dom, other = "fwd", "bwd"
    dom_ms = mf
    achieved = ab[dom] / (dom_ms / 1e3) / 1e9
    kname = {"persistent": "k_traverse_persistent<float,4,%s>" if pass_units <= 1 else
                           "k_traverse_persistent<float,4,%s," + str(min(pass_units, 4)) + ",1>",
             "levels": "k_traverse_level<float,4,%s,1>", "staged": "k_traverse_staged<float,4,%s>",
             "cluster": "k_traverse_cluster<float,4,%s," + str(pass_units or 4) + ">",
             "sync": "k_traverse_sync<float,4,%s>"}[schedule]
    if schedule == "persistent" and item_slots >= 2 and pass_units <= 1:
        kname = "k_traverse_multi<float,4,%s," + str(min(item_slots, 4)) + ">"
    kname = kname % ("false" if dom == "fwd" else "true")
    tpu = measured_traffic(dom, kname)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None if tpu is None else round(tpu * ab["updates"]),
                "kernel": kname,
                "bytes_per_launch": ab[dom], "bytes_per_update": round(ab[dom + "_per_update"], 3),
                "bytes_note": "p counted once per call; with p read once per source the update moves "
                              f"{ab['fwd_per_update_input_per_source']:.2f} B",
                "peak_kind": f"{peak_kind} hbm_gbs",
                "concurrent_with_other_direction": concurrent,
                "pair_achieved_gbs": round((ab["fwd"] + ab["bwd"]) / (ms / 1e3) / 1e9, 1),
                "pair_frac": round((ab["fwd"] + ab["bwd"]) / (ms / 1e3) / 1e9 / peak, 4),
                "pair_note": "J p and J^T y algorithmic bytes over the whole step; with the directions concurrent "
                             "each kernel's own duration covers the time it shares the GPU",
                "other_direction": {"dir": other, "ms": round(mb, 4), "includes": "k_source_sum_vec",
                                    "frac": round(ab[other] / (mb / 1e3) / 1e9 / peak, 4)}}

    # ---- the plain form on the same B300: directional sweeping of the same operator, the
    # same right-hand sides per source (R = 64, FP32), timed with CUDA events around whole
    # solves (each cycle ends with the stopping test's device-to-host read)
    sweep = None
    if not args.no_sweep:
        q = torch.randn((S, N, R), device=dev, dtype=dtype, generator=gen)
        xs = torch.empty_like(q)
        so = eik.default_opts(sweep_tol=args.sweep_tol)
        tan.sweep(q, transpose=False, opts=so, out=xs)       # builds the slotted weights and the cycle graph
        tan.sweep(q, transpose=True, opts=so, out=xs)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        _, c1 = tan.sweep(q, transpose=False, opts=so, out=xs)
        ev[1].record(stream)
        _, c2 = tan.sweep(q, transpose=True, opts=so, out=xs)
        ev[2].record(stream)
        torch.cuda.synchronize()
        tf, tb = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        sweep_value = 2.0 * N * S * R / ((tf + tb) / 1e3)
        sweep = {"value": sweep_value, "unit": UNIT, "cycles": [c1, c2], "R": R, "tol": args.sweep_tol,
                 "ms": [round(tf, 3), round(tb, 3)], "ms_per_cycle": [round(tf / c1, 3), round(tb / c2, 3)],
                 "visits_per_update": (1 << g.ndim) * (c1 + c2) / 2.0,
                 "speedup_btf_over_sweep": round(value / sweep_value, 1)}
        del q, xs
        torch.cuda.empty_cache()

    cpu = None if args.no_cpu else cpu_baseline(wl, args.cpu_sample_sources)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64blocks",
        "data": "synthetic (seeded recipe of the 3-D tomography-scale config; no public dataset)",
        "config": {"workload": workload, "grid": list(g.n), "nodes": N, "sources_per_gpu": S, "rhs": R,
                   "receivers": n_rec, "precision": "FP32 substitution, FP64 SCC blocks",
                   "schedule": schedule, "autotuned": tuned,
                   "directions": "J p and J^T y concurrently on two streams (split_dirs)" if concurrent else "in order",
                   "waits": "levels" if args.level_waits else "items", "l2": "inputs larger than L2 (dT/lam 3.3 GB per direction)",
                   "parallelism": f"source-sharded x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": upd_step / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(e2e_ms, 4),
                "copies": "every step: p and y from pinned host memory, d_rec and g back; double-buffered on two "
                          "copy streams, overlapping the neighbouring steps' traversals"},
        "gpu_launches": args.steps * (3 if schedule in ("persistent", "cluster", "sync") else (2 * max(x["levels"] for x in st) + 3)),
        "clocks": clocks,
        "sweep_baseline": sweep,
        "setup": {"eik_forward_s": round(t_state, 3), "eik_cycles": cyc, "tangent_build_s": round(t_setup, 3),
                  "levels_max": max(x["levels"] for x in st), "nontrivial_scc": sum(x["nontrivial"] for x in st),
                  "largest_scc": max(x["largest"] for x in st), "edges_per_node": sum(x["edges"] for x in st) / (S * N)},
        "kernel_ms": {"fwd": round(mf, 4), "bwd": round(mb, 4)},
    }
    tan.free()
    if not args.no_extras and world == 1:
        # the other workloads of this path, recorded on the same line (setup times and the
        # stress grids are not part of the headline value)
        del p, y, d_rec, gvec, p_h, y_h, drec_h, g_h, p_ds, y_ds, drec_ds, g_ds
        torch.cuda.empty_cache()
        for key, fn in (("gauss_newton_iteration_config4", gauss_newton_iteration_config4),
                        ("stress_config5", lambda: stress_config5(check_oracle=not args.no_cpu))):
            try:
                out[key] = fn()
            except Exception as e:   # an extra never takes the headline line down with it
                out[key] = {"error": f"{type(e).__name__}: {e}"[:300]}
            torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_lsqr(args):
    """Config 4: 201 x 201 x 101 grid, 64 sources, 2500 receivers, one right-hand side;
    20 LSQR iterations on J with every iteration replayed from a CUDA graph.  Prints one
    JSON line (paired node-updates/s of the Krylov loop, setup times)."""
    import torch

    from paper_2609_14982_b300 import eik
    from paper_2609_14982_b300 import workloads as W
    torch.cuda.set_device(0)
    wl = W.config4()
    g = wl.grid
    src = wl.src if args.sources <= 0 else wl.src[:args.sources]
    S, N = len(src), g.N
    dg = eik.DeviceGrid(g)
    s = torch.tensor(wl.s, device="cuda")
    t0 = time.time()
    # setup only: the state solve uses FP32 arithmetic away from the sources
    T, cyc = eik.eik_forward(dg, s, src, opts=eik.default_opts(eik_fp32=1))
    torch.cuda.synchronize()
    t_state = time.time() - t0
    t0 = time.time()
    # one right-hand side per Krylov step: 256-position items (one pass of 256 threads)
    tan = eik.Tangent(dg, T, s, src, rec=wl.rec, opts=eik.default_opts(chunk=KRYLOV_CHUNK, item_slots=KRYLOV_SLOTS))
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    del T
    st = [tan.stats(a) for a in range(S)]
    dtype = torch.float64 if args.lsqr_dtype == "f64" else torch.float32
    b = torch.randn((S, len(wl.rec)), device="cuda", dtype=dtype, generator=torch.Generator("cuda").manual_seed(20264))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        L = eik.LSQR(tan, dtype=dtype)
        L.start(b)
        L.iterate(1, use_graph=True)           # capture + first replay
        L.start(b)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.iterate(20, use_graph=True)
        e1.record(stream)
        stream.synchronize()
        x, sc = L.solution()
    tan.status()
    ms = e0.elapsed_time(e1) / 20
    upd = 2.0 * N * S
    out = {"metric": METRIC, "value": upd / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 20, "warmup": 1,
           "ms_per_step": ms, "higher_is_better": True, "dtype": args.lsqr_dtype,
           "config": {"workload": f"3d-201x201x101-S{S}-lsqr20 (config: Gauss-Newton inner solve)", "nodes": N,
                      "sources": S, "receivers": len(wl.rec), "step": "one LSQR iteration (J v, J^T u, vector ops), CUDA graph"},
           "lsqr": {"phibar": sc["phibar"], "iterations": 20},
           "setup": {"eik_forward_s": round(t_state, 2), "eik_cycles": cyc, "tangent_build_s": round(t_setup, 2),
                     "levels_max": max(x["levels"] for x in st), "nontrivial_scc": sum(x["nontrivial"] for x in st),
                     "largest_scc": max(x["largest"] for x in st)}}
    print(json.dumps(out), flush=True)
    L.free()
    tan.free()


def run_gn(args):
    """Config 4 grid (201 x 201 x 101, 64 sources, 2500 receivers) as the Gauss-Newton
    inner solve of Sec. 4.5: LSMR on K = [W_d J; lam R; lam S_k] with the paper's settings
    (nodal velocity model; W_d = 1 / sigma, sigma = 0.3 ms floor and 0.3 % of the
    traveltime in quadrature; lam = 0.01, gamma = 0.1; stop at |K^T r| <= 1e-4 |K| |r|).
    Times 20 graph-replayed iterations; reports the iterations the stopping rule needed."""
    import torch

    from paper_2609_14982_b300 import eik
    from paper_2609_14982_b300 import workloads as W
    torch.cuda.set_device(0)
    wl = W.config4()
    g = wl.grid
    src = wl.src if args.sources <= 0 else wl.src[:args.sources]
    S, N = len(src), g.N
    dg = eik.DeviceGrid(g)
    s = torch.tensor(wl.s, device="cuda")
    t0 = time.time()
    T, cyc = eik.eik_forward(dg, s, src, opts=eik.default_opts(eik_fp32=1))
    torch.cuda.synchronize()
    t_state = time.time() - t0
    t0 = time.time()
    tan = eik.Tangent(dg, T, s, src, rec=wl.rec, opts=eik.default_opts(model=eik.MODEL_VELOCITY, chunk=KRYLOV_CHUNK,
                                                                                     item_slots=KRYLOV_SLOTS))
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    rec = torch.as_tensor(np.asarray(wl.rec, dtype=np.int64), device="cuda")
    d = T[:, rec]                                       # predicted traveltimes [S, n_rec]
    del T
    sigma = torch.sqrt(3e-4 ** 2 + (3e-3 * d) ** 2)
    wd = (1.0 / sigma).contiguous()
    gen = torch.Generator("cuda").manual_seed(20265)
    r = sigma * torch.randn(d.shape, device="cuda", dtype=torch.float64, generator=gen)
    dtype = torch.float64 if args.lsqr_dtype == "f64" else torch.float32
    if args.cells:
        # cell velocities: the mean of each hexahedron's corner-node velocities
        v = (1.0 / s).reshape(g.n)
        vc = sum(v[i:i + g.n[0] - 1, j:j + g.n[1] - 1, k:k + g.n[2] - 1]
                 for i in (0, 1) for j in (0, 1) for k in (0, 1)) / 8.0
        vmodel = vc.contiguous().reshape(-1)
    else:
        vmodel = (1.0 / s).contiguous()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gn = eik.GN(tan, wd, vmodel, 0.01, 0.1, dtype=dtype, cells=args.cells)
        b = gn.rhs(r)
        gn.start(b)
        gn.iterate(1, use_graph=True)           # capture + first replay
        gn.start(b)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gn.iterate(20, use_graph=True)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / 20
        _, sc = gn.lsmr(b, atol=1e-4, max_iters=args.gn_max_iters, check_every=5)
    tan.status()
    upd = 2.0 * N * S
    out = {"metric": METRIC, "value": upd / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 20, "warmup": 1,
           "ms_per_step": ms, "higher_is_better": True, "dtype": args.lsqr_dtype,
           "config": {"workload": f"3d-201x201x101-S{S}-lsmr{'-cells' if args.cells else ''} (Gauss-Newton inner solve, Sec. 4.5)",
                      "nodes": N, "model": "cells" if args.cells else "nodes", "model_size": gn.n_model,
                      "sources": S, "receivers": len(wl.rec), "rows": gn.n_rows, "lambda": 0.01, "gamma": 0.1,
                      "step": "one LSMR iteration on K (J v, J^T u, W_d / R / S_k epilogues), CUDA graph"},
           "lsmr": {"iterations_to_atol_1e-4": int(sc["iters"]), "normr": sc["normr"], "normar": sc["normar"],
                    "norma": sc["norma"], "converged": sc["normar"] <= 1e-4 * sc["norma"] * sc["normr"]},
           "setup": {"eik_forward_s": round(t_state, 2), "eik_cycles": cyc, "tangent_build_s": round(t_setup, 2)}}
    print(json.dumps(out), flush=True)
    gn.free()
    tan.free()


def stress_config5(steps: int = 3, check_oracle: bool = True, sweep: bool = True) -> dict:
    """Config 5, the uneven-batch stress case: three steep-hill grids (slopes up to about
    55 deg) -- 101x101x51 (32 sources, R = 8), 161x121x61 (32, R = 32), 201x201x101 (64,
    R = 128) -- traversed together: J p of all three grids in ONE persistent launch (the
    work items of all three in one merged step-major order, two items held per CTA) and
    J^T y (summed over sources) in one more (tangent_apply_batch), with every tangent's
    workspace holding all its right-hand sides.  Per grid: the error of J p and
    J^T y against the FP64 oracle on a sampled source and four columns (the oracle builds
    its tangent from the same state), and the node-updates/s of BTF against GPU
    directional sweeping on a 4-source slice of the grid at R = min(R, 32)."""
    import torch

    from paper_2609_14982_b300 import eik
    from paper_2609_14982_b300 import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    tans, ps, ys, info, wls, states = [], [], [], [], [], []
    t0 = time.time()
    for w in range(3):
        wl = W.config5_grid(w)
        g = wl.grid
        dg = eik.DeviceGrid(g, device=dev)
        s = torch.tensor(wl.s, device=dev)
        ts = time.time()
        T, cyc = eik.eik_forward(dg, s, wl.src, opts=eik.default_opts(eik_fp32=1))
        torch.cuda.synchronize()
        t_state = time.time() - ts
        tb = time.time()
        tan = eik.Tangent(dg, T, s, wl.src, rec=wl.rec)
        torch.cuda.synchronize()
        t_build = time.time() - tb
        st = [tan.stats(a) for a in range(wl.S)]
        states.append((dg, s, T[:4].clone(), T[0].cpu().numpy()))
        del T
        gen = torch.Generator(dev).manual_seed(wl.seed)
        ps.append(torch.randn((g.N, wl.R), device=dev, generator=gen))
        ys.append(torch.randn((wl.S, len(wl.rec), wl.R), device=dev, generator=gen))
        tans.append(tan)
        wls.append(wl)
        info.append({"grid": list(g.n), "nodes": g.N, "sources": wl.S, "rhs": wl.R, "receivers": len(wl.rec),
                     "max_slope_deg": round(wl.notes.get("max_slope_deg", 0.0), 1),
                     "levels_max": max(x["levels"] for x in st), "nontrivial_scc": sum(x["nontrivial"] for x in st),
                     "largest_scc": max(x["largest"] for x in st), "eik_forward_s": round(t_state, 2),
                     "eik_cycles": cyc, "tangent_build_s": round(t_build, 2)})
    # largest grid first: clusters take its (longest) sources first
    order = [2, 1, 0]
    bt = [tans[k] for k in order]
    bp = [ps[k] for k in order]
    by = [ys[k] for k in order]
    eik.apply_batch(bt, bp)
    eik.apply_T_batch(bt, by)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1, e2 in ev:
        e0.record(stream)
        eik.apply_batch(bt, bp)
        e1.record(stream)
        eik.apply_T_batch(bt, by)
        e2.record(stream)
    torch.cuda.synchronize()
    for t in tans:
        t.status()
    tf = statistics.median(a.elapsed_time(b) for a, b, _ in ev)
    tbk = statistics.median(b.elapsed_time(c) for _, b, c in ev)
    upd = sum(2.0 * t.N * t.S * wl.R for t, wl in zip(tans, wls))
    out = {"workload": "3d-stress: 101x101x51 S32 R8 + 161x121x61 S32 R32 + 201x201x101 S64 R128",
           "launch": "one persistent launch per direction for all three grids (tangent_apply_batch: merged "
                     "step-major item order, two items held per CTA)",
           "value": upd / ((tf + tbk) / 1e3), "unit": UNIT, "ms_fwd": round(tf, 3), "ms_bwd": round(tbk, 3),
           "grids": info}
    jp_all = eik.apply_batch(bt, bp)
    torch.cuda.synchronize()
    for k, w in enumerate(order):
        tan, wl, (dg, s, T4, T0h) = tans[w], wls[w], states[w]
        g = wl.grid
        cols = [0, wl.R // 3, (2 * wl.R) // 3, wl.R - 1]
        if check_oracle:
            import oracle as O
            _, G, _ = O.metric(g)
            ot = O.build_tangent(g, G, T0h, wl.s, int(wl.src[0]))
            pn = ps[w][:, cols].double().cpu().numpy()
            ref = O.J([ot], wl.s, wl.rec, pn)[0]
            got = jp_all[k][0][:, cols].double().cpu().numpy()
            e_j = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
            # J^T of source 0 alone: data only on source 0, the source sum is then J_0^T y_0
            y0 = torch.zeros((wl.S, len(wl.rec), 4), device=dev)
            y0[0] = ys[w][0][:, cols]
            g0, _ = tan.apply_T(y0.contiguous(), sum_sources=True)
            refT = O.JT([ot], wl.s, wl.rec, y0[:1].double().cpu().numpy())
            e_t = float(np.max(np.abs(g0.double().cpu().numpy() - refT)) / np.max(np.abs(refT)))
            info[w]["err_vs_oracle"] = {"J": e_j, "JT": e_t, "source": 0, "columns": cols}
        if sweep:
            Rs = min(wl.R, 32)
            small = eik.Tangent(dg, T4, s, wl.src[:4], rec=wl.rec)
            q = torch.randn((4, g.N, Rs), device=dev, generator=torch.Generator(dev).manual_seed(wl.seed + 1))
            xb = torch.empty_like(q)
            so = eik.default_opts(sweep_tol=1e-6)
            small.solve(q, out=xb); small.solve_T(q, out=xb)
            small.sweep(q, transpose=False, opts=so, out=xb); small.sweep(q, transpose=True, opts=so, out=xb)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            e[0].record(stream)
            small.solve(q, out=xb)
            small.solve_T(q, out=xb)
            e[1].record(stream)
            _, c1 = small.sweep(q, transpose=False, opts=so, out=xb)
            e[2].record(stream)
            _, c2 = small.sweep(q, transpose=True, opts=so, out=xb)
            e[3].record(stream)
            torch.cuda.synchronize()
            small.status()
            n_upd = 2.0 * 4 * g.N * Rs
            t_btf, t_sw = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[3])
            info[w]["sweep_vs_btf"] = {"sources": 4, "R": Rs, "tol": 1e-6, "cycles": [c1, c2],
                                       "btf_node_updates_per_s": n_upd / (t_btf / 1e3),
                                       "sweep_node_updates_per_s": n_upd / (t_sw / 1e3),
                                       "btf_over_sweep": round(t_sw / t_btf, 1)}
            small.free()
            del q, xb
    for t in tans:
        t.free()
    del tans, ps, ys, jp_all, states
    torch.cuda.empty_cache()
    out["total_s"] = round(time.time() - t0, 1)
    return out


def gauss_newton_iteration_config4(lsqr_iters: int = 20) -> dict:
    """One outer Gauss-Newton iteration of Alg. 1 on the 201x201x101 grid (64 sources, 2500
    receivers): Phase I (state solve with the FP32 far field, tangent_build) and the inner
    solve of 20 LSQR iterations on J (FP64 vectors, every iteration replayed from a CUDA
    graph).  Reports each part and the total."""
    import torch

    from paper_2609_14982_b300 import eik
    from paper_2609_14982_b300 import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = W.config4()
    g = wl.grid
    dg = eik.DeviceGrid(g, device=dev)
    s = torch.tensor(wl.s, device=dev)
    b = torch.randn((wl.S, len(wl.rec)), device=dev, dtype=torch.float64,
                    generator=torch.Generator(dev).manual_seed(20264))
    # module load and first allocations outside the timed iteration
    eik.eik_forward(dg, s, wl.src[:1], opts=eik.default_opts(eik_fp32=1, eik_max_cycles=4000))
    torch.cuda.synchronize()
    t0 = time.time()
    T, cyc = eik.eik_forward(dg, s, wl.src, opts=eik.default_opts(eik_fp32=1))
    torch.cuda.synchronize()
    t1 = time.time()
    tan = eik.Tangent(dg, T, s, wl.src, rec=wl.rec, opts=eik.default_opts(chunk=KRYLOV_CHUNK, item_slots=KRYLOV_SLOTS))
    torch.cuda.synchronize()
    t2 = time.time()
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        L = eik.LSQR(tan, dtype=torch.float64)
        L.start(b)
        L.iterate(lsqr_iters, use_graph=True)
        x, sc = L.solution()
    side.synchronize()
    t3 = time.time()
    # the same iterations once more, graph already captured: the steady-state cost
    with torch.cuda.stream(side):
        L.start(b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        L.iterate(lsqr_iters, use_graph=True)
        e1.record(side)
    side.synchronize()
    tan.status()
    ms_iter = e0.elapsed_time(e1) / lsqr_iters
    L.free()
    tan.free()
    # the next outer iteration: the model takes the LSQR direction as a 1 % step (largest
    # change 1 % of the smallest slowness), and Phase I is redone -- the state solve warm
    # started from this iteration's traveltimes, a new tangent, 20 LSQR iterations
    s2 = s + x * (0.01 * float(s.min()) / float(x.abs().max()))
    torch.cuda.synchronize()
    u0 = time.time()
    T2, cyc2 = eik.eik_forward(dg, s2, wl.src, opts=eik.default_opts(eik_fp32=1), T_init=T)
    torch.cuda.synchronize()
    u1 = time.time()
    del T
    tan = eik.Tangent(dg, T2, s2, wl.src, rec=wl.rec, opts=eik.default_opts(chunk=KRYLOV_CHUNK, item_slots=KRYLOV_SLOTS))
    torch.cuda.synchronize()
    u2 = time.time()
    del T2
    with torch.cuda.stream(side):
        L = eik.LSQR(tan, dtype=torch.float64)
        L.start(b)
        L.iterate(lsqr_iters, use_graph=True)
        _, sc2 = L.solution()
    side.synchronize()
    u3 = time.time()
    tan.status()
    L.free()
    tan.free()
    torch.cuda.empty_cache()
    return {"workload": "3d-201x201x101-S64, 2500 receivers: state + tangent_build + 20 LSQR iterations",
            "eik_forward_s": round(t1 - t0, 3), "eik_cycles": cyc, "tangent_build_s": round(t2 - t1, 3),
            "lsqr_first_20_s": round(t3 - t2, 3), "lsqr_ms_per_iteration": round(ms_iter, 3),
            "iteration_total_s": round(t3 - t0, 3), "lsqr_phibar": sc["phibar"],
            "source_nodes_per_s_build": wl.S * g.N / (t2 - t1),
            "next_iteration": {"model_step": "LSQR direction scaled to 1 % of the smallest slowness",
                               "eik_forward_warm_s": round(u1 - u0, 3), "eik_cycles": cyc2,
                               "tangent_build_s": round(u2 - u1, 3), "lsqr_20_s": round(u3 - u2, 3),
                               "iteration_total_s": round(u3 - u0, 3)}}


def run_stress(args):
    """Config 5 alone as one JSON line (see stress_config5)."""
    import torch
    torch.cuda.set_device(0)
    r = stress_config5(steps=max(args.steps // 2, 3), check_oracle=not args.no_cpu, sweep=not args.no_sweep)
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": max(args.steps // 2, 3),
           "warmup": 1, "ms_per_step": r["ms_fwd"] + r["ms_bwd"], "higher_is_better": True,
           "dtype": "f32+f64blocks", "data": "synthetic (seeded steep-hill recipe; no public dataset)",
           "config": {"workload": r["workload"], "launch": r["launch"], "grids": r["grids"]}}
    print(json.dumps(out), flush=True)


def run_state(args):
    """Phase I state solve alone (Sec. 2.1-2.2 reading: factored full-metric LF sweeping):
    the 3-D apply workload (101x101x51, 25 sources) in FP64 and with the FP32 far field,
    and the 201x201x101 grid with 64 sources (FP32 far field).  Reports seconds, cycles
    and node-updates/s (sources x interior nodes x 2^D orderings x cycles per second)."""
    import torch

    from paper_2609_14982_b300 import eik
    from paper_2609_14982_b300 import workloads as W
    torch.cuda.set_device(0)
    rows = []
    runs = ((W.config3(), 0), (W.config3(), 1), (W.config4(), 1))
    if args.state_cycles > 0:
        runs = runs[1:2]     # a short profiling case: the 3-D apply grid, FP32 far field, a few cycles
    for wl, fp32 in runs:
        g = wl.grid
        dg = eik.DeviceGrid(g)
        s = torch.tensor(wl.s, device="cuda")
        if args.state_cycles <= 0:
            eik.eik_forward(dg, s, wl.src[:1], opts=eik.default_opts(eik_fp32=fp32))   # warm-up (module load)
        torch.cuda.synchronize()
        t0 = time.time()
        if args.state_cycles > 0:
            try:
                eik.eik_forward(dg, s, wl.src, opts=eik.default_opts(eik_fp32=fp32, eik_max_cycles=args.state_cycles))
            except eik.EikError as e:
                if e.code != -4:      # EIK_ERR_NOT_CONVERGED is expected after so few cycles
                    raise
            torch.cuda.synchronize()
            rows.append({"grid": list(g.n), "sources": wl.S, "cycles": args.state_cycles,
                         "seconds": round(time.time() - t0, 3)})
            continue
        T, cyc = eik.eik_forward(dg, s, wl.src, opts=eik.default_opts(eik_fp32=fp32))
        torch.cuda.synchronize()
        sec = time.time() - t0
        interior = int(np.prod([m - 2 for m in g.n[:g.ndim]]))
        upd = float(wl.S) * interior * (1 << g.ndim) * cyc
        rows.append({"grid": list(g.n), "sources": wl.S, "fp32_far_field": bool(fp32), "seconds": round(sec, 3),
                     "cycles": cyc, "node_updates_per_s": upd / sec})
        del T
    if args.state_cycles > 0:
        print(json.dumps({"workload": "state solve, profiling case", "runs": rows}), flush=True)
        return
    out = {"metric": "eik_forward node-updates/s (LF sweeping, all sources)", "value": rows[-1]["node_updates_per_s"],
           "unit": "node-updates/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": rows[-1]["seconds"] * 1e3,
           "higher_is_better": True, "dtype": "f64 (f32 far field where marked)", "data": "synthetic",
           "config": {"workload": "state solve: 3d-101x101x51-S25 (f64, f32 far) + 3d-201x201x101-S64 (f32 far)",
                      "runs": rows}}
    print(json.dumps(out), flush=True)


def run_tables(args):
    """The paper's structure-stress grids (Sec. 5.2.2, Table 3 refinement of case C: the
    curved-surface map with A = 500 m, eps_T = 0.05, quarter source), one source each:
    tangent_build time, SCC statistics, and J p + J^T y node-updates/s at R = 64 (FP32)."""
    import torch

    from paper_2609_14982_b300 import eik
    from paper_2609_14982_b300 import workloads as W
    torch.cuda.set_device(0)
    rows, tot_upd, tot_ms = [], 0.0, 0.0
    for n in ((21, 21, 13), (41, 41, 25), (61, 61, 37), (81, 81, 49)):
        g = W.graph_grid(n, 500.0)
        src = W.quarter_source(g)
        st = W.curved_state(g, src, 0.05)
        dg = eik.DeviceGrid(g)
        T = torch.tensor(st.T[None], device="cuda")
        s = torch.tensor(st.s, device="cuda")
        rec = np.array([g.index(i, j, 0) for i in range(0, n[0], 4) for j in range(0, n[1], 4)], dtype=np.int32)
        eik.Tangent(dg, T, s, [src], rec=rec).free()          # warm-up (module load, first allocations)
        torch.cuda.synchronize()
        t0 = time.time()
        tan = eik.Tangent(dg, T, s, [src], rec=rec)
        torch.cuda.synchronize()
        t_build = time.time() - t0
        x = tan.stats(0)
        gen = torch.Generator("cuda").manual_seed(5)
        p = torch.randn((g.N, 64), device="cuda", generator=gen)
        y = torch.randn((1, len(rec), 64), device="cuda", generator=gen)
        for _ in range(3):
            tan.apply(p, shared_model=True)
            tan.apply_T(y, sum_sources=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            tan.apply(p, shared_model=True)
            tan.apply_T(y, sum_sources=True)
        e1.record()
        torch.cuda.synchronize()
        tan.status()
        ms = e0.elapsed_time(e1) / 10
        upd = 2.0 * g.N * 64
        tot_upd += upd
        tot_ms += ms
        rows.append({"grid": list(n), "nodes": g.N, "nontrivial_scc": x["nontrivial"], "cyclic_nodes": x["cyclic_nodes"],
                     "largest_scc": x["largest"], "levels": x["levels"], "tangent_build_ms": round(t_build * 1e3, 2),
                     "apply_pair_ms": round(ms, 3), "node_updates_per_s": upd / (ms / 1e3)})
        tan.free()
    out = {"metric": METRIC, "value": tot_upd / (tot_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 10, "warmup": 3,
           "ms_per_step": tot_ms, "higher_is_better": True, "dtype": "f32+f64blocks", "data": "synthetic",
           "config": {"workload": "Table 3 grids (case C, one source, R 64)", "grids": rows}}
    print(json.dumps(out), flush=True)


def host_info() -> dict:
    """The host the oracle is timed on: its hardware threads and CPU model."""
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"host_threads": os.cpu_count(), "cpu_model": model}


def cpu_baseline(wl, n_src: int, R: int = 32) -> dict:
    """The CPU oracle as it stands (single-threaded C, FP64 block traversal) on a bounded
    sample of the workload: `n_src` sources (their states from the oracle's own state
    solve), R right-hand sides each, one J and one J^T solve per right-hand side."""
    import oracle as O
    g = wl.grid
    _, G, _ = O.metric(g)
    rng = np.random.default_rng(7)
    t_apply = 0.0
    upd = 0
    for a in range(n_src):
        k = int(wl.src[(a * 7) % len(wl.src)])
        T, _ = O.eik_forward(g, wl.s, k)
        t = O.build_tangent(g, G, T, wl.s, k)
        q = rng.standard_normal((g.N, R))
        t0 = time.perf_counter()
        for r in range(R):
            O.solve(t, q[:, r])
            O.solve_T(t, q[:, r])
        t_apply += time.perf_counter() - t0
        upd += 2 * g.N * R
    return {"value": upd / t_apply, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_src} sources x {R} RHS of the full grid, J and J^T solves, FP64, {t_apply:.1f} s timed",
            **host_info()}


def run_reference(args):
    """The reference arm: the CPU oracle timed on the host, same metric and workload,
    each step a bounded sample (one source, a few right-hand sides)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2609_14982_b300 import workloads as W
    wl = W.config3()
    g = wl.grid
    _, G, _ = O.metric(g)
    k = int(wl.src[12])
    T, _ = O.eik_forward(g, wl.s, k)
    t = O.build_tangent(g, G, T, wl.s, k)
    rng = np.random.default_rng(3)
    Rs = 8
    q = rng.standard_normal((g.N, Rs))

    def step():
        for r in range(Rs):
            O.solve(t, q[:, r])
            O.solve_T(t, q[:, r])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = 2 * g.N * Rs / dt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": f"1 source x {Rs} RHS per step"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"1 source x {Rs} RHS, J and J^T solves per step", **host_info()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--schedule", choices=["persistent", "levels", "staged", "cluster", "sync"], default="persistent")
    ap.add_argument("--state-cycles", type=int, default=0,
                    help="--workload state: only the 3-D apply grid (FP32 far field) for this many cycles (profiling)")
    ap.add_argument("--split-dirs", action="store_true",
                    help="run J p and J^T y of a step at once on two streams (2 CTAs per SM each unless given)")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="pick the traversal setting by timing a short candidate list before the timed region")
    ap.add_argument("--cluster-size", type=int, default=0, help="cluster schedule: CTAs per cluster (0 = auto)")
    ap.add_argument("--cluster-threads", type=int, default=0, help="cluster schedule: threads per CTA (0 = 256)")
    ap.add_argument("--pass-units", type=int, default=0, help="cluster schedule: units per thread per round (2 or 4)")
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--item-slots", type=int, default=0, help="persistent schedule: work items held per CTA (2..4)")
    ap.add_argument("--chunk", type=int, default=0, help="positions per work item (default: the library's, 64)")
    ap.add_argument("--level-waits", action="store_true",
                    help="persistent items wait for their whole previous level, not only their upstream items")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the Gauss-Newton iteration and the three-grid stress batch on the headline line")
    ap.add_argument("--sweep-tol", type=float, default=1e-6,
                    help="sweeping baseline: stop at max |dx| <= tol max |x| over a cycle (FP32 path)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-sources", type=int, default=2)
    ap.add_argument("--sources", type=int, default=0, help="use only the first K sources (small profiling case)")
    ap.add_argument("--state-cache", default="", help="load/save the solved states (.npy) to skip the state solve")
    ap.add_argument("--gn-max-iters", type=int, default=300)
    ap.add_argument("--cells", action="store_true", help="gn workload: the model on the grid cells")
    ap.add_argument("--workload", choices=["apply", "lsqr", "gn", "stress", "state", "tables"], default="apply",
                    help="apply: the benchmark line (3-D apply config); lsqr: the 20-iteration Krylov config; "
                         "gn: LSMR on the augmented Gauss-Newton operator (Sec. 4.5); "
                         "stress: the three steep-hill grids with right-hand-side chunking; "
                         "state: the state solve alone; tables: the paper's Table 3 grids")
    ap.add_argument("--lsqr-dtype", choices=["f64", "f32"], default="f64")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "lsqr":
        run_lsqr(args)
    elif args.workload == "gn":
        run_gn(args)
    elif args.workload == "stress":
        run_stress(args)
    elif args.workload == "state":
        run_state(args)
    elif args.workload == "tables":
        run_tables(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark: candidate pairs refined per second on the pathology-shaped join.

Workload (one step = the join's whole query path over one batch): A = 10,000
nucleus meshes (noisy icospheres, level 4/5, 5,120-20,480 triangles), B = 500
vessel meshes (16-sided capped tubes along cubic B-splines, 10k-50k
triangles), one unit cube on the 2^18 grid.  Per step: the device bounding-box
filter join produces the candidate pairs, every candidate is refined
(bidirectional edge piercing with early exit, then +z parity containment) and
the intersecting pairs are compacted.  Meshes and their BVHs are resident
(loading and BVH build are reported separately, as in the paper's measurement
of query time).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate pairs refined/s & segment–tri tests/s; p50/p99 query latency"
FRONT_LEVELS = {"stream": -2, "wave": 14, "none": -1}   # front end -> pj_join_opts.wave_levels
UNIT = "pairs/s"
WORKLOAD = ("pathology join: 10,000 nuclei (icosphere L4/L5, 10% smooth radial noise, "
            "log-normal radius mean 1/200 box) x 500 vessels (16-sided capped tubes on cubic "
            "B-splines, 10k-50k triangles, radius 1/300-1/100 box), 2^18 grid, float32, "
            "intersects predicate, candidates from the device bounding-box join")


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(ms_step: float, units: int, dist, device: str):
    """Whole-job numbers: the slowest rank's step time and the units (candidate
    pairs) all ranks processed per step.  No collective touches the data path;
    this is the only one, after the timed region."""
    if dist is None:
        return ms_step, units
    import torch
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.int64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def make_workload(seed: int, n_nuclei: int = 10000, n_vessels: int = 500):
    from paper_2609_24513_gb300 import synth
    return synth.pathology(seed, n_nuclei, n_vessels)


def profile_traffic(kernel: str, kernel_src: str):
    """DRAM bytes per launch of `kernel` on the pathology workload from the
    committed ncu summary profiles/<kernel>_pathology.md, if that summary was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "%s_pathology.md" % kernel)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"source sha1:\s*([0-9a-f]{12})", txt)
    t = re.search(r"dram bytes per full launch:\s*([0-9.eE+]+)", txt)
    if not m or not t:
        return None
    h = hashlib.sha1(open(kernel_src, "rb").read()).hexdigest()[:12]
    return float(t.group(1)) if h == m.group(1) else None


def cpu_baseline(A, B, cand, seconds: float, seed: int):
    """The oracle (tier 2) on bounded random samples: one thread, then the
    same per-pair code sharded over every host core.  The all-core figure is
    the line's value; `cores` is the number of threads it used."""
    import oracle
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(cand))
    done, tests, t0 = 0, 0, time.perf_counter()
    while done < len(order) and time.perf_counter() - t0 < seconds:
        blk = cand[order[done:done + 8]]
        _, st = oracle.join(A, B, blk, tier=2, stats=True)
        tests += int(st[0])
        done += len(blk)
    el = time.perf_counter() - t0
    single = {"value": done / el, "cores": 1, "segtri_tests_per_s": tests / el,
              "sample": "%d candidate pairs, %.1f s" % (done, el)}
    # all cores: a disjoint sample of (about) the same wall time
    cores = oracle.host_cores()
    n = min(len(order) - done, max(cores, int(single["value"] * cores * seconds)))
    sel = cand[order[done:done + n]]
    t0 = time.perf_counter()
    _, st = oracle.join(A, B, sel, tier=2, stats=True, threads=cores)
    el_all = time.perf_counter() - t0
    return {"value": len(sel) / el_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d candidate pairs drawn uniformly (seed %d), oracle tier 2 "
                      "(bounding-box-pruned brute force, exact int64) sharded over %d threads, "
                      "%.1f s" % (len(sel), len(cand), seed, cores, el_all),
            "segtri_tests_per_s": int(st[0]) / el_all,
            "single_core": single}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_2609_24513_gb300 import synth
    oracle.build()
    A, B = make_workload(args.seed, args.nuclei, args.vessels)
    cand = oracle.mbb_candidates(A, B)
    rng = np.random.default_rng(args.seed)
    cores = oracle.host_cores()
    # each timed step gets an equal share of the run's time budget (at most
    # --ref-step-s, at least 0.5 s): a sample of the candidates sized from
    # the per-core rate of a short single-threaded calibration, refined by
    # the same per-pair code sharded over every host core
    per_step = min(args.ref_step_s, max(0.5, args.ref_total_s / max(1, args.steps)))
    sel = cand[rng.permutation(len(cand))]
    t0, n = time.perf_counter(), 0
    while n < len(sel) and time.perf_counter() - t0 < 1.0:
        oracle.join(A, B, sel[n:n + 8], tier=2)
        n += len(sel[n:n + 8])
    rate1 = n / (time.perf_counter() - t0)
    times, counts = [], []
    for step in range(args.warmup + args.steps):
        sel = cand[rng.permutation(len(cand))]
        limit = per_step if step >= args.warmup else min(per_step, 0.5)
        m = int(min(len(sel), max(cores, rate1 * cores * limit)))
        t0 = time.perf_counter()
        oracle.join(A, B, sel[:m], tier=2, threads=cores)
        el = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(el)
            counts.append(m)
    value = sum(counts) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "candidates": int(len(cand)),
                       "step": "bounded sample of the candidates, %.1f s of oracle work" % per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d candidate pairs per step, uniform random, sharded "
                                       "over %d threads" % (int(np.mean(counts)), cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2609_24513_gb300 import pierce
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    t0 = time.perf_counter()
    A, B = make_workload(args.seed + 1000 * rank, args.nuclei, args.vessels)  # one per rank
    gen_s = time.perf_counter() - t0
    ctx = pierce.Context(local_rank)
    stream = torch.cuda.Stream()                     # every step and event on one stream
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    ha, hb = ctx.load(A), ctx.load(B)
    load_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx.build(ha, args.width, args.leaf)
    ctx.build(hb, args.width, args.leaf)
    build_s = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    opts = dict(width=args.width, leaf_size=args.leaf, warps_per_pair=args.warps,
                use_graph=args.graph, out_host=False, stream=stream,
                wave_levels=FRONT_LEVELS[args.front])

    def step():
        res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, **opts)
        info = (int(res.n_candidates), int(res.count), res.refine_ms)
        pierce.pj_free_pairs(ctx.h, res)
        return info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.reset_counters()
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, C, K = 0.0, 0, 0
    for _ in range(args.steps):
        flush.zero_()                                   # evict L2 between steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda.nvtx.range_push("step")          # lets a profiler pick the timed steps
        C, K, _ = step()
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    cnt = ctx.counters()
    ms_step, C_all = aggregate_ranks(total_ms / args.steps, C, dist, "cuda")
    value = C_all / (ms_step / 1000.0)
    segtri_s = cnt["segtri_tests"] / (total_ms / 1000.0)
    launches = cnt["kernel_launches"]
    # phase and kernel breakdown (same join, not replayed from a graph, with
    # CUDA events on the join's stream between the phases and around every
    # breadth-first launch)
    ctx.reset_counters()
    keys = ("mbb_ms", "parity_ms", "front_ms", "tasks_ms", "refine_ms", "compact_ms", "expand_ms",
            "leaf_ms", "device_ms")
    ph = {k: [] for k in keys}
    for _ in range(args.steps):
        flush.zero_()
        res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, **dict(opts, use_graph=False,
                                                                  kernel_times=True))
        for k in ph:
            ph[k].append(getattr(res, k))
        pierce.pj_free_pairs(ctx.h, res)
    torch.cuda.synchronize()
    pc = ctx.counters()
    phase_ms = {k: float(np.median(v)) for k, v in ph.items()}
    per_step = {k: pc[k] / args.steps for k in ("bytes_fetched", "bytes_parity", "bytes_expand",
                                                 "bytes_leaf", "bytes_tasks")}
    peak, peak_kind = measured_peaks()
    # kernel families of one step: (step ms, algorithmic bytes, launches)
    if args.front == "stream":
        # k_stream also takes the long parity rays (bytes_tasks)
        fam = {"k_stream": (phase_ms["front_ms"], per_step["bytes_expand"] + per_step["bytes_leaf"]
                            + per_step["bytes_tasks"], 1),
               "k_wave_parity": (phase_ms["parity_ms"],
                                 per_step["bytes_parity"] - per_step["bytes_tasks"], 1)}
    elif args.front == "wave":
        levels = FRONT_LEVELS["wave"]
        fam = {"k_wave_expand": (phase_ms["expand_ms"], per_step["bytes_expand"], levels),
               "k_wave_leaf": (phase_ms["leaf_ms"], per_step["bytes_leaf"], levels),
               "k_wave_parity+handover": (phase_ms["parity_ms"], per_step["bytes_parity"], 2),
               "k_refine_tasks": (phase_ms["tasks_ms"], per_step["bytes_tasks"], 3)}
    else:
        fam = {"k_refine+k_refine_tasks": (phase_ms["refine_ms"], per_step["bytes_fetched"], 3)}
    dom = max(fam, key=lambda k: fam[k][0])
    d_ms, d_bytes, d_launch = fam[dom]
    achieved = d_bytes / (max(d_ms, 1e-6) / 1000.0) / 1e9
    traffic = profile_traffic(dom, os.path.join(ROOT, "paper_2609_24513_gb300", "csrc",
                                                 "pj_join.cu"))
    kernels = {k: {"ms_per_step": round(v[0], 4), "launches_per_step": v[2],
                   "bytes_per_launch": v[1] / v[2],
                   "achieved_gbs": v[1] / (max(v[0], 1e-6) / 1000.0) / 1e9}
               for k, v in fam.items()}
    line_e2e = None
    cand_host = _candidates_host(ctx, ha, hb, C)
    if not args.no_e2e:
        line_e2e = _end_to_end(ctx, ha, hb, cand_host, args, flush, stream, dist, pierce)
    serving = None if args.no_serving else _serving_summary(ctx, pierce, ha, hb, args.seed)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "candidates_per_step": C, "pairs_per_step": K,
                       "bvh_width": args.width, "leaf_size": args.leaf,
                       "warps_per_pair": args.warps or 1, "cuda_graph": bool(args.graph),
                       "front_end": args.front,
                       "l2": "256 MB buffer written between timed steps",
                       "setup_s": {"generate": round(gen_s, 2), "load": round(load_s, 3),
                                   "bvh_build": round(build_s, 3)}},
            "segtri_tests_per_s": segtri_s,
            "exact_fallback_frac": cnt["exact_fallbacks"] / max(1, cnt["segtri_tests"]),
            "counters_per_step": {k: v / args.steps for k, v in cnt.items()},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": dom, "launches_per_step": d_launch,
                         "launch_ms": d_ms / d_launch, "bytes_per_launch": d_bytes / d_launch,
                         "peak_source": peak_kind, "kernels": kernels,
                         "refinement_phase": {
                             "ms": phase_ms["refine_ms"], "bytes": per_step["bytes_fetched"],
                             "achieved_gbs": per_step["bytes_fetched"] /
                             (phase_ms["refine_ms"] / 1000.0) / 1e9,
                             "parity_ms": phase_ms["parity_ms"], "front_ms": phase_ms["front_ms"],
                             "tasks_ms": phase_ms["tasks_ms"], "mbb_ms": phase_ms["mbb_ms"],
                             "compact_ms": phase_ms["compact_ms"],
                             "join_ms_not_replayed": phase_ms["device_ms"]}},
            "e2e": line_e2e,
            "clocks": clk}
    if serving:
        # the metric's latency part: window queries on the same resident
        # datasets at 2,000 queries/s (Poisson), submit to results on the host
        line["p50_ms"] = serving["poisson_2000qps"]["p50_ms"]
        line["p99_ms"] = serving["poisson_2000qps"]["p99_ms"]
        line["serving"] = serving
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A, B, cand_host, args.cpu_seconds, args.seed)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _end_to_end(ctx, ha, hb, cand_host, args, flush, stream, dist, pierce):
    """The same metric through the public call with host buffers: the
    candidate list comes from pinned host memory each step and the result
    pairs go back to host memory; wall-clock timed with a synchronize on both
    sides of every step."""
    import torch
    pinned = torch.from_numpy(cand_host).pin_memory()
    cand_np = pinned.numpy()
    e2e_t, e2e_k = 0.0, 0
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = pierce.pj_join_intersects_ex(ctx.h, ha, hb, cand=cand_np, width=args.width,
                                         leaf_size=args.leaf, warps_per_pair=args.warps,
                                         wave_levels=FRONT_LEVELS[args.front],
                                         out_host=True, stream=stream)
        pairs = pierce.pairs_to_numpy(r)
        pierce.pj_free_pairs(ctx.h, r)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_t += el
            e2e_k = len(pairs)
    e2e_ms, e2e_units = aggregate_ranks(1000.0 * e2e_t / args.steps, len(cand_np), dist, "cuda")
    return {"value": e2e_units / (e2e_ms / 1000.0), "unit": UNIT,
            "h2d_bytes_per_step": int(cand_np.nbytes), "d2h_bytes_per_step": int(8 * e2e_k + 8)}


def _serving_summary(ctx, pierce, ha, hb, seed, n_alone=200, n_poisson=1000, n_burst=800):
    """Window join queries through pj_submit / pj_poll on the resident
    datasets: one at a time, as Poisson streams at 1,000 and 2,000 queries/s
    (the windows run from a few meshes to the whole datasets, so 2,000/s is
    about 85 % of one-at-a-time capacity) and as a burst submitted at once (a
    saturating load, so that continuous batching forms batches); p50/p99
    latency, throughput and mean batch size of each, and whether every answer
    equals the same query served alone."""
    from paper_2609_24513_gb300 import synth
    lo, hi = synth.serving_windows(seed + 77, max(n_alone, n_poisson, n_burst))
    _serve_stream(ctx, pierce, ha, hb, lo[:64], hi[:64], np.zeros(64))   # warm-up
    alone_ans, alone_st = [], []
    t0 = time.perf_counter()
    for k in range(n_alone):
        a, st = ctx.poll(ctx.submit(ha, hb, lo[k], hi[k]), wait=True)
        alone_ans.append(a)
        alone_st.append(st)
    out = {"alone": _latency_summary(alone_st, time.perf_counter() - t0)}
    identical = True
    for name, n, arr in (("poisson_1000qps", n_poisson, synth.poisson_arrivals(seed + 103, 1000.0, n_poisson)),
                         ("poisson_2000qps", n_poisson, synth.poisson_arrivals(seed + 101, 2000.0, n_poisson)),
                         ("burst", n_burst, np.zeros(n_burst))):
        ans, st, span = _serve_stream(ctx, pierce, ha, hb, lo[:n], hi[:n], arr)
        for k in range(min(n, n_alone)):
            identical &= bool(np.array_equal(ans[k], alone_ans[k]))
        out[name] = _latency_summary(st, span)
    out["answers_identical_to_alone"] = identical
    out["burst_speedup_over_alone_qps"] = (out["burst"]["queries_per_s"] /
                                           out["alone"]["queries_per_s"])
    return out


def _candidates_host(ctx, ha, hb, n):
    """The bounding-box candidates as a host array (the end-to-end query input),
    from the mesh boxes the library computed at load time."""
    return _mbb_host(ctx, ha, hb, n)


def _mbb_host(ctx, ha, hb, n):
    from paper_2609_24513_gb300 import pierce
    aabb_a, _, _ = pierce.pj_export_mesh_data(ctx.h, ha, _nm(ctx, ha), _nt(ctx, ha))
    aabb_b, _, _ = pierce.pj_export_mesh_data(ctx.h, hb, _nm(ctx, hb), _nt(ctx, hb))
    out = []
    for i in range(len(aabb_a)):
        a = aabb_a[i]
        ok = np.all((a[:3] <= aabb_b[:, 3:]) & (aabb_b[:, :3] <= a[3:]), axis=1)
        js = np.nonzero(ok)[0]
        out.append(np.stack([np.full(len(js), i), js], axis=1))
    cand = np.concatenate(out).astype(np.int32)
    assert len(cand) == n
    return np.ascontiguousarray(cand)


def _nm(ctx, h):
    from paper_2609_24513_gb300 import pierce
    return pierce.pj_dataset_info_get(ctx.h, h)["n_meshes"]


def _nt(ctx, h):
    from paper_2609_24513_gb300 import pierce
    return pierce.pj_dataset_info_get(ctx.h, h)["n_tris"]


def _timed_joins(ctx, pierce, torch, ha, hb, steps, flush, **kw):
    """Median device time (ms) of `steps` joins after one warm-up, plus the
    last result's counts."""
    t, info = [], None
    for r in range(steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        e0.record(s)
        res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, stream=s, **kw)
        e1.record(s)
        e1.synchronize()
        info = (int(res.n_candidates), int(res.count))
        pierce.pj_free_pairs(ctx.h, res)
        if r > 0:
            t.append(e0.elapsed_time(e1))
    return float(np.median(t)), info


def run_batching(args):
    """Batching workload: 100,000 instanced candidate pairs with log-uniform
    face counts in [200, 50,000]; the autotuner picks (W, L, warps per pair)
    on a 2 % sample; the persistent graph-replayed join is compared with one
    launch per candidate."""
    import torch
    from paper_2609_24513_gb300 import pierce, synth
    torch.cuda.set_stream(torch.cuda.Stream())
    t0 = time.perf_counter()
    A, B, cand, off, cls = synth.batching(args.seed + 1000)
    gen_s = time.perf_counter() - t0
    ctx = pierce.Context(0)
    ha, hb = ctx.load(A), ctx.load(B)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    best, table = pierce.pj_autotune(ctx.h, ha, hb, cand=cand, widths=(2, 4, 8),
                                     leaf_sizes=(1, 2, 4, 8), warps=(1, 2, 4), wave_levels=(0,),
                                     sample_permille=20, repeats=3, seed=args.seed)
    tune_s = time.perf_counter() - t0
    kw = {k: best[k] for k in ("width", "leaf_size", "warps_per_pair", "wave_levels")}
    d_cand = torch.from_numpy(cand).cuda()
    d_off = torch.from_numpy(off).cuda()
    clocks = ClockSampler(0)
    clocks.start()
    ms, (C, K) = _timed_joins(ctx, pierce, torch, ha, hb, args.steps, flush, cand=d_cand,
                              cand_offsets=d_off, use_graph=True, out_host=False, **kw)
    clk = clocks.stop()
    ms_pp, (C2, K2) = _timed_joins(ctx, pierce, torch, ha, hb, 1, flush, cand=d_cand,
                                   cand_offsets=d_off, out_host=False,
                                   launch_mode=pierce.PJ_LAUNCH_PER_PAIR,
                                   width=kw["width"], leaf_size=kw["leaf_size"])
    assert (C2, K2) == (C, K)
    line = {"metric": METRIC, "value": C / (ms / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+int64", "data": "synthetic",
            "config": {"workload": "batching: 100,000 instanced candidate pairs, 2,000 + 2,000 "
                                   "template meshes (noisy spheres / swept tubes), faces "
                                   "log-uniform in [200, 50,000], placements 30 % crossing, "
                                   "10 % containment, 60 % disjoint with overlapping boxes",
                       "candidates": C, "pairs": K, "best": best,
                       "setup_s": {"generate": round(gen_s, 2), "autotune": round(tune_s, 2)}},
            "one_launch_per_pair": {"ms": ms_pp, "value": C / (ms_pp / 1000.0),
                                    "speedup_of_persistent": ms_pp / ms},
            "autotune_top": sorted(table, key=lambda r: r["ms"])[:8],
            "autotune_worst": sorted(table, key=lambda r: r["ms"])[-3:],
            "clocks": clk}
    ctx.close()
    print(json.dumps(line), flush=True)


def run_urban(args):
    """Urban precision stress: self join of 50,000 buildings plus 5,000 boxes
    and cylinders (5 % of buildings in exactly touching pairs); FP32-filtered
    leaves against all-int64 leaves, with the filter's fallback rate."""
    import torch
    from paper_2609_24513_gb300 import pierce, synth
    torch.cuda.set_stream(torch.cuda.Stream())
    t0 = time.perf_counter()
    U = synth.urban(args.seed + 3000)
    gen_s = time.perf_counter() - t0
    ctx = pierce.Context(0)
    h = ctx.load(U)
    ctx.build(h, args.width, args.leaf)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {}
    for name, mode in (("filtered", pierce.PJ_LEAF_FILTERED), ("int64", pierce.PJ_LEAF_EXACT)):
        ctx.reset_counters()
        ms, (C, K) = _timed_joins(ctx, pierce, torch, h, h, args.steps, flush, self_join=True,
                                  use_graph=True, out_host=False, leaf_mode=mode)
        c = ctx.counters()
        out[name] = {"ms": ms, "value": C / (ms / 1000.0), "pairs": K,
                     "segtri_tests_per_step": c["segtri_tests"] / (args.steps + 1),
                     "exact_fallbacks_per_step": c["exact_fallbacks"] / (args.steps + 1),
                     "fallback_rate": c["exact_fallbacks"] / max(1, c["segtri_tests"])}
    assert out["filtered"]["pairs"] == out["int64"]["pairs"]
    line = {"metric": METRIC, "value": out["filtered"]["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": out["filtered"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+int64", "data": "synthetic",
            "config": {"workload": "urban self join: 50,000 extruded star-shaped buildings "
                                   "(6-64 sides, pitched roofs, 100-2,000 faces) on a jittered "
                                   "grid, 5 % in exactly touching pairs, plus 5,000 boxes and "
                                   "cylinders", "candidates": C,
                       "meshes": int(U.nmesh), "triangles": int(len(U.tris)),
                       "generate_s": round(gen_s, 2)},
            "leaves": out}
    ctx.close()
    print(json.dumps(line), flush=True)


def _serve_stream(ctx, pierce, ha, hb, lo, hi, arrivals):
    """Submit query k at arrivals[k] seconds (a submitting thread) while this
    thread collects; returns (answers, stats, makespan seconds)."""
    n = len(lo)
    tickets = [None] * n
    ready = [threading.Event() for _ in range(n)]
    err = []

    def submitter():
        try:
            t0 = time.perf_counter()
            for k in range(n):
                d = arrivals[k] - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                tickets[k] = ctx.submit(ha, hb, lo[k], hi[k])
                ready[k].set()
        except Exception as e:  # reported by the collector
            err.append(e)
            for r in ready:
                r.set()

    th = threading.Thread(target=submitter)
    t_start = time.perf_counter()
    th.start()
    answers, stats = [None] * n, [None] * n
    for k in range(n):
        ready[k].wait()
        if err:
            break
        answers[k], stats[k] = ctx.poll(tickets[k], wait=True)
    th.join()
    if err:
        raise err[0]
    return answers, stats, time.perf_counter() - t_start


def _latency_summary(stats, makespan):
    lat = np.array([(s["t_done"] - s["t_submit"]) * 1000.0 for s in stats])
    qwait = np.array([(s["t_admit"] - s["t_submit"]) * 1000.0 for s in stats])
    pairs = sum(int(s["n_pairs"]) for s in stats)
    cands = sum(int(s["n_candidates"]) for s in stats)
    return {"queries": len(stats), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "p50_admit_wait_ms": float(np.percentile(qwait, 50)),
            "pairs_per_s": pairs / makespan, "candidates_per_s": cands / makespan,
            "queries_per_s": len(stats) / makespan, "makespan_s": makespan,
            "mean_batch_queries": float(np.mean([s["batch_queries"] for s in stats]))}


def run_serving(args):
    """Serving: the pathology datasets resident with their BVHs; Poisson
    streams of cube-window join queries (window volume log-uniform in
    [1e-3, 1] of the cube, i.e. about 10 to 10,000 nuclei per query) at
    several rates, admitted under a 40 GiB device budget and batched
    continuously on 4 streams; p50/p99 latency (submit to results on the
    host) and pairs/s per rate, against the same queries served one at a
    time, whose answers must be identical."""
    from paper_2609_24513_gb300 import pierce, synth
    A, B = make_workload(args.seed, args.nuclei, args.vessels)
    ctx = pierce.Context(0, serve_streams=4, budget_bytes=40 << 30)
    ha, hb = ctx.load(A), ctx.load(B)
    ctx.build(ha, args.width, args.leaf)
    ctx.build(hb, args.width, args.leaf)
    rates = [float(r) for r in args.rates.split(",")]
    n_alone = args.alone_queries
    counts = [int(min(args.max_queries, max(100, r * args.seconds_per_rate))) for r in rates]
    # one window list; every run takes a prefix of it
    lo, hi = synth.serving_windows(args.seed + 77, max(counts + [n_alone, 64]))
    # warm-up: every serving stream grows its scratch
    for _ in range(args.warmup):
        _serve_stream(ctx, pierce, ha, hb, lo[:64], hi[:64], np.zeros(64))
    # one query at a time: submit, wait for it, then the next
    alone_ans, alone_st = [], []
    t0 = time.perf_counter()
    for k in range(n_alone):
        a, st = ctx.poll(ctx.submit(ha, hb, lo[k], hi[k]), wait=True)
        alone_ans.append(a)
        alone_st.append(st)
    alone = _latency_summary(alone_st, time.perf_counter() - t0)
    clocks = ClockSampler(0)
    clocks.start()
    per_rate = {}
    identical = True
    for i, rate in enumerate(rates):
        n = counts[i]
        arr = synth.poisson_arrivals(args.seed + 100 + i, rate, n)
        ans, st, span = _serve_stream(ctx, pierce, ha, hb, lo[:n], hi[:n], arr)
        for k in range(min(n, n_alone)):   # same windows as the alone run
            identical &= bool(np.array_equal(ans[k], alone_ans[k]))
        per_rate[str(int(rate))] = _latency_summary(st, span)
    clk = clocks.stop()
    ctx.close()
    top = per_rate[str(int(rates[-1]))]
    line = {"metric": METRIC, "value": top["pairs_per_s"], "unit": "intersecting pairs/s",
            "n_gpus": 1, "steps": len(rates), "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+int64", "data": "synthetic",
            "config": {"workload": "serving: " + WORKLOAD + "; Poisson streams of cube-window "
                                   "join queries, window volume log-uniform in [1e-3, 1] of "
                                   "the cube, 40 GiB admission budget, 4 serving streams",
                       "rates_qps": rates, "alone_queries": n_alone},
            "alone": alone, "per_rate": per_rate, "answers_identical_to_alone": identical,
            "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=2001)
    ap.add_argument("--width", type=int, default=4)
    ap.add_argument("--leaf", type=int, default=2)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--graph", type=int, default=1)
    ap.add_argument("--front", default="stream", choices=sorted(FRONT_LEVELS),
                    help="refinement front end: streaming persistent kernel, breadth-first "
                         "levels, or none (per-warp passes only)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=10.0)
    ap.add_argument("--ref-total-s", type=float, default=120.0,
                    help="reference arm: seconds of oracle work over all timed steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the short serving run (p50/p99 latency) of the default line")
    ap.add_argument("--nuclei", type=int, default=10000)
    ap.add_argument("--vessels", type=int, default=500)
    ap.add_argument("--workload", default="pathology",
                    choices=["pathology", "batching", "urban", "serving"])
    ap.add_argument("--rates", default="50,100,200,500,1000,2000")
    ap.add_argument("--seconds-per-rate", type=float, default=2.0)
    ap.add_argument("--max-queries", type=int, default=4000)
    ap.add_argument("--alone-queries", type=int, default=400)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batching":
        run_batching(args)
    elif args.workload == "urban":
        run_urban(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()

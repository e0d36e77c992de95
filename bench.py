#!/usr/bin/env python
"""Benchmark of the GB300 convolved Count-sketch path on the star-join workload.

Workload (one "step" = the whole hot path once): a star join F(K1..K5) with
10^8 fact tuples whose five int64 foreign-key columns are Zipf(1.1) over
[0, 10^6), and five dimension tables D_i(K_i) of 10^6 uniform keys; sketch
width m = 2^16, d = 9 median rows.  A step zeroes the six sketches, updates
them with all 1.05 * 10^8 tuples (Algorithm 2; F is one 5-attribute convolved
sketch) and estimates the 6-way join (Algorithm 3: four circular
cross-correlations and one Hadamard product per row, median over rows).

Printed: one JSON line.  value = tuples/s of whole steps with the inputs
resident in HBM; e2e = the same through the C ABI from pinned host buffers,
host-to-device copies inside the timed region; roofline = the dominant kernel
(the fact-table update) against its bound; cpu_baseline = the CPU oracle on a
bounded sample, extrapolated to a full step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tuple updates/sec and join estimates/sec at 1 GB300; % HBM roofline; p99 ms"
HBM_FALLBACK_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fact-rows", type=int, default=100_000_000)
    ap.add_argument("--dim-rows", type=int, default=1_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-tuples", type=int, default=1_000_000)
    ap.add_argument("--workload", default="star",
                    choices=["star", "batched", "serving", "chain3", "chain8", "subqueries", "shapes"],
                    help="star: the headline step; batched: 256 relations, persistent plan vs per-relation "
                         "launches; serving: request loop latency")
    ap.add_argument("--requests", type=int, default=4000)
    ap.add_argument("--serving-rates", default="0.1,0.3,0.5,0.7,0.9",
                    help="serving: offered arrival rates as fractions of the saturated request rate")
    ap.add_argument("--sweep-requests", type=int, default=10_000,
                    help="serving: requests per offered-rate point")
    ap.add_argument("--no-domains", action="store_true",
                    help="do not declare the key domains (every tuple is hashed; no key tables)")
    ap.add_argument("--estimate-priority", default="high", choices=["high", "normal"],
                    help="stream priority of the estimates that overlap the next step's update (fused "
                         "estimator with the two-phase update: high 3.51 vs normal 3.62-3.63 ms per step, "
                         "its estimate kernels fill the SMs between phase-2 waves; with the single-phase "
                         "update normal 5.93 vs high 6.09; FP64: high 6.89 vs normal 7.71)")
    ap.add_argument("--plan-config", default=None,
                    help="batched workload: chunk_tuples,threads,ctas_per_sm,smem_max_counters[,smem16_max_counters] "
                         "instead of autotuning")
    ap.add_argument("--estimator", default="fused", choices=["fft64", "ntt", "fused"],
                    help="exact estimator arithmetic of the star step (identical rows from each)")
    ap.add_argument("--dims-concurrent", type=int, default=1, choices=[0, 1],
                    help="pipelined star steps: 1 = the five dimension updates on a second stream beside the "
                         "fact table's (their own counters), 0 = after it on the same stream")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="do not overlap step i's estimate with step i+1's update")
    ap.add_argument("--workloads", default="chain3,batched,chain8,serving,subqueries",
                    help="configs run after the star step (one GPU only) and reported under 'workloads'")
    ap.add_argument("--no-workloads", action="store_true", help="report the star step only")
    return ap.parse_args()


def declared_domains(args, wl):
    """Per relation, the key domains the workload declares (None: undeclared)."""
    return [None] * wl.r if args.no_domains else wl.domains


def star_config(args, total: int) -> dict:
    """The workload description both arms print (the same keys and values)."""
    return {"workload": workload_name(args), "relations": 6, "tuples_per_step": total, "m": 65536, "d": 9,
            "key_domains": "undeclared" if args.no_domains else "declared [0, 1e6) per column",
            "l2": "inputs (4.2 GB of keys) larger than L2; no flush needed"}


def workload_name(args) -> str:
    return (f"star join F(K1..K5) x D1..D5: F {args.fact_rows:.0e} rows Zipf s=1.1 over [0,1e6), "
            f"D_i {args.dim_rows:.0e} rows uniform over [0,1e6); m=65536, d=9, seed 42")


def percentile(xs, q):
    """Nearest-rank percentile."""
    ys = sorted(xs)
    k = max(1, int(-(-q * len(ys) // 100)))
    return ys[min(len(ys), k) - 1]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


# --------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------------------------
# CPU oracle baseline (bounded sample, extrapolated to one full step)
# --------------------------------------------------------------------------------------

def cpu_oracle_step_seconds(wl_cpu_cols, total_rows, m, d, seed, sample_tuples, threads=None):
    """Times the CPU oracle on a sample of every relation's tuples and on a sample of
    the estimator's correlation outputs; returns (extrapolated seconds per full step,
    threads used, description of the sample).  threads: all host cores by default."""
    import numpy as np

    import oracle as O
    threads = threads or os.cpu_count() or 1
    q = O.canonical_query([5, 1, 1, 1, 1, 1], [(0, i, 1 + i, 0) for i in range(5)])
    co = O.draw_coefficients(seed, d, q.n_comp, len(q.edges))
    update_s = 0.0
    sketches = []
    for k, cols in enumerate(wl_cpu_cols):
        ns = cols.shape[1]
        t0 = time.perf_counter()
        sk = O.sketch_relation(q, co, k, cols, None, m, threads=threads)
        dt = time.perf_counter() - t0
        update_s += dt * total_rows[k] / ns
        sketches.append(sk)
    # estimator: one correlation step of row 0 on a sample of output bins
    a = sketches[2][0].tolist()
    x = sketches[0][0].tolist()
    bins = list(range(0, m, 64))
    t0 = time.perf_counter()
    O.correlate(a, x, threads=threads, bins=bins)
    dt = time.perf_counter() - t0
    corr_steps = 4
    est_s = dt * (m / len(bins)) * corr_steps * d
    desc = (f"oracle update of the first {wl_cpu_cols[0].shape[1]} tuples of each relation, scaled by each "
            f"relation's row count; one exact O(m^2) correlation on {len(bins)} of {m} output bins, scaled to "
            f"{corr_steps} steps x {d} rows")
    return update_s + est_s, threads, desc, update_s, est_s


# --------------------------------------------------------------------------------------
# main arms
# --------------------------------------------------------------------------------------

def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle, as it stands, on bounded samples of the same
    workload; each step extrapolates one full step's time."""
    import torch

    import synth
    if rank != 0:
        return
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    ns = args.cpu_sample_tuples
    wl = synth.star(n_fact=ns, n_dim=min(ns, args.dim_rows), device=dev)
    cols = [r.cols.cpu().numpy() for r in wl.relations]
    rows = [args.fact_rows] + [args.dim_rows] * 5
    times = []
    for it in range(args.warmup + args.steps):
        sec, threads, desc, _, _ = cpu_oracle_step_seconds(cols, rows, wl.m, wl.d, wl.hash_seed, ns)
        if it >= args.warmup:
            times.append(sec)
    total = sum(rows)
    ms = statistics.mean(times) * 1e3
    val = total / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "tuples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": star_config(args, total),
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": desc, "value": val, "unit": "tuples/s"},
            "e2e": {"value": val, "unit": "tuples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def gpu_id(local=0) -> str:
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        return str(local)


def run_ours(args, world, rank, local):
    import torch

    import paper_2402_15953_gb300 as pkg
    import synth
    from paper_2402_15953_gb300 import build as pkg_build

    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    pkg_build.build()
    pkg.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = 42 + rank
    wl = synth.star(n_fact=args.fact_rows, n_dim=args.dim_rows, seed=seed, device="cuda")
    torch.cuda.synchronize()
    rels = [r.cols for r in wl.relations]
    total = sum(int(c.shape[1]) for c in rels)
    s = pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed, device=dev)
    s.set_estimator(args.estimator)
    stream = torch.cuda.current_stream()
    doms = declared_domains(args, wl)

    def step(ev=None):
        s.reset()
        for k, c in enumerate(rels):
            if ev is not None and k == 0:
                ev[0].record(stream)
            s.update(k, c, domain=doms[k])
            if ev is not None and k == 0:
                ev[1].record(stream)
        if ev is not None:
            ev[2].record(stream)
        return s.estimate()

    for _ in range(args.warmup):
        est = step()
    torch.cuda.synchronize()
    barrier(world)

    clk = ClockSampler(gpu_id(local))
    clk.start()
    time.sleep(0.25)
    launches0 = pkg.sk_launch_count()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier(world)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        e = evs[i]
        e[3].record(stream)
        est = step(e)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = pkg.sk_launch_count() - launches0
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [evs[i][3].elapsed_time(evs[i + 1][3]) if i + 1 < args.steps else evs[i][3].elapsed_time(t_end)
               for i in range(args.steps)]
    upd_fact_ms = [e[0].elapsed_time(e[1]) for e in evs]
    upd_all_ms = [e[3].elapsed_time(e[2]) for e in evs]
    ms_per_step = max_over_ranks(world, total_ms / args.steps)
    value = world * total / (ms_per_step / 1e3)

    # The same estimate in each exact arithmetic (identical rows): the FP64 FFT with its
    # certificate, the GF(q) number-theoretic transform, the fused product of spectra modulo
    # CRT primes (this query qualifies).
    by_arith = {}
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name in ("fft64", "ntt", "fused"):
        s.set_estimator(name)
        alt = s.estimate()
        torch.cuda.synchronize()
        e_a.record(stream)
        for _ in range(args.steps):
            alt = s.estimate()
        e_b.record(stream)
        torch.cuda.synchronize()
        by_arith[name] = (e_a.elapsed_time(e_b) / args.steps, alt)
    s.set_estimator(args.estimator)

    # Pipelined steps: two counter buffers; step i's update runs on the update stream while
    # step i-1's estimate runs on the estimate stream (the update is integer-bound, the FFTs
    # FP64-bound, so they share the SMs).  Every step still does the whole path on its own
    # batch; only the overlap between consecutive steps differs.
    pipe = None
    if not args.no_pipeline:
        s2 = pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed, device=dev)
        s2.set_estimator(args.estimator)
        sets = [s, s2]
        upd = torch.cuda.Stream()
        upd_dims = torch.cuda.Stream()
        est_stream = torch.cuda.Stream(priority=-1 if args.estimate_priority == "high" else 0)
        evs2 = [torch.cuda.Event() for _ in range(2)]
        evs_dims = [torch.cuda.Event() for _ in range(2)]
        ev_reset = [torch.cuda.Event() for _ in range(2)]

        def run_pipelined(k_steps, t_start=None):
            outs = []
            for i in range(k_steps + 1):
                if i < k_steps:
                    cur = sets[i % 2]
                    with torch.cuda.stream(upd):
                        if i == 0 and t_start is not None:
                            t_start.record(upd)
                        cur.reset()
                        if args.dims_concurrent:
                            # the dimension relations' updates (their own counters) on a second
                            # stream once the counters are reset, beside the fact table's
                            ev_reset[i % 2].record(upd)
                            cur.update(0, rels[0], domain=doms[0])
                        else:
                            for kk, c in enumerate(rels):
                                cur.update(kk, c, domain=doms[kk])
                        evs2[i % 2].record(upd)
                    if args.dims_concurrent:
                        with torch.cuda.stream(upd_dims):
                            upd_dims.wait_event(ev_reset[i % 2])
                            for kk in range(1, len(rels)):
                                cur.update(kk, rels[kk], domain=doms[kk])
                            evs_dims[i % 2].record(upd_dims)
                if i >= 1:
                    with torch.cuda.stream(est_stream):
                        est_stream.wait_event(evs2[(i - 1) % 2])
                        if args.dims_concurrent:
                            est_stream.wait_event(evs_dims[(i - 1) % 2])
                        outs.append(sets[(i - 1) % 2].estimate())
            return outs

        run_pipelined(args.warmup)
        torch.cuda.synchronize()
        barrier(world)
        launches_p0 = pkg.sk_launch_count()
        # device time: from an event on the update stream before the first step's reset to an
        # event after the last estimate, recorded on the estimate stream (estimate() returns
        # once its stream's work is done, and that work waited on every update)
        p_start, p_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pouts = run_pipelined(args.steps, p_start)
        p_end.record(est_stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(world, p_start.elapsed_time(p_end) / args.steps)
        pipe = {"ms_per_step": pms, "value": world * total / (pms / 1e3),
                "gpu_launches": pkg.sk_launch_count() - launches_p0,
                "same_median_as_serial": all(o["median"] == est["median"] for o in pouts),
                "estimate_stream_priority": args.estimate_priority,
                "dimension_updates_on_second_stream": bool(args.dims_concurrent),
                "timing": "CUDA events: update stream before the first reset to the estimate stream after the last estimate"}
        s2.close()
    clocks = clk.stop()   # sampled over the serial and the pipelined timed regions

    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    fact_bytes = 8 * 5 * args.fact_rows
    fact_ms = statistics.mean(upd_fact_ms)
    achieved_gbs = fact_bytes / (fact_ms / 1e3) / 1e9
    mulmods_per_fact_tuple = wl.d * 5 * (1 + 3 * 1)
    fact_s = fact_ms / 1e3
    tables = not args.no_domains
    if tables:
        # The fact-table update call is three launches, timed together: k_key_table_l24 hashes
        # the 5 x 1e6 declared domain keys once (9 rows each, 24-byte records), k_tab_items
        # gathers the five records of each of the 1e8 tuples and appends every row's bin to its
        # warp's region of that row (phase 1), k_part_accum reads one part's items of a row and
        # adds them into a half-row int32 sketch in shared memory, flushing each counter once
        # (phase 2).
        # HBM roofline: algorithmic bytes = the 40 key bytes per tuple.  traffic = DRAM bytes
        # of one ncu capture of both phases at 2e7 rows (k_tab_items 1.4755 GB read + 0.4119 GB
        # written, k_part_accum 0.3665 + 0.0002 GB: key stream, record misses and the items'
        # round trip) scaled to this row count, plus the table write (5e6 x 24 B).
        # L2 roofline beside it: L2 requests per tuple from the same capture (5.71: 5.21 in
        # phase 1, 0.50 in phase 2; 16.35 with one 64-bit reduction per counter update).
        # The bound phase 1 meets is the L1 data pipe: 5.97 wavefronts per tuple (one per
        # record gather and lane, plus the key loads and item stores), 82 % of its peak of one
        # wavefront per clock and SM in that capture.
        traffic = (1.4755 + 0.4119 + 0.3665 + 0.0002) * args.fact_rows / 2e7 + 5 * 1_000_000 * 24 / 1e9
        kernel = "k_key_table_l24 + k_tab_items<5,24B> + k_part_accum (fact table F, two-phase)"
        l2_req_per_tuple = 5.71
        l2_peak = 188 * 2.016e9
        l2_rate = l2_req_per_tuple * args.fact_rows / fact_s
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak, "traffic": traffic, "kernel": kernel,
                    "work": "40 key bytes per fact tuple (5 int64 columns)",
                    "traffic_unit": "GB per launch (ncu, 2e7-row launches scaled, + table write)",
                    "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"}
        extra = {"roofline_l2": {"bound": "l2_requests", "achieved": l2_rate / 1e9, "peak": l2_peak / 1e9,
                                 "unit": "G requests/s", "frac": l2_rate / l2_peak,
                                 "per_tuple": l2_req_per_tuple, "kernel": kernel,
                                 "source": "ncu lts__t_requests of k_tab_items + k_part_accum (2e7 rows)"},
                 "roofline_l1_phase1": {"bound": "l1_data_pipe_wavefronts", "per_tuple": 5.97,
                                        "frac_ncu": 0.824, "kernel": "k_tab_items<5,24B>",
                                        "source": "ncu l1tex__data_pipe_lsu_wavefronts (2e7 rows)"}}
    else:
        # Per-tuple hashing (no declared domains): integer-ALU roofline, algorithmic work =
        # GF(2^61-1) Horner multiply-add steps (1 per bin hash, 3 per sign hash), peak = the
        # step rate of the same arithmetic without loads, atomics or combination (6.4 steps
        # per clock per SM measured) x 152 SMs x 2.07 GHz.  traffic: DRAM bytes of one ncu
        # capture of k_update (2e7-row launch: 808.2 MB), scaled to this launch's row count.
        steps_per_s = args.fact_rows * mulmods_per_fact_tuple / fact_s
        alu_peak_steps = 6.4 * 152 * 2.07e9
        traffic = 808.2e6 * args.fact_rows / 2e7 / 1e9
        roofline = {"bound": "alu", "achieved": steps_per_s / 1e9, "peak": alu_peak_steps / 1e9, "unit": "Gstep/s",
                    "frac": steps_per_s / alu_peak_steps, "traffic": traffic,
                    "kernel": "k_update<5,pow2,global,DEG1> (fact table F)",
                    "work": f"{mulmods_per_fact_tuple} GF(2^61-1) Horner steps per fact tuple",
                    "traffic_unit": "GB per launch (ncu, 2e7-row launch scaled)"}
        extra = {"roofline_hbm": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": achieved_gbs / hbm_peak, "traffic": traffic, "traffic_unit": "GB per launch",
                                  "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"}}
    # counter updates of the fact table (one per row and tuple), as a rate over the same call
    extra["counter_updates"] = {"per_tuple": wl.d, "achieved": wl.d * args.fact_rows / fact_s / 1e9,
                                "unit": "G updates/s",
                                "kind": ("shared-memory reductions into half-row int32 sketches, one 64-bit flush per "
                                         "counter and CTA" if tables else
                                         "red.global.add.u64 into the L2-resident sketch")}

    serial = {"ms_per_step": ms_per_step, "value": value, "gpu_launches": launches}
    if pipe is not None and pipe["value"] > value:
        value, ms_per_step, launches = pipe["value"], pipe["ms_per_step"], pipe["gpu_launches"]

    line = {
        "metric": METRIC, "value": value, "unit": "tuples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic", "estimator": args.estimator,
        "config": star_config(args, total),
        "parallelism": f"replicas x{world}", "pipelined": pipe is not None and value == pipe["value"],
        "serial_steps": serial, "pipelined_steps": pipe,
        "estimates_per_s": world * 1e3 / ms_per_step,
        "p50_ms": statistics.median(step_ms), "p99_ms": percentile(step_ms, 99.0),
        "update_ms": statistics.mean(upd_all_ms), "estimate_ms": statistics.mean(step_ms) - statistics.mean(upd_all_ms),
        "fact_update_ms": fact_ms,
        **{f"estimate_{name}": {"estimate_ms": ms_e, "identical_rows": alt["rows"] == est["rows"],
                                "limbs_or_primes": alt["max_limbs"], "limb_bits": alt["limb_bits"],
                                "step_ms_serial_with_it": statistics.mean(upd_all_ms) + ms_e}
           for name, (ms_e, alt) in by_arith.items()},
        "roofline": roofline, **extra,
        "estimate_check": {"median": str(est["median"]), "max_residual": est["max_residual"],
                           "max_limbs": est["max_limbs"], "limb_bits": est["limb_bits"]},
        "gpu_launches": launches, "clocks": clocks,
    }

    if not args.no_e2e:
        staged = run_e2e(args, s, wl, stream, world)
        direct = run_e2e_direct(args, s, wl, stream, world)
        direct_p = run_e2e_direct_pipelined(args, wl, world)
        alts = {"staged_copies": staged, "direct_host_reads": direct, "direct_host_reads_pipelined": direct_p}
        line["e2e"] = dict(max(alts.values(), key=lambda x: x["value"]))
        line["e2e_alternatives"] = alts
        # the host link's own rate, for scale: the e2e step moves all key bytes across it
        link = h2d_link_gbs()
        moved = line["e2e"]["h2d_bytes_per_step"] / (line["e2e"]["ms_per_step"] / 1e3) / 1e9
        line["e2e"]["h2d_gbs"] = moved
        line["e2e"]["h2d_link_gbs_measured"] = link
        line["e2e"]["link_frac"] = moved / link
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        ns = min(args.cpu_sample_tuples, args.fact_rows)
        cols = [c[:, :ns].cpu().numpy() for c in rels]
        rows = [int(c.shape[1]) for c in rels]
        sec, threads, desc, _, _ = cpu_oracle_step_seconds(cols, rows, wl.m, wl.d, wl.hash_seed, ns)
        line["cpu_baseline"] = {"value": total / sec, "unit": "tuples/s", "cores": threads, "kind": "oracle",
                                "sample": desc}
        # the paper's setting is one CPU core: the same oracle on one thread, smaller sample
        ns1 = max(1, ns // 10)
        sec1, _, desc1, _, _ = cpu_oracle_step_seconds([c[:, :ns1] for c in cols], rows, wl.m, wl.d, wl.hash_seed,
                                                       ns1, threads=1)
        line["cpu_baseline_1core"] = {"value": total / sec1, "unit": "tuples/s", "cores": 1, "kind": "oracle",
                                      "sample": desc1}
    s.close()
    if not args.no_workloads and world == 1:
        # every other configuration of the workload set, each with its own timed region,
        # clock samples and parity checks, after the star's inputs are released
        del rels, wl
        torch.cuda.empty_cache()
        line["workloads"] = {}
        for name in [x for x in args.workloads.split(",") if x]:
            try:
                line["workloads"][name] = run_workload(args, world, rank, name)
            except Exception as ex:   # one failing configuration must not hide the others
                line["workloads"][name] = {"error": repr(ex)}
            torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(line), flush=True)


def h2d_link_gbs():
    """Best of five 2 GiB copies from page-locked host memory to the device (CUDA events):
    the host link's copy rate on this machine."""
    import torch
    h = torch.empty(1 << 28, dtype=torch.int64, pin_memory=True)
    h.fill_(1)
    dev = torch.empty(1 << 28, dtype=torch.int64, device="cuda")
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dev.copy_(h, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, h.numel() * 8 / (e0.elapsed_time(e1) * 1e6))
    del h, dev
    return best


def run_e2e(args, s, wl, stream, world):
    """Same steps through the public API from pinned host buffers: every step copies all
    key columns host-to-device (pipelined in chunks on a copy stream) and reads the
    estimate back."""
    import torch
    host = [r.cols.cpu().pin_memory() for r in wl.relations]
    chunk = 1 << 23
    maxa = max(h.shape[0] for h in host)
    bufs = [torch.empty((maxa, chunk), dtype=torch.int64, device="cuda") for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    free_ev = [torch.cuda.Event() for _ in range(2)]
    for e in free_ev:
        e.record(stream)
    h2d = sum(h.numel() * 8 for h in host)
    doms = declared_domains(args, wl)

    def step():
        s.reset()
        slot = 0
        for k, h in enumerate(host):
            a, n = h.shape
            for i0 in range(0, n, chunk):
                i1 = min(n, i0 + chunk)
                b = bufs[slot]
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(free_ev[slot])
                    for u in range(a):
                        b[u, : i1 - i0].copy_(h[u, i0:i1], non_blocking=True)
                    ready = torch.cuda.Event()
                    ready.record(copy_stream)
                stream.wait_event(ready)
                s.update(k, b[:a, : i1 - i0], domain=doms[k])
                free_ev[slot].record(stream)
                slot ^= 1
        return s.estimate()

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    steps = max(3, args.steps // 3)
    # device time with CUDA events: from the step's stream before the first copy is issued to
    # the same stream after the last estimate (which waited on every copy and update)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    dt = max_over_ranks(world, e0.elapsed_time(e1) / 1e3 / steps)
    total = sum(h.shape[1] for h in host)
    d = wl.d
    d2h = 4 * (8 + 3 * d * 32 + 8) + 2 * d * 32 + 4
    return {"value": world * total / dt, "unit": "tuples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "steps": steps, "method": "pipelined cudaMemcpyAsync of 8M-row chunks"}


def run_batched(args, world, rank):
    """256 relations (lognormal row counts 1e3..1e7, 1-4 Zipf columns, m = 2^10..2^18, d = 7,
    +-1 weights with 10% deletions): one step resets the 256 sketches and applies every
    relation's batch, (a) one sk_sketch_reset and one sk_sketch_update_batch launch per
    relation, (b) one sk_update_plan_zero and one persistent sk_update_plan_run (autotuned),
    (c) the same captured in a CUDA graph.  Parity: the sketches of (a) and (b) are equal,
    and the three smallest relations' sketches equal the CPU oracle's; the 256 estimates are
    identical from one FP64 call per set, one fused call per set and one sk_estimate_many."""
    import numpy as np
    import torch

    import paper_2402_15953_gb300 as pkg
    import synth
    from paper_2402_15953_gb300 import build as pkg_build
    pkg_build.build()
    wl = synth.batched(seed=42 + rank, device="cuda")
    total = sum(b.relation.n for b in wl)
    sa = [pkg.SketchSet(b.num_join_attrs, b.edges, b.m, b.d, b.hash_seed) for b in wl]
    sb = [pkg.SketchSet(b.num_join_attrs, b.edges, b.m, b.d, b.hash_seed) for b in wl]
    plan = pkg.UpdatePlan([(s, 0, b.relation.cols, b.relation.weights) for s, b in zip(sb, wl)])
    stream = torch.cuda.current_stream()
    if args.plan_config:
        plan.set_config(*[int(x) for x in args.plan_config.split(",")])
        best, tune_ms = plan.config(), 0.0
    else:
        best, tune_ms = plan.autotune()

    def step_a():
        for s, b in zip(sa, wl):
            s.reset()
            s.update(0, b.relation.cols, b.relation.weights)

    def step_b():
        plan.zero()     # the 256 relations' counters, one launch
        plan.run()

    def timeit(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(world, e0.elapsed_time(e1) / steps)

    clk = ClockSampler(gpu_id())
    clk.start()
    time.sleep(0.2)
    ms_a = timeit(step_a, args.steps)
    ms_b = timeit(step_b, args.steps)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        step_b()
    side.synchronize()
    with torch.cuda.graph(g, stream=side):
        step_b()
    ms_c = timeit(g.replay, args.steps)
    clocks = clk.stop()
    step_a()
    step_b()
    torch.cuda.synchronize()
    same = all(torch.equal(x.counters, y.counters) for x, y in zip(sa, sb))
    # the oracle on the three smallest relations (all d rows of relation 0)
    import oracle as O
    O.build()
    oracle_ok = True
    for i in sorted(range(len(wl)), key=lambda j: wl[j].relation.n)[:3]:
        b = wl[i]
        q = O.canonical_query(b.num_join_attrs, b.edges)
        co = O.draw_coefficients(b.hash_seed, b.d, q.n_comp, len(q.edges))
        want = O.sketch_relation(q, co, 0, b.relation.cols.cpu().numpy(), b.relation.weights.cpu().numpy(), b.m,
                                 threads=os.cpu_count() or 1)
        oracle_ok = oracle_ok and bool(np.array_equal(sb[i].counters[0].cpu().numpy(), want))

    # estimating all 256 sets: one sk_estimate_join per set (FP64, then fused) against one
    # sk_estimate_many call (fused sets grouped by width).  Each dimension relation first gets
    # 2e4 keys from the fact column it joins, so every estimate is of a non-empty join.
    for s, b in zip(sb, wl):
        for k in range(1, len(b.num_join_attrs)):
            s.update(k, b.relation.cols[k - 1:k, :20_000].contiguous())

    def est_seq():
        return [x.estimate() for x in sb]

    def est_many():
        return pkg.estimate_many(sb)

    def host_time(fn, reps):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / reps, out

    reps = max(1, args.steps // 5)
    for x in sb:
        x.set_estimator("fft64")
    seq_fft_ms, rows_fft = host_time(est_seq, reps)
    for x in sb:
        x.set_estimator("fused")
    seq_fu_ms, rows_fu = host_time(est_seq, reps)
    many_ms, rows_many = host_time(est_many, reps)
    est_same = [e["rows"] for e in rows_fft] == [e["rows"] for e in rows_many] == [e["rows"] for e in rows_fu]
    estimates = {"sets": len(sb), "one_call_per_set_fft64_ms": seq_fft_ms, "one_call_per_set_fused_ms": seq_fu_ms,
                 "estimate_many_fused_ms": many_ms, "estimates_per_s_many": len(sb) / (many_ms / 1e3),
                 "identical_rows": est_same}
    line = {"metric": "batched build: tuples/s for 256 relations", "value": world * total / (ms_c / 1e3),
            "unit": "tuples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_c,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": "256 relations, rows lognormal(median 1e5, sigma 1.5) in [1e3, 1e7], 1-4 Zipf "
                                   "columns (s in [0.8, 1.4], domains 1e4..1e7), m = 2^10..2^18, d = 7, +-1 weights "
                                   "with 10% deletions", "tuples_per_step": total},
            "per_relation_launches_ms": ms_a, "persistent_plan_ms": ms_b, "persistent_plan_graph_ms": ms_c,
            "speedup_vs_per_relation": ms_a / ms_c, "autotuned": best, "estimates": estimates, "clocks": clocks,
            "parity": {"plan_equals_per_relation": same, "smallest_3_relations_equal_oracle": oracle_ok,
                       "estimates_identical_fft64_fused_many": est_same,
                       "ok": bool(same and oracle_ok and est_same)}}
    plan.close()
    for s in sa + sb:
        s.close()
    return line


def run_serving(args, world, rank):
    """64 live sets (chains of 2-6 relations, m = 2^14..2^18, d = 9); update batches of
    log-uniform 1e3..1e6 tuples (Zipf 1.1 keys over 1e6, 5% of rows deleted) and estimate
    requests, 10:1, Poisson arrivals; HBM budget 32 GB.  First every request is submitted
    at once (saturated throughput), then arrivals at 10, 30, 50, 70 and 90% of that rate, 1e4
    requests per point; latency = arrival to result on the host.  Parity: every estimate of the saturated run equals the
    same request run one by one, and the oracle's for two sets."""
    import numpy as np
    import torch

    import synth
    from paper_2402_15953_gb300 import build as pkg_build
    from paper_2402_15953_gb300.serve import SketchServer
    pkg_build.build()
    rng = np.random.default_rng(7 + rank)
    n_sets = 64
    sets = []
    for i in range(n_sets):
        r = int(rng.integers(2, 7))
        attrs = [1 if k in (0, r - 1) else 2 for k in range(r)]
        edges = [(k, 0 if k == 0 else 1, k + 1, 0) for k in range(r - 1)]
        sets.append((attrs, edges, 1 << int(rng.integers(14, 19)), 9, int(rng.integers(1 << 62))))
    pool = []
    for j in range(48):
        n = int(round(10 ** rng.uniform(3, 6)))
        for a in (1, 2):
            cols = torch.stack([synth.zipf_keys(n, 1.1, 1_000_000, synth.sub_seed(j, a, c), "cuda") for c in range(a)])
            w = torch.where(torch.rand(n, device="cuda") < 0.05, -1, 1).to(torch.int64)
            pool.append((a, cols.cpu().pin_memory(), w.cpu().pin_memory()))
    by_arity = {1: [p for p in pool if p[0] == 1], 2: [p for p in pool if p[0] == 2]}

    def make_trace(count, seed):
        g = np.random.default_rng(seed)
        tr = []
        for j in range(count):
            sid = int(g.integers(n_sets))
            if j % 11 == 10:
                tr.append(("estimate", sid))
            else:
                attrs = sets[sid][0]
                rel = int(g.integers(len(attrs)))
                _, cols, w = by_arity[attrs[rel]][int(g.integers(len(by_arity[attrs[rel]])))]
                tr.append(("update", sid, rel, cols, w))
        return tr

    def run(trace, rate):
        srv = SketchServer(hbm_budget_bytes=32 << 30, update_slots=16, estimate_workers=4)
        for i, (a, e, m, d, sd) in enumerate(sets):
            srv.register_set(i, a, e, m, d, sd)
            srv.sets[i].sset.set_estimator(args.estimator)
        reqs = []
        t0 = time.perf_counter()

        def producer():
            gaps = np.random.default_rng(99).exponential(1.0 / rate, size=len(trace)) if rate else None
            t = time.perf_counter()
            for j, r in enumerate(trace):
                if rate:
                    t += gaps[j]
                    while time.perf_counter() < t:
                        pass
                if r[0] == "update":
                    reqs.append(srv.submit_update(r[1], r[2], r[3], r[4]))
                else:
                    reqs.append(srv.submit_estimate(r[1]))

        th = threading.Thread(target=producer)
        th.start()
        while th.is_alive() or srv.pending():
            srv.serve(until_idle=True)
            time.sleep(1e-4)
        th.join()
        srv.serve(until_idle=True)
        wall = time.perf_counter() - t0
        srv.close()
        lat = sorted(r.latency * 1e3 for r in reqs)
        est = sorted(r.latency * 1e3 for r in reqs if r.kind == "estimate")
        tuples = sum(r.cols.shape[1] for r in reqs if r.kind == "update")
        errors = sum(1 for r in reqs if r.error)
        rows = {j: r.result["rows"] for j, r in enumerate(reqs) if r.kind == "estimate" and r.result is not None}
        return {"requests": len(reqs), "wall_s": wall, "requests_per_s": len(reqs) / wall,
                "tuples_per_s": tuples / wall, "p50_ms": lat[len(lat) // 2], "p99_ms": percentile(lat, 99.0),
                "estimate_p50_ms": est[len(est) // 2] if est else None,
                "estimate_p99_ms": percentile(est, 99.0) if est else None, "errors": errors}, rows

    def sequential(trace):
        """Baseline: the same requests one at a time, each update a copy plus its own launch,
        each estimate after the previous request completed (no overlap, no admission)."""
        from paper_2402_15953_gb300 import SketchSet
        live = [SketchSet(a, e, m, d, sd) for (a, e, m, d, sd) in sets]
        for x in live:
            x.set_estimator(args.estimator)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tuples = 0
        rows = {}
        for j, r in enumerate(trace):
            if r[0] == "update":
                live[r[1]].update(r[2], r[3].cuda(non_blocking=True), r[4].cuda(non_blocking=True))
                torch.cuda.synchronize()
                tuples += r[3].shape[1]
            else:
                rows[j] = live[r[1]].estimate()["rows"]
        wall = time.perf_counter() - t0
        for x in live:
            x.close()
        return {"requests": len(trace), "wall_s": wall, "requests_per_s": len(trace) / wall,
                "tuples_per_s": tuples / wall}, rows

    def capacity(trace):
        """The server's own throughput: every request queued on a held server, then
        released at once (the timed region starts at the release)."""
        srv = SketchServer(hbm_budget_bytes=32 << 30, update_slots=16, estimate_workers=4)
        for i, (a, e, m, d, sd) in enumerate(sets):
            srv.register_set(i, a, e, m, d, sd)
            srv.sets[i].sset.set_estimator(args.estimator)
        srv.hold(True)
        reqs = [srv.submit_update(r[1], r[2], r[3], r[4]) if r[0] == "update" else srv.submit_estimate(r[1])
                for r in trace]
        t0 = time.perf_counter()
        srv.hold(False)
        srv.serve(until_idle=True)
        wall = time.perf_counter() - t0
        srv.close()
        tuples = sum(r.cols.shape[1] for r in reqs if r.kind == "update")
        return {"requests": len(reqs), "wall_s": wall, "requests_per_s": len(reqs) / wall,
                "tuples_per_s": tuples / wall, "errors": sum(1 for r in reqs if r.error)}

    def oracle_check(trace, rows):
        """The CPU oracle's Algorithm 3 for the last estimate of up to two two-relation sets
        (whose estimate is one inner product per row), over that set's updates before it."""
        import oracle as O
        O.build()
        cands = []
        for sid, (a, e, m, d, sd) in enumerate(sets):
            if len(a) != 2:
                continue
            last = max((j for j, r in enumerate(trace) if r[0] == "estimate" and r[1] == sid), default=None)
            if last is None:
                continue
            n = sum(r[3].shape[1] for r in trace[:last] if r[0] == "update" and r[1] == sid)
            cands.append((n, sid, last))
        checked, ok = [], True
        for n, sid, last in sorted(cands)[:2]:
            a, e, m, d, sd = sets[sid]
            q = O.canonical_query(a, e)
            co = O.draw_coefficients(sd, d, q.n_comp, len(q.edges))
            acc = [np.zeros((d, m), dtype=np.int64) for _ in a]
            for r in trace[:last]:
                if r[0] == "update" and r[1] == sid:
                    acc[r[2]] += O.sketch_relation(q, co, r[2], r[3].numpy(), r[4].numpy(), m,
                                                   threads=os.cpu_count() or 1)
            ref = O.estimate(q, acc)
            ok = ok and rows.get(last) == ref.rows
            checked.append({"set": sid, "request": last, "tuples": n})
        return ok, checked

    trace = make_trace(args.requests, 1)
    run(make_trace(200, 2), None)           # warm-up (scratch allocation, kernel attributes)
    clk = ClockSampler(gpu_id())
    clk.start()
    time.sleep(0.2)
    sat, sat_rows = run(trace, None)
    cap = capacity(trace)
    seq, seq_rows = sequential(trace)
    points = {"saturated": sat, "server_capacity": cap, "sequential_one_by_one": seq}
    sweep = make_trace(args.sweep_requests, 3)
    for frac in [float(x) for x in args.serving_rates.split(",") if x]:
        pt, _ = run(sweep, frac * sat["requests_per_s"])
        pt["offered_requests_per_s"] = frac * sat["requests_per_s"]
        points[f"rate_{int(round(frac * 100))}pct"] = pt
    clocks = clk.stop()
    mixed_equal = set(sat_rows) == set(seq_rows) and all(sat_rows[j] == seq_rows[j] for j in seq_rows)
    oracle_ok, checked = oracle_check(trace, seq_rows)
    line = {"metric": "serving: p50/p99 request latency and throughput", "value": sat["tuples_per_s"],
            "unit": "tuples/s", "n_gpus": world, "steps": args.requests, "warmup": 200,
            "ms_per_step": 1e3 / sat["requests_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "estimator": args.estimator,
            "config": {"workload": "64 live sets (chains of 2-6 relations, m = 2^14..2^18, d = 9); update batches "
                                   "log-uniform 1e3..1e6 tuples, Zipf 1.1 keys over 1e6, 5% deletions; 10 updates : "
                                   "1 estimate; Poisson arrivals; HBM budget 32 GB"},
            "points": points, "capacity_vs_one_by_one": cap["requests_per_s"] / seq["requests_per_s"],
            "clocks": clocks,
            "parity": {"mixed_equals_one_by_one": mixed_equal, "estimates_compared": len(seq_rows),
                       "oracle_last_estimate_of": checked, "oracle_equal": oracle_ok,
                       "ok": bool(mixed_equal and oracle_ok and sat["errors"] == 0)}}
    return line


def run_e2e_direct(args, s, wl, stream, world):
    """Same steps through the C ABI with the key columns in page-locked host memory passed
    straight to sk_sketch_update_batch: the update kernel reads them across the host link
    (NVLink-C2C on Grace-Blackwell), so the host-to-device transfer happens inside the
    kernel; the estimate is read back as usual."""
    import torch

    import paper_2402_15953_gb300 as pkg
    host = [r.cols.cpu().pin_memory() for r in wl.relations]
    h2d = sum(h.numel() * 8 for h in host)
    sid = stream.cuda_stream
    doms = declared_domains(args, wl)

    def step():
        s.reset()
        for k, h in enumerate(host):
            pkg.sk_sketch_update_batch(s.handle, k, int(h.shape[1]), h.data_ptr(), int(h.stride(0)), None, doms[k],
                                       sid)
        return s.estimate()

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    steps = max(3, args.steps // 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    dt = max_over_ranks(world, e0.elapsed_time(e1) / 1e3 / steps)
    total = sum(h.shape[1] for h in host)
    d = wl.d
    d2h = 4 * (256 + (1 + 3 * d) * 8) + 2 * d * 32 + 4
    return {"value": world * total / dt, "unit": "tuples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "steps": steps, "method": "kernels read pinned host columns directly"}


def run_e2e_direct_pipelined(args, wl, world):
    """As run_e2e_direct, with two sketch sets so that step i's estimate (device work plus its
    read-back) runs while step i+1's update kernels read the next batch across the host link:
    every step still moves all of its key columns from host memory and reads back its
    estimate inside the timed region."""
    import torch

    import paper_2402_15953_gb300 as pkg
    host = [r.cols.cpu().pin_memory() for r in wl.relations]
    h2d = sum(h.numel() * 8 for h in host)
    doms = declared_domains(args, wl)
    sets = [pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed) for _ in range(2)]
    for x in sets:
        x.set_estimator(args.estimator)
    upd, est = torch.cuda.Stream(), torch.cuda.Stream(priority=-1 if args.estimate_priority == "high" else 0)
    done = [torch.cuda.Event() for _ in range(2)]

    def run(k_steps):
        outs = []
        for i in range(k_steps + 1):
            if i < k_steps:
                with torch.cuda.stream(upd):
                    cur = sets[i % 2]
                    cur.reset()
                    for k, h in enumerate(host):
                        pkg.sk_sketch_update_batch(cur.handle, k, int(h.shape[1]), h.data_ptr(), int(h.stride(0)),
                                                   None, doms[k], upd.cuda_stream)
                    done[i % 2].record(upd)
            if i >= 1:
                with torch.cuda.stream(est):
                    est.wait_event(done[(i - 1) % 2])
                    outs.append(sets[(i - 1) % 2].estimate())
        return outs

    run(max(1, args.warmup))
    torch.cuda.synchronize()
    barrier(world)
    steps = max(3, args.steps // 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(upd)
    outs = run(steps)
    e1.record(est)
    torch.cuda.synchronize()
    dt = max_over_ranks(world, e0.elapsed_time(e1) / 1e3 / steps)
    for x in sets:
        x.close()
    total = sum(h.shape[1] for h in host)
    d = wl.d
    d2h = 4 * (256 + (1 + 3 * d) * 8) + 2 * d * 32 + 4
    return {"value": world * total / dt, "unit": "tuples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "steps": steps, "estimates": len(outs),
            "method": "kernels read pinned host columns directly; step i's estimate overlaps step i+1's reads"}


def run_small_config(args, world, rank, which):
    """chain3: R1(A) - R2(A,B) - R3(B), 1e4 rows each, m = 256, d = 5 (launch-latency bound);
    chain8: 8-relation chain, 1e7 Zipf(1.2) rows each, m = 2^20, d = 16 (estimator at scale).
    Times the update of all relations and the estimate separately with CUDA events.
    Parity: chain3 in full against the CPU oracle (every sketch, every row, the median);
    chain8 by identical rows from the three exact arithmetics and one sampled sketch row
    of a two-column relation against the oracle."""
    import numpy as np
    import torch

    import oracle as O
    import paper_2402_15953_gb300 as pkg
    import synth
    from paper_2402_15953_gb300 import build as pkg_build
    pkg_build.build()
    O.build()
    wl = synth.chain3(device="cuda") if which == "chain3" else synth.chain(device="cuda")
    s = pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed)
    s.set_estimator(args.estimator)
    stream = torch.cuda.current_stream()
    reps = args.steps if which == "chain3" else max(3, args.steps // 10)
    doms = declared_domains(args, wl)

    def upd():
        s.reset()
        for k, rel in enumerate(wl.relations):
            s.update(k, rel.cols, domain=doms[k])

    for _ in range(args.warmup):
        upd()
        est = s.estimate()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    up, es = [], []
    clk = ClockSampler(gpu_id())
    clk.start()
    time.sleep(0.2)
    for _ in range(reps):
        e[0].record(stream)
        upd()
        e[1].record(stream)
        est = s.estimate()
        e[2].record(stream)
        torch.cuda.synchronize()
        up.append(e[0].elapsed_time(e[1]))
        es.append(e[1].elapsed_time(e[2]))
    clocks = clk.stop()
    by_arith, arith_ms = {}, {}
    for arith in ("fft64", "ntt", "fused"):
        s.set_estimator(arith)
        s.estimate()                      # scratch and twiddles for this arithmetic
        e[0].record(stream)
        by_arith[arith] = s.estimate()
        e[1].record(stream)
        torch.cuda.synchronize()
        arith_ms[arith] = e[0].elapsed_time(e[1])
    s.set_estimator(args.estimator)
    same = all(x["rows"] == est["rows"] for x in by_arith.values())
    q = O.canonical_query(wl.num_join_attrs, wl.edges)
    co = O.draw_coefficients(wl.hash_seed, wl.d, q.n_comp, len(q.edges))
    threads = os.cpu_count() or 1
    if which == "chain3":
        rels = [(r.cols.cpu().numpy(), None) for r in wl.relations]
        sk = O.sketch_all(q, co, rels, wl.m, threads=threads)
        got = s.counters.cpu().numpy()
        ref = O.estimate(q, sk)
        sk_ok = all(np.array_equal(got[k], sk[k]) for k in range(len(sk)))
        parity = {"sketches_equal_oracle": sk_ok, "rows_equal_oracle": est["rows"] == ref.rows,
                  "median_equal_oracle": est["median"] == ref.median, "arithmetics_identical": same,
                  "exact_join_size": str(O.exact_join_size(q, rels)),
                  "ok": bool(sk_ok and est["rows"] == ref.rows and est["median"] == ref.median and same)}
    else:
        k, row = 3, 5   # a two-column inner relation, one of its 16 rows
        ref = O.sketch_relation(q, co[[row]], k, wl.relations[k].cols.cpu().numpy(), None, wl.m, threads=threads)
        row_ok = bool(np.array_equal(s.counters[k][row].cpu().numpy(), ref[0]))
        parity = {"arithmetics_identical": same, "sampled_sketch_row_equals_oracle": {"relation": k, "row": row,
                                                                                      "equal": row_ok},
                  "ok": bool(same and row_ok)}
    tot = sum(r.n for r in wl.relations)
    ms = statistics.mean(up) + statistics.mean(es)
    line = {"metric": f"{which}: update and estimate time", "value": tot / (ms / 1e3), "unit": "tuples/s",
            "n_gpus": world, "steps": reps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "estimator": args.estimator,
            "config": {"workload": which, "tuples_per_step": tot, "m": wl.m, "d": wl.d},
            "update_us": 1e3 * statistics.mean(up), "estimate_us": 1e3 * statistics.mean(es),
            "estimate_p99_us": 1e3 * percentile(es, 99.0), "estimates_per_s": 1e3 / statistics.mean(es),
            "estimate_ms_by_arithmetic": arith_ms, "median": str(est["median"]), "max_limbs": est["max_limbs"],
            "clocks": clocks, "parity": parity}
    s.close()
    return line


def run_subqueries(args, world, rank):
    """Plan enumeration (Section 3.4): the star join F(K1..K4) x D1..D4 (F 2e7 rows, 4 Zipf(1.1)
    columns over [0, 1e6); D_i 1e6 uniform rows; m = 2^16, d = 9) and all 15 of its connected
    sub-queries (every non-empty subset of the 4 joins).  A step resets the sketches, updates
    every relation and estimates every sub-query.  Family: one sk_family (one pass per relation,
    19 shared view sketches, sub-queries estimated on worker streams).  Against: one
    SketchSet per sub-query (47 relation sketches, each relation updated once per sub-query it
    is in, estimates one after another).  Parity: the full sub-query's rows equal a plain set's,
    and the sub-query of join 0 equals the CPU oracle on two rows."""
    import itertools

    import torch

    import paper_2402_15953_gb300 as pkg
    import synth
    from paper_2402_15953_gb300 import build as pkg_build
    pkg_build.build()
    n_fact, n_dim, k = 20_000_000, 1_000_000, 4
    wl = synth.star(n_fact=n_fact, n_dim=n_dim, k=k, seed=42 + rank, device="cuda")
    subs = [list(c) for size in range(1, k + 1) for c in itertools.combinations(range(k), size)]
    stream = torch.cuda.current_stream()
    total = sum(r.n for r in wl.relations)

    fam = pkg.SketchFamily(wl.num_join_attrs, wl.edges, subs, wl.m, wl.d, wl.hash_seed)
    fam.set_estimator(args.estimator)
    doms = declared_domains(args, wl)

    def fam_step():
        fam.reset()
        for kk, rel in enumerate(wl.relations):
            fam.update(kk, rel.cols, domain=doms[kk])
        return fam.estimate()

    # one SketchSet per sub-query, over the columns that sub-query joins
    naive = []
    for sub in subs:
        dims = [1 + j for j in sub]
        attrs = [len(sub)] + [1] * len(sub)
        edges = [(0, t, 1 + t, 0) for t in range(len(sub))]
        fcols = wl.relations[0].cols[sub].contiguous() if len(sub) < k else wl.relations[0].cols
        fdom = None if doms[0] is None else [doms[0][j] for j in sub]
        naive.append((pkg.SketchSet(attrs, edges, wl.m, wl.d, wl.hash_seed),
                      [fcols] + [wl.relations[dd].cols for dd in dims], [fdom] + [doms[dd] for dd in dims]))
        naive[-1][0].set_estimator(args.estimator)

    def naive_step():
        outs = []
        for sset, cols, cdoms in naive:
            sset.reset()
            for kk, c in enumerate(cols):
                sset.update(kk, c, domain=cdoms[kk])
            outs.append(sset.estimate())
        return outs

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / reps, out

    reps = max(3, args.steps // 3)
    clk = ClockSampler(gpu_id())
    clk.start()
    time.sleep(0.2)
    launches0 = pkg.sk_launch_count()
    fam_ms, fam_out = timed(fam_step, reps)
    launches = (pkg.sk_launch_count() - launches0) // (reps + max(1, args.warmup))
    # update alone (device time)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fam.reset()
        for kk, rel in enumerate(wl.relations):
            fam.update(kk, rel.cols, domain=doms[kk])
    e1.record(stream)
    torch.cuda.synchronize()
    fam_upd_ms = e0.elapsed_time(e1) / reps
    naive_ms, naive_out = timed(naive_step, reps)
    clocks = clk.stop()
    info = fam.info()
    same_full = fam_out[-1]["rows"] == naive_out[-1]["rows"]
    # the oracle for sub-query {join 0} (F's first column with D1; an inner product per row),
    # rows 0 and 1, with the functions Section 3.4's reuse assigns it
    import oracle as O
    O.build()
    q = O.canonical_query(wl.num_join_attrs, wl.edges)
    co = O.draw_coefficients(wl.hash_seed, wl.d, q.n_comp, len(q.edges))
    sq = O.subquery(wl.num_join_attrs, wl.edges, co, subs[0])
    rels = [(r.cols.cpu().numpy(), None) for r in wl.relations]
    sub_rels = O.subquery_relations(sq, rels)
    sk = O.sketch_all(sq.query, sq.coeffs[[0, 1]], sub_rels, wl.m, threads=os.cpu_count() or 1)
    ref = O.estimate(sq.query, sk)
    oracle_ok = fam_out[0]["rows"][:2] == ref.rows
    line = {"metric": "sub-query family: estimates/s of all connected sub-queries with their updates",
            "value": world * len(subs) / (fam_ms / 1e3), "unit": "sub-query estimates/s", "n_gpus": world,
            "steps": reps, "warmup": args.warmup, "ms_per_step": fam_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "estimator": args.estimator,
            "config": {"workload": f"star F(K1..K{k}) {n_fact:.0e} rows Zipf 1.1 over [0,1e6), D_i {n_dim:.0e} "
                                   f"uniform; m=65536, d=9; all {len(subs)} connected sub-queries",
                       "tuples_per_step": total,
                       "key_domains": "undeclared" if args.no_domains else "declared [0, 1e6) per column"},
            "family": {"ms_per_step": fam_ms, "update_ms": fam_upd_ms, "estimate_ms": fam_ms - fam_upd_ms,
                       "views": info["views"], "counter_bytes": info["counter_bytes"],
                       "gpu_launches_per_step": launches},
            "one_set_per_subquery": {"ms_per_step": naive_ms, "relation_sketches": sum(len(c) for _, c, _ in naive)},
            "speedup": naive_ms / fam_ms, "clocks": clocks,
            "parity": {"full_query_rows_equal_plain_set": same_full,
                       "subquery_join0_rows_0_1_equal_oracle": oracle_ok, "ok": bool(same_full and oracle_ok)}}
    for sset, _, _ in naive:
        sset.close()
    fam.close()
    return line


def run_shapes(args, world, rank):
    """Estimator arithmetics beyond the pairwise power-of-two case: (a) Figure 3's query
    (a component of three attributes) with 10^6 Zipf(1.1) rows per relation over [0, 1e6),
    m = 2^16, d = 9; (b) a three-relation chain with 10^6 Zipf(1.2) rows per relation at
    the paper's width m = 10^6, d = 5.  Times one estimate in each exact arithmetic (FP64
    FFT with certificate, GF(q) transform with limbs, Algorithm 3's schedule modulo CRT
    primes) with CUDA events and checks the rows are identical."""
    import torch

    import paper_2402_15953_gb300 as pkg
    import synth
    from paper_2402_15953_gb300 import build as pkg_build
    pkg_build.build()
    stream = torch.cuda.current_stream()
    attrs, edges = synth.fig3_query()
    fig3_rels = [synth.random_relation(1_000_000, [1_000_000] * a, 60 + k, device="cuda", zipf_s=1.1).cols
                 for k, a in enumerate(attrs)]
    ch = synth.chain(r=3, n=1_000_000, m=1_000_000, d=5, device="cuda")
    cases = [("figure3 m=2^16 d=9", attrs, edges, 1 << 16, 9, 42, fig3_rels),
             ("chain3 m=10^6 d=5", ch.num_join_attrs, ch.edges, ch.m, ch.d, ch.hash_seed,
              [r.cols for r in ch.relations])]
    reps = max(3, args.steps // 5)
    out = {}
    for name, at, ed, m, d, seed, rels in cases:
        st = pkg.SketchSet(at, ed, m, d, seed)
        for k, c in enumerate(rels):
            st.update(k, c)
        res = {}
        rows = None
        for arith in ("fft64", "ntt", "fused"):
            st.set_estimator(arith)
            for _ in range(args.warmup):
                est = st.estimate()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                est = st.estimate()
            e1.record(stream)
            torch.cuda.synchronize()
            res[arith] = {"estimate_ms": e0.elapsed_time(e1) / reps, "limbs_or_primes": est["max_limbs"],
                          "limb_bits": est["limb_bits"]}
            rows = est["rows"] if rows is None else rows
            res[arith]["identical_rows"] = est["rows"] == rows
        res["median"] = str(est["median"])
        out[name] = res
        st.close()
    fu = [v["fused"]["estimate_ms"] for v in out.values()]
    line = {"metric": "estimates/s beyond the pairwise power-of-two case (schedule modulo CRT primes)",
            "value": len(fu) * 1e3 / sum(fu), "unit": "estimates/s", "n_gpus": world, "steps": reps,
            "warmup": args.warmup, "ms_per_step": sum(fu), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "shapes: figure3 m=2^16 d=9; chain3 m=10^6 d=5"}, "cases": out}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_workload(args, world, rank, name):
    if name == "batched":
        return run_batched(args, world, rank)
    if name == "serving":
        return run_serving(args, world, rank)
    if name in ("chain3", "chain8"):
        return run_small_config(args, world, rank, name)
    return run_subqueries(args, world, rank)


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload in ("batched", "serving", "chain3", "chain8", "subqueries"):
        line = run_workload(args, world, rank, args.workload)
        if rank == 0:
            print(json.dumps(line), flush=True)
    elif args.workload == "shapes":
        run_shapes(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Seconds per amplitude of random-circuit amplitudes on one GB300 (or N).

Workload (default): Bristlecone-70, depth 1+32+1, seeded circuit by the
prescription of Sec. 1, one random output bitstring per amplitude batch.
The planner builds a contraction tree and slices indices so that every
slice's largest intermediate fits the target; a step contracts a fixed
range of slices (Sec. 1 subtasks) and the time per amplitude is
extrapolated to all 2^k slices: s/amplitude = step time * 2^k / (slices per
step * ranks) / bitstrings. Preprocessing (tree, slicing, plan, bind) is
excluded, as in Sec. 1.

Under torchrun each rank contracts its own slice ranges (no data exchange in
the path) and the per-rank FP64 partial sums are reduced once per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (lattice kind, rows, cols, n_qubits, depth t, circuit seed, log2 target, bitstring seed)
    "bristlecone70_d32": ("bristlecone", 0, 0, 70, 32, 3, 30, 103),
    "grid7x7_d32": ("grid", 7, 7, 49, 32, 2, 24, 102),
    "grid7x7_d40": ("grid", 7, 7, 49, 40, 5, 24, 105),
    "grid4x4_d10": ("grid", 4, 4, 16, 10, 1, 0, 101),
    "bristlecone70_d36": ("bristlecone", 0, 0, 70, 36, 3, 30, 103),
    "bristlecone70_d40": ("bristlecone", 0, 0, 70, 40, 3, 30, 103),
    "bristlecone70_d28": ("bristlecone", 0, 0, 70, 28, 3, 30, 103),
    "bristlecone70_d32_open12": ("bristlecone", 0, 0, 70, 32, 3, 30, 103),
}
# The default mode: scaled split FP16, the tensor-core mode that meets the
# 1e-5 bar against the FP64 oracle on every full-size workload (split BF16 is
# faster per product but misses it on the Bristlecone-70 tree; its error is
# reported beside the others)
DEFAULT_PRECISION = "fp16x3"
# Workload shapes beyond the circuit: exact slice count, bitstrings per step
# and per group (config 2: a tree with 2^10 slices and 64 bitstrings, which
# run as one batch of 64, the batch hyperedge of the network)
WORKLOAD_SHAPE = {"grid7x7_d32": {"k_slices": 10, "bitstrings": 64, "batch_log2": 6},
                  # qubits 0..11 left open: every contraction yields the 4096
                  # amplitudes of all their output assignments (the rest of
                  # the bitstring uniform random)
                  "bristlecone70_d32_open12": {"open_qubits": 12}}
# Table 2 (1449 x 88 vCPU), context only
PAPER_S_PER_AMP = {"bristlecone70_d32": 0.43, "bristlecone70_d36": 5.6, "bristlecone70_d40": 580.7}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bristlecone70_d32",
                    choices=sorted(WORKLOADS) + ["serving_mix", "porter_thomas"])
    ap.add_argument("--amplitudes", type=int, default=200_000,
                    help="porter_thomas: random bitstrings contracted (Sec. 2: 200,000 at depth 1+28+1)")
    ap.add_argument("--queries", type=int, default=96, help="serving_mix: queries in the Poisson stream")
    ap.add_argument("--precision", default="auto", choices=["auto", "c64", "tf32x3", "bf16x3", "fp16x3", "c128"])
    ap.add_argument("--batch-log2", type=int, default=0)
    ap.add_argument("--open-qubits", type=int, default=0,
                    help="leave output qubits 0..N-1 open: 2^N correlated amplitudes per bitstring and contraction")
    ap.add_argument("--slices", type=int, default=0, help="slices per step (0: auto)")
    ap.add_argument("--log2-max", type=int, default=0, help="slicing target (0: workload default)")
    ap.add_argument("--k-slices", type=int, default=0,
                    help="slice exactly this many indices (config 2: 10), instead of slicing to a size target")
    ap.add_argument("--bitstrings", type=int, default=0,
                    help="bitstrings per step (0: 2^batch-log2); groups of 2^batch-log2 are contracted together")
    ap.add_argument("--restarts", type=int, default=16384,
                    help="tree search restarts (untimed preprocessing, run on all host threads)")
    ap.add_argument("--reconfigure", type=int, default=0,
                    help="tree search: exact re-optimisation of windows of this many subtrees (0: off; the "
                         "cheaper Bristlecone-70 tree it finds misses the 1e-5 bar in split TF32)")
    ap.add_argument("--tree-file", default="",
                    help="load the tensor-core modes' tree from this .npy if it exists, else save it there")
    ap.add_argument("--algorithm", default="elimination", choices=["auto", "greedy", "elimination"])
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: time each tensor-core step's launch choices when the plan is bound (untimed "
                         "preprocessing) and keep the fastest; 0: built-in defaults")
    ap.add_argument("--direct-queue", type=int, default=0,
                    help="1: each run of small direct steps between products is one persistent queue launch; "
                         "0: one launch per dependency level (measured no slower)")
    ap.add_argument("--compare-direct", type=int, default=0,
                    help="rounds of an interleaved comparison with the other direct-step launch form (same "
                         "tree, same autotuned products, same slice windows; 0: off)")
    ap.add_argument("--tune-file", default="",
                    help="load the autotuner's choices for the main plan from this .json if it exists, else save "
                         "them there after binding (a profiler run then reproduces the timed run's plan)")
    ap.add_argument("--tree-seed", type=int, default=7)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the same workload in the other precision modes")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    return ap.parse_args()


def make_circuit_spec(w):
    import tz_inputs as ti
    kind, rows, cols, nq, t, seed, _, _ = WORKLOADS[w]
    lat = ti.grid(rows, cols) if kind == "grid" else ti.bristlecone(nq)
    return ti.circuit_to_spec(lat.n_qubits, ti.generate_circuit(lat, t, seed)), lat.n_qubits


_TREES = {}


def build_plan(tz, spec, args, precision, stream, device, log2_max, max_rows=0):
    circ = tz.tz_circuit_from_spec(spec)
    net = tz.tz_network_from_circuit(circ, args.batch_log2, tuple(range(args.open_qubits)))
    t0 = time.perf_counter()
    # the time model that scores trees tells the CUDA-core modes from the
    # tensor-core ones only, so the three tensor-core modes share one search
    tc_mode = precision not in ("c64", "c128")
    key = (spec, precision if not tc_mode else "tensor-core", log2_max, args.open_qubits)
    cache = args.tree_file if tc_mode else ""
    if key not in _TREES and cache and os.path.exists(cache):
        _TREES[key] = np.load(cache)
    if key not in _TREES:
        _TREES[key] = tz.tz_path_greedy(net, restarts=args.restarts, seed=args.tree_seed,
                                        log2_max_intermediate=log2_max, precision=precision,
                                        algorithm=args.algorithm, reconfigure=args.reconfigure).pairs()
        if cache:
            np.save(cache, _TREES[key])
    tree = tz.tz_tree_from_pairs(net, _TREES[key])
    if args.k_slices > 0:
        sliced = tz.tz_slice_select(net, tree, 1, args.k_slices)
    else:
        sliced = tz.tz_slice_select(net, tree, log2_max, 40) if log2_max > 0 else []
    plan = tz.tz_plan_create(net, tree, sliced, precision=precision, device=device, stream=stream, use_graph=True,
                             max_bitstrings=max_rows or args.bitstrings or 1 << max(args.batch_log2, 0),
                             autotune=bool(args.autotune), direct_queue=bool(args.direct_queue))
    prep_s = time.perf_counter() - t0
    return plan, sliced, prep_s


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), \
            d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 1900.0, 1700.0, 2070.0, "fallback"


# DRAM bytes (read + write) per tensor-core product launch, averaged over the
# 13 product launches of one step, from one ncu capture of the bench command
# itself with its autotuned choices fixed by --tune-file
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass;
# profiles/launch_list_bristlecone70_d32_fp16x3.md), keyed by (precision,
# workload). A mode or workload without an up-to-date capture reports null.
TC_DRAM_BYTES_PER_LAUNCH = {("fp16x3", "bristlecone70_d32"): 2.0430e9}


def plan_roofline(plan, precision, ms_per_group):
    """Plan-level roofline: T_roof = sum over the per-slice steps of
    max(hardware flops / peak of the mode, algorithmic bytes / HBM), plus the
    permutes (read + write at HBM speed); its ratio to the measured time of one
    group (one slice, one bitstring batch)."""
    hbm, bf16, _, sm_mhz, src = measured_peaks()
    simt = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    tc = {"tf32x3": bf16 * 1.1 / 2.25, "bf16x3": bf16, "fp16x3": bf16}.get(precision)
    fp64 = simt / 64   # GB300 FP64 CUDA-core rate, 1/64 of FP32
    d = json.loads(plan.describe())
    size = [1 << len(t["lay"]) for t in d["tensors"]]
    lay = [set(t["lay"]) for t in d["tensors"]]
    esz = 16 if precision == "c128" else 8
    t = 0.0
    for st in d["steps"]:
        if not st["var"]:
            continue
        a, b, c = st["a"], st["b"], st["c"]
        nbytes = esz * (size[a] + size[b] + size[c])
        if st["gemm"]:
            fl = 8.0 * st["batch"] * st["M"] * st["N"] * st["K"]
        else:
            fl = 8.0 * (1 << len(lay[a] | lay[b]))
        if st["gemm"] and st["tc"] and not st.get("tc_simt") and tc:
            tf = 3 * fl / (tc * 1e12)
        else:
            tf = fl / ((fp64 if precision == "c128" else simt) * 1e12)
        t += max(tf, nbytes / (hbm * 1e9))
    for it in d["var_items"]:
        if it[0] == 2:  # permute: read and write the tensor
            t += 2 * esz * size[it[1]] / (hbm * 1e9)
    return {"t_roof_ms": t * 1e3, "t_measured_ms": ms_per_group, "frac": t * 1e3 / ms_per_group,
            "peaks": f"{src}: HBM {hbm:.0f} GB/s, tensor {tc or 0:.0f} TF/s, FP32 {simt:.1f} TF/s"}


def top_profiled_items(plan, precision, n=10):
    """The n most expensive launch items of the profiled groups: kind, GEMM
    shape, ms per group, achieved rates and the item's own roofline time
    (max of algorithmic bytes / HBM peak and issued flops / its unit's peak)."""
    hbm, tc, _, _, _ = measured_peaks()
    if precision == "tf32x3":
        tc *= 1.1 / 2.25
    steps = json.loads(plan.describe())["steps"]
    items = plan.profile_items()
    groups = max([it["launches"] for it in items if it["kind"] == "leaves"] or [1])
    out = []
    for i, it in enumerate(items):
        if it["ms"] <= 0:
            continue
        ms = it["ms"] / groups
        rate = tc * (3 if precision in ("tf32x3", "bf16x3", "fp16x3") and it["kind"] == "gemm_tc" else 1)
        if it["kind"] != "gemm_tc":
            rate = 80.5 if precision != "c128" else 1.3   # CUDA-core FP32 (FP64) peak, TF/s
        issued = it["flops"] * (3 if it["kind"] == "gemm_tc" and precision in ("tf32x3", "bf16x3", "fp16x3") else 1)
        t_roof = max(it["bytes"] / (hbm * 1e9), issued / (tc * 1e12 if it["kind"] == "gemm_tc" else rate * 1e12))
        e = {"item": i, "kind": it["kind"], "ms_per_group": ms, "gbs": it["bytes"] / (ms / 1e3) / 1e9,
             "useful_tflops": it["flops"] / (ms / 1e3) / 1e12, "roofline_ms": t_roof * 1e3,
             "frac": t_roof * 1e3 / ms}
        if it["step"] >= 0:
            st = steps[it["step"]]
            e["shape"] = {"batch": st["batch"], "M": st["M"], "N": st["N"], "K": st["K"],
                          "out": "row-major" if st["row_major"] else "scatter",
                          "choice": {1: "simt", 2: "stream"}.get(st["tc_simt"],
                                                                 ("pairs" if st["tc_pair"] == 1 else "single")
                                                                 if st["tc"] else "simt")}
        out.append(e)
    out.sort(key=lambda e: -e["ms_per_group"])
    return out[:n]


def roofline(prof, precision, workload):
    """Dominant kernel kind of the profiled pass and its roofline position."""
    hbm, bf16, bf16_s, sm_mhz, src = measured_peaks()
    kinds = {k: v for k, v in prof.items() if v["launches"] > 0}
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    d = kinds[dom]
    total_ms = sum(v["ms"] for v in kinds.values())
    sec = d["ms"] / 1e3
    fp32_alu_tflops = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12   # FFMA lanes x 2 flops x max clock
    out = {"kernel": dom, "launches": d["launches"], "share_of_step": d["ms"] / total_ms if total_ms else None,
           "traffic": None}
    if dom == "gemm_tc":
        ratio = {"tf32x3": 1.1 / 2.25, "bf16x3": 1.0, "fp16x3": 1.0}[precision]   # nominal dense : BF16
        peak = bf16 * ratio
        out.update(bound="tensor", unit="TFLOP/s", achieved=d["flops"] / sec / 1e12, peak=peak,
                   peak_source=f"{src} bf16 x nominal {precision[:4]}/bf16 ratio",
                   issued_tflops=3 * d["flops"] / sec / 1e12)
        if (precision, workload) in TC_DRAM_BYTES_PER_LAUNCH:
            out["traffic"] = TC_DRAM_BYTES_PER_LAUNCH[(precision, workload)]
            out["traffic_note"] = ("DRAM bytes per product launch, mean over one step's launches, from an ncu "
                                   "capture of this command; algorithmic bytes per launch: algorithmic_bytes")
        else:
            out["traffic_note"] = "null: no ncu capture of this mode and workload with the current kernel"
        out["algorithmic_bytes"] = d["bytes"] / d["launches"]
    elif dom == "gemm_simt":
        out.update(bound="alu", unit="TFLOP/s", achieved=d["flops"] / sec / 1e12, peak=fp32_alu_tflops,
                   peak_source="152 SMs x 128 FP32 lanes x 2 flops x max SM clock")
    else:
        out.update(bound="hbm", unit="GB/s", achieved=d["bytes"] / sec / 1e9, peak=hbm, peak_source=f"{src} copy")
    out["frac"] = out["achieved"] / out["peak"]
    out["achieved_bytes_gbs"] = d["bytes"] / sec / 1e9
    out["per_kind_ms"] = {k: round(v["ms"], 3) for k, v in kinds.items()}
    return out


# Largest factor (log2 entries) the path-sum oracle may create when timed
ORACLE_MAX_LOG2 = 25


def oracle_segments(tz, spec, pairs, batch_log2=0, cap=18, open_qubits=0):
    """Sliced segments for the CPU baseline: the GPU tree, sliced further to
    a 2^cap intermediate cap, so that one slice is a bounded unit of oracle
    work (the sum over all slices is the amplitude, Sec. 1). Open output
    qubits are never sliced, so the segments also slice the closed circuit."""
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), batch_log2, tuple(range(open_qubits)))
    tree = tz.tz_tree_from_pairs(net, pairs)
    sl = tz.tz_slice_select(net, tree, cap, 40)
    return [net.index_info(e) for e in sl]


def cpu_oracle_sample(spec, segs, bits, budget_s):
    """Time the FP64 path-sum oracle, as it stands, on a bounded sample of
    the workload: the partial amplitudes of slices 0, 1, 2, ... of the given
    slicing until the budget is spent; extrapolate to all 2^k slices of one
    amplitude. Cores: the BLAS threads numpy's einsum runs on."""
    from oracle import pathsum
    t0 = time.perf_counter()
    c = pathsum.SegmentContractor(spec, sliced=segs, max_log2=ORACLE_MAX_LOG2)
    setup = time.perf_counter() - t0
    k = len(segs)
    done = 0
    t1 = time.perf_counter()
    while done < (1 << k):
        c.partial(bits, done)
        done += 1
        if time.perf_counter() - t1 > budget_s:
            break
    el = time.perf_counter() - t1
    s_per_amp = el / done * (1 << k)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": s_per_amp, "unit": "s/amplitude", "cores": cores, "kind": "oracle",
            "sample": f"{done} of 2^{k} slice partials of one amplitude by the FP64 path-sum oracle (its own "
                      f"elimination order, largest factor 2^{c.width - 1}, {len(c.extra)} extra segments of its own), "
                      f"{el:.1f} s, extrapolated x 2^{k}/{done}; oracle setup {setup:.1f} s"}


def run_serving(args):
    """Continuous-batching server over resident plans: grids 4x4..7x7 at
    depths 1+16+1, 1+24+1, 1+32+1; queries of 1..256 bitstrings on uniformly
    chosen circuits. The saturation rate is measured on a burst; then a Poisson
    stream at 0.8x that rate gives the sustained amplitudes/s and the server's
    p50/p99 query latency (submit to completion)."""
    import torch
    import paper_1907_11217_gb300 as tz
    import tz_inputs as ti
    precision = args.precision if args.precision != "auto" else DEFAULT_PRECISION
    torch.cuda.set_device(0)
    plans = []
    t0 = time.perf_counter()
    for (r, c) in ((4, 4), (5, 5), (6, 6), (7, 7)):
        for t in (16, 24, 32):
            spec = ti.circuit_to_spec(r * c, ti.generate_circuit(ti.grid(r, c), t, 4))
            net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 6)
            tree = tz.tz_path_greedy(net, restarts=16, seed=7, log2_max_intermediate=26, precision=precision,
                                     algorithm="elimination")
            sliced = tz.tz_slice_select(net, tree, 26, 40)
            plan = tz.tz_plan_create(net, tree, sliced, precision=precision, max_bitstrings=256, use_graph=True)
            plan.bind()
            plans.append((plan, r * c, f"{r}x{c}_d{t}", len(sliced)))
    prep_s = time.perf_counter() - t0
    scratch = max(p[0].stats()["scratch_bytes"] for p in plans)
    srv = tz.tz_server_create(arena_bytes=4 * scratch + (1 << 20), max_inflight=4)
    rng = np.random.default_rng(4)

    def make_queries(n, seed):
        q = []
        for i in range(n):
            j = int(rng.integers(len(plans)))
            nb = int(rng.integers(1, 257))
            q.append((j, ti.random_bitstrings(plans[j][1], nb, seed + i)))
        return q

    def drain(tickets, limit_s=600):
        done = {}
        t_end = time.perf_counter() + limit_s
        while len(done) < len(tickets) and time.perf_counter() < t_end:
            for t in tickets:
                if t not in done and srv.poll(t) is not None:
                    done[t] = time.perf_counter()
        return done

    # warm-up: every plan once
    drain([srv.submit(p[0], ti.random_bitstrings(p[1], 4, 7)) for p in plans])
    # saturation: a burst of queries submitted at once
    burst = make_queries(args.queries // 2, 10_000)
    t0 = time.perf_counter()
    tk = [srv.submit(plans[j][0], b) for j, b in burst]
    drain(tk)
    sat = sum(len(b) for _, b in burst) / (time.perf_counter() - t0)
    # Poisson stream at 0.8x saturation (queries per second from the mean query size)
    stream = make_queries(args.queries, 20_000)
    mean_b = np.mean([len(b) for _, b in stream])
    rate_q = 0.8 * sat / mean_b
    gaps = rng.exponential(1.0 / rate_q, size=len(stream))
    srv.close()
    srv = tz.tz_server_create(arena_bytes=4 * scratch + (1 << 20), max_inflight=4)  # stream-only statistics
    t0 = time.perf_counter()
    tickets, t_next, t_sub, done = [], t0, {}, {}
    for (j, b), g in zip(stream, gaps):
        t_next += g
        while time.perf_counter() < t_next:
            # completions are polled while the next arrival is awaited, so
            # each query's latency ends when it finished, not when polled
            for t in tickets:
                if t not in done and srv.poll(t) is not None:
                    done[t] = time.perf_counter()
        t = srv.submit(plans[j][0], b)
        t_sub[t] = time.perf_counter()
        tickets.append(t)
    done.update(drain([t for t in tickets if t not in done]))
    elapsed = max(done.values()) - t0
    p50, p99, n_done = srv.latency()
    amps = sum(len(b) for _, b in stream)
    # latency by class: queries on unsliced plans (one slice) and on sliced
    # ones (hundreds of slices: long by their own work)
    by_class = {}
    for t, (j, b) in zip(tickets, stream):
        cls = "sliced" if plans[j][3] > 0 else "unsliced"
        by_class.setdefault(cls, []).append((done[t] - t_sub[t]) * 1e3)
    class_lat = {c: {"queries": len(v), "p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}
                 for c, v in by_class.items()}
    line = {"metric": "amplitudes/s (serving mix, Poisson arrivals at 0.8x saturation)",
            "value": amps / elapsed, "unit": "amplitudes/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": precision, "data": "synthetic (seeded circuits by the Sec. 1 prescription, uniform bitstrings)",
            "config": {"workload": "serving_mix", "circuits": [p[2] for p in plans], "slices": [p[3] for p in plans],
                       "bitstrings_per_query": "uniform 1..256", "queries": len(stream),
                       "arrival_rate_qps": rate_q, "saturation_amps_per_s": sat, "plans_prep_s": prep_s,
                       "max_inflight": 4},
            "latency_ms": {"p50": p50 * 1e3, "p99": p99 * 1e3, "queries": n_done, "by_class": class_lat},
            "vs_baseline": None}
    print(json.dumps(line))
    srv.close()


def porter_thomas_stats(np_vals):
    """Sec. 2: for a random circuit deep enough, x = N p (N = 2^n, p = |a|^2)
    over uniform random bitstrings follows the density e^-x. Moments, the
    fraction above 1, a histogram against the expected counts, the chi-square
    statistic and the Kolmogorov-Smirnov distance to 1 - e^-x."""
    x = np.asarray(np_vals, dtype=np.float64)
    m = len(x)
    edges = np.concatenate([np.arange(0.0, 8.0, 0.5), [np.inf]])
    counts, _ = np.histogram(x, bins=edges)
    expected = m * (np.exp(-edges[:-1]) - np.exp(-edges[1:]))
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    xs = np.sort(x)
    cdf = 1.0 - np.exp(-xs)
    ks = float(max(np.max(np.arange(1, m + 1) / m - cdf), np.max(cdf - np.arange(m) / m)))
    return {"amplitudes": m, "mean": float(x.mean()), "mean_tolerance_3sigma": 3.0 / math.sqrt(m),
            "second_moment": float((x ** 2).mean()), "second_moment_expected": 2.0,
            "frac_above_1": float((x > 1).mean()), "frac_above_1_expected": math.exp(-1.0),
            "ks_distance": ks, "ks_critical_1pct": 1.63 / math.sqrt(m),
            "chi2": chi2, "chi2_dof": len(counts) - 1,
            "histogram": {"edges": [float(e) for e in edges[:-1]] + ["inf"], "counts": [int(c) for c in counts],
                          "expected": [round(float(e), 1) for e in expected]}}


def run_porter_thomas(args):
    """Sec. 2, the Porter-Thomas check at scale: amplitudes of 200,000
    uniform random bitstrings of a Bristlecone-70 depth 1+28+1 circuit (Table 2
    measures this configuration at 0.04 s per amplitude), contracted in calls
    of up to 4096 bitstrings through the device entry point; seconds per
    amplitude over all of them, and the distribution of N p against e^-x."""
    import torch
    import paper_1907_11217_gb300 as tz
    import tz_inputs as ti
    precision = args.precision if args.precision != "auto" else DEFAULT_PRECISION
    torch.cuda.set_device(0)
    workload = "bristlecone70_d28"
    spec, nq = make_circuit_spec(workload)
    log2_max = args.log2_max or WORKLOADS[workload][6]
    stream = torch.cuda.Stream()
    chunk = 4096
    args.batch_log2 = max(args.batch_log2, 0)
    plan, sliced, prep_s = build_plan(tz, spec, args, precision, stream, 0, log2_max, max_rows=chunk)
    st = plan.stats()
    plan.bind()
    bits = ti.random_bitstrings(nq, args.amplitudes, 28_200)
    d_bits = torch.from_numpy(bits).cuda()
    d_out = torch.empty(2 * args.amplitudes, dtype=torch.float64, device="cuda")

    def run_all():
        for lo in range(0, args.amplitudes, chunk):
            hi = min(args.amplitudes, lo + chunk)
            tz.tz_contract_amplitudes_device(plan, d_bits[lo:hi], d_out[2 * lo:2 * hi])

    # warm-up on the first chunk (captures the graph), then all amplitudes
    tz.tz_contract_amplitudes_device(plan, d_bits[:min(chunk, args.amplitudes)], d_out)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        run_all()
        ev1.record(stream)
        torch.cuda.synchronize()
    tz.tz_plan_status(plan)
    sec = ev0.elapsed_time(ev1) / 1e3
    amps = d_out.cpu().numpy().view(np.complex128)
    stats = porter_thomas_stats(np.abs(amps) ** 2 * 2.0 ** nq)
    line = {"metric": metric_name("bristlecone70_d28_porter_thomas"), "value": sec / args.amplitudes,
            "unit": "s/amplitude", "n_gpus": 1, "higher_is_better": False, "dtype": precision,
            "data": "synthetic (seeded circuit by the Sec. 1 prescription, uniform random bitstrings)",
            "config": {"workload": "bristlecone70_d28_porter_thomas", "n_qubits": nq, "depth": "1+28+1",
                       "amplitudes": args.amplitudes, "bitstrings_per_call": chunk,
                       "batch_bitstrings_per_group": 1 << args.batch_log2, "k_sliced": len(sliced),
                       "tree_restarts": args.restarts, "preprocessing_s": prep_s,
                       "flops_per_amplitude": st["flops_per_group"] * 2.0 ** st["k"] / 2 ** args.batch_log2},
            "total_s": sec, "contraction_tflops": st["flops_per_group"] * 2.0 ** st["k"] / 2 ** args.batch_log2
            * args.amplitudes / sec / 1e12,
            "vs_baseline": (sec / args.amplitudes) / 0.04, "paper_s_per_amplitude": 0.04,
            "porter_thomas": stats, "clocks": clk.summary()}
    print(json.dumps(line))


def metric_name(workload):
    """The metric string both arms print (the driver compares them)."""
    return f"sec/amplitude ({workload})"


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import tz_inputs as ti
    import paper_1907_11217_gb300 as tz
    spec, nq = make_circuit_spec(args.workload)
    log2_max = args.log2_max or WORKLOADS[args.workload][6]
    circ = tz.tz_circuit_from_spec(spec)
    net = tz.tz_network_from_circuit(circ, 0)
    # the same tree as the GPU arm's tensor-core modes (host preprocessing,
    # untimed), sliced further into oracle-sized slices
    tree = tz.tz_path_greedy(net, restarts=args.restarts, seed=args.tree_seed, log2_max_intermediate=log2_max,
                             precision="bf16x3", algorithm=args.algorithm)
    segs = oracle_segments(tz, spec, tree.pairs())
    bits = ti.random_bitstrings(nq, 1, WORKLOADS[args.workload][7])[0]
    per = max(2.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(spec, segs, bits, per)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.median(x["value"] for x in vals)
    line = {"impl": "reference", "metric": metric_name(args.workload), "value": v, "unit": "s/amplitude",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "oracle_slices_log2": len(segs)},
            "cpu_baseline": {"kind": "oracle", "cores": vals[-1]["cores"], "sample": vals[-1]["sample"], "value": v,
                             "unit": "s/amplitude"},
            "e2e": {"value": v, "unit": "s/amplitude", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    for key, v in WORKLOAD_SHAPE.get(args.workload, {}).items():
        if not getattr(args, key):
            setattr(args, key, v)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "serving_mix":
        run_serving(args)
        return
    if args.workload == "porter_thomas":
        run_porter_thomas(args)
        return
    import torch
    import paper_1907_11217_gb300 as tz
    import tz_inputs as ti

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
        # every rank searches the same tree (the search is deterministic and
        # independent of its thread count): share the host's cores among the
        # ranks of this node instead of oversubscribing them
        if "TZ_PATH_THREADS" not in os.environ:
            per_node = int(os.environ.get("LOCAL_WORLD_SIZE", str(world)))
            os.environ["TZ_PATH_THREADS"] = str(max(1, (os.cpu_count() or 1) // max(1, per_node)))
    torch.cuda.set_device(local)
    device = local

    precision = args.precision
    if precision == "auto":
        precision = DEFAULT_PRECISION if tz._lib.lib() and _tc_available(tz) else "c64"
    spec, nq = make_circuit_spec(args.workload)
    log2_max = args.log2_max or WORKLOADS[args.workload][6]
    stream = torch.cuda.Stream(device=device)
    plan, sliced, prep_s = build_plan(tz, spec, args, precision, stream, device, log2_max)
    st = plan.stats()
    tune_loaded = bool(args.tune_file) and os.path.exists(args.tune_file)
    if tune_loaded:
        for e in json.load(open(args.tune_file)):
            tz.tz_tune_preset(precision, *e)
    plan.bind()
    if args.tune_file and not tune_loaded:
        d = json.loads(plan.describe())
        json.dump([[s["batch"], s["M"], s["N"], s["K"], 0 if s["row_major"] else 1, s["tc_pair"], s["tc_ksplit"],
                    s["tc_simt"]] for s in d["steps"]
                   if s["var"] and s["gemm"] and (s["tc"] or (s["K"] <= 32 and not s["skinny"]))],
                  open(args.tune_file, "w"))
    plan_bind_ms = plan.stats()["bind_ms"]
    n_tuned = plan.stats()["n_tuned_steps"]
    st = plan.stats()   # the launch count follows the autotuned choices
    k = len(sliced)
    n_slices = 1 << k
    B = args.bitstrings or 1 << args.batch_log2
    bits = ti.random_bitstrings(nq, B, WORKLOADS[args.workload][7] + rank)
    d_bits = torch.from_numpy(bits).to(f"cuda:{device}")
    A = B << args.open_qubits   # amplitudes per contraction of the B bitstrings
    d_out = torch.zeros(2 * A, dtype=torch.float64, device=f"cuda:{device}")

    # ranks split the slices of one amplitude; with fewer slices than ranks
    # (the default tree has none) they are replicas instead: each contracts
    # whole amplitudes of its own bitstrings, and nothing is reduced
    replicas = dist and n_slices < world
    from paper_1907_11217_gb300 import shard

    # slices per step: ~3 s of estimated work (a fixed 2^12 when that is smaller), at least 1
    S = args.slices
    if S <= 0:
        plan.set_slice_range(0, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tz.tz_contract_amplitudes_device(plan, d_bits, d_out)
        stream.synchronize()
        one = time.perf_counter() - t0
        S = int(max(1, min(4096, n_slices // (1 if replicas else world), 3.0 / max(one, 1e-6))))
    # a power of two that divides the slice range: every step's window is whole
    S = shard.window_size(n_slices, 1 if replicas else world, S)

    def slice_range(step):
        if replicas:
            return shard.step_window(n_slices, 1, 0, S, step)
        return shard.step_window(n_slices, world, rank, S, step)

    def one_step(step, reduce=True):
        lo, hi = slice_range(step)
        plan.set_slice_range(lo, hi)
        tz.tz_contract_amplitudes_device(plan, d_bits, d_out)
        if dist and reduce and not replicas:
            with torch.cuda.stream(stream):
                shard.reduce_partials(d_out)

    for w in range(args.warmup):
        one_step(w)
    torch.cuda.synchronize()
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(device) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            one_step(args.warmup + i)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device=f"cuda:{device}")
        td.all_reduce(t, op=td.ReduceOp.MAX)
        ms = float(t.item())
    # slices of one amplitude per step, all ranks together; replicas each
    # contract their own amplitudes
    slices_per_step = S * world
    s_per_amp = ms / 1e3 * n_slices / slices_per_step / A
    chunks = -(-B // (1 << args.batch_log2))   # groups of 2^batch_log2 bitstrings per slice
    flops_step = st["flops_per_group"] * slices_per_step * chunks
    tflops = flops_step / (ms / 1e3) / 1e12

    # end to end through the host API: bitstrings in from host memory, FP64
    # amplitudes back to host memory, every step
    plan_e2e = plan
    e2e_times = []
    for i in range(max(1, args.steps)):
        lo, hi = slice_range(args.warmup + i)
        plan_e2e.set_slice_range(lo, hi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tz.tz_contract_amplitudes(plan_e2e, bits)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_times) * n_slices / slices_per_step / A

    # per-kernel profile of one more step (events around every launch)
    plan.profile_enable(True)
    one_step(args.warmup + args.steps, reduce=False)
    prof = plan.profile()
    top_items = top_profiled_items(plan, precision)
    plan.profile_enable(False)
    rl = roofline(prof, precision, args.workload)
    rl["plan_roofline"] = plan_roofline(plan, precision, ms / S / chunks)
    per_launch = {k: v["launches"] for k, v in prof.items()}
    per_kind_ms = {k: v["ms"] for k, v in prof.items()}
    launches_per_call = 1 + S * chunks * st["n_launches_per_group"]

    # the other direct-step launch form on the same tree and slice windows,
    # interleaved step by step with this plan (the autotuner's cached choices
    # make the products identical), so that drifts in clock and power hit both
    direct_compare = None
    if args.compare_direct > 0 and world == 1:
        p3, _, _ = build_plan(tz, spec, argparse.Namespace(**{**vars(args), "direct_queue": 1 - args.direct_queue}),
                              precision, stream, device, log2_max)
        p3.bind()
        t_one, t_other = [], []
        for r in range(args.compare_direct):
            for pl, acc in ((plan, t_one), (p3, t_other)):
                lo, hi = slice_range(r)
                pl.set_slice_range(lo, hi)
                tz.tz_contract_amplitudes_device(pl, d_bits, d_out)   # warm: the window's first run
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tz.tz_contract_amplitudes_device(pl, d_bits, d_out)
                e1.record(stream)
                torch.cuda.synchronize()
                acc.append(e0.elapsed_time(e1) / (hi - lo))
        names = ("queue", "per dependency level") if args.direct_queue else ("per dependency level", "queue")
        direct_compare = {"ms_per_slice": {names[0]: statistics.median(t_one), names[1]: statistics.median(t_other)},
                          "launches_per_slice": {names[0]: st["n_launches_per_group"],
                                                 names[1]: p3.stats()["n_launches_per_group"]},
                          "rounds": args.compare_direct, "slices_per_round": S}
        p3.close()

    # the same workload in the other modes (split precision against complex64),
    # each with its own tree and plan, timed over the same slice windows
    compare = None
    segs = plan.sliced_segments()
    if world == 1 and not args.no_compare:
        compare = {}
        plan.close()  # free its workspace before the other plans bind theirs
        for other in ("c64", "bf16x3", "fp16x3", "tf32x3"):
            if other == precision:
                continue
            p2, _, _ = build_plan(tz, spec, args, other, stream, device, log2_max)
            st2 = p2.stats()
            p2.bind()
            k2 = st2["k"]
            n2 = 1 << k2
            S2 = max(1, min(S, n2))

            def step2(i):
                lo = (i * S2) % n2
                p2.set_slice_range(lo, min(n2, lo + S2))
                tz.tz_contract_amplitudes_device(p2, d_bits, d_out)

            step2(0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(2):
                step2(1 + i)
            e1.record(stream)
            torch.cuda.synchronize()
            ms2 = e0.elapsed_time(e1) / 2
            compare[other] = {"s_per_amplitude": ms2 / 1e3 * n2 / S2 / A,
                              "contraction_tflops": st2["flops_per_group"] * S2 / (ms2 / 1e3) / 1e12,
                              "k_sliced": k2}
            p2.close()

    if rank != 0:
        if dist:
            td.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        tc_key = (spec, "tensor-core" if precision not in ("c64", "c128") else precision, log2_max,
                  args.open_qubits)
        cpu = cpu_oracle_sample(spec, oracle_segments(tz, spec, _TREES[tc_key], args.batch_log2,
                                                      open_qubits=args.open_qubits), bits[0], args.cpu_seconds)
    paper = PAPER_S_PER_AMP.get(args.workload)
    line = {
        "metric": metric_name(args.workload),
        "value": s_per_amp, "unit": "s/amplitude", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": (s_per_amp / paper) if paper else None,
        "dtype": precision, "data": "synthetic (seeded circuit by the Sec. 1 prescription, uniform random bitstrings)",
        "config": {"workload": args.workload, "n_qubits": nq, "depth": f"1+{WORKLOADS[args.workload][4]}+1",
                   "batch_bitstrings": B, "open_qubits": args.open_qubits, "amplitudes_per_step": A,
                   "k_sliced": k, "slices_total": n_slices,
                   "slices_per_step": slices_per_step, "log2_max_intermediate": st["max_log2"],
                   "tree_restarts": args.restarts, "tree_reconfigure": args.reconfigure, "preprocessing_s": prep_s,
                   "l2": "intermediates larger than L2" if st["max_log2"] >= 25 else "working set may fit L2",
                   "parallelism": f"replicas x{world}" if replicas else f"slices x{world}",
                   "extrapolation": f"step time x 2^{k} / {slices_per_step} slices per step / {A} amplitudes"},
        "contraction_tflops": tflops,
        "plan": {"flops_per_slice": st["flops_per_group"], "bytes_per_slice": st["bytes_per_group"],
                 "permute_bytes_per_slice": st["permute_bytes_per_group"], "steps": st["n_steps"],
                 "gemm_steps": st["n_gemm_steps"], "launches_per_slice": st["n_launches_per_group"],
                 "workspace_gb": st["workspace_bytes"] / 1e9,
                 "const_steps": st["n_const_steps"], "const_flops": st["const_flops"],
                 "bind_ms": plan_bind_ms, "autotuned_steps": n_tuned,
                 "direct_launch": "queue" if args.direct_queue else "per dependency level"},
        "e2e": {"value": e2e_s, "unit": "s/amplitude", "h2d_bytes_per_step": int(bits.nbytes),
                "d2h_bytes_per_step": 16 * A},
        "roofline": rl,
        "compare": compare,
        "direct_compare": direct_compare,
        "cpu_baseline": cpu,
        "gpu_launches": args.steps * launches_per_call,
        "profiled_launches_per_kind": per_launch,
        "profiled_ms_per_kind": per_kind_ms,
        "profiled_top_items": top_items,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    if dist:
        td.destroy_process_group()


def _tc_available(tz):
    try:
        return tz.tz_op_cgemm_scratch_bytes("tf32x3", 1, 1024, 64, 64) >= 0
    except tz.TzError:
        return False


if __name__ == "__main__":
    main()

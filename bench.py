#!/usr/bin/env python3
"""Benchmark of the GB300 Born-series path: Born terms/s on the 2048^2
absorbing/dispersive tissue workload (4096^2 padded FFT convolution).

A step is one pass of the whole hot path over one synthetic problem: build V
from c(x), alpha(x) (tbs_set_medium), deposit the 128-element focused array
(tbs_set_sources), and run the series to the FP64 residual 1e-6 (<= 64 terms)
with the device-side stop test (tbs_solve).  The Ghat plan is built once per
(N, k0) before timing and reported as plan_ms.

value  = N^2 x terms summed / device time, inputs resident in HBM, L2 flushed
         (256 MiB write) between timed steps, max over ranks;
e2e    = the same metric with the inputs in pinned HOST memory: the H2D copy
         of c and alpha, the host amplitudes and the D2H read of psi and the
         info records are inside each timed step.

The same JSON line carries, beside the contract's keys, the roofline of the
dominant kernel (live CUDA-event times; DRAM traffic from the committed ncu
summary when it was taken on the current kernel sources), the oracle timed on
a bounded sample (cpu_baseline), and extras: the cuFFT baseline, the
broadband sweep batched vs one-at-a-time plus its time signal, the adjoint
(stored and checkpointed terms), the 2048^2 second harmonic, the paper's
periodic 4096^2 runs (Table 2, and the 1100 m/s cylinder with the convergent
Born series preconditioner) and its five-harmonic nonlinear run.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --cpu-baseline-configs      (the oracle on every workload)
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Born terms/s (grid pts×terms/s) at 2048² c64, % HBM peak; batched & adjoint vs plain"
UNIT = "grid-pt*terms/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cfg2", choices=["cfg1", "cfg2", "cfg3"])
    ap.add_argument("--n", type=int, default=None, help="override the grid side (smaller case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paper-case", default=None,
                    help="only run one of the paper's periodic 4096^2 cases (e.g. homogeneous) and exit; "
                         "with --no-graph its kernels launch from the host (for profiling)")
    ap.add_argument("--cpu-baseline-configs", action="store_true",
                    help="only time the oracle on every workload (host cores, a few minutes) and exit")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the cuFFT-baseline, batched-sweep and adjoint comparisons")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only warm-up and timed steps (for profiler launch lists)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the term loop on the stream instead of the cached graph (ncu cannot "
                         "profile kernels of graphs that hold conditional nodes); same kernels, and "
                         "max_terms gated launches per kernel")
    return ap.parse_args()


def make_workload(args):
    from paper_2507_13754_gb300 import workloads as W
    if args.workload == "cfg1":
        return W.cfg1(**({"n": args.n} if args.n else {}))
    if args.workload == "cfg3":
        return W.cfg3(**({"n": args.n} if args.n else {}))
    return W.cfg2(**({"n": args.n} if args.n else {}))


def describe(w):
    return {"cfg1": "2D TBS lossless disk, %d^2 padded to %d^2, 1 MHz, 32 emitters, 24 terms",
            "cfg2": "2D TBS absorbing/dispersive tissue, %d^2 padded to %d^2, 5 MHz, 128-element "
                    "focused array, residual 1e-6 (<=64 terms)",
            "cfg3": "2D TBS nonlinear medium fundamental, %d^2 padded to %d^2, 2 MHz, 64 elements, "
                    "residual 1e-6"}[w.name.split("_")[0]]


def source_hash():
    from paper_2507_13754_gb300 import build
    return build.source_hash()


def measured_peak():
    try:
        j = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel, workload_name):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        j = json.load(open(path))
        e = j[kernel][workload_name]
        if e.get("source_hash") != source_hash():
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples (every 50 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region starts once the sampler delivers (<= 3 s)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The oracle (complex128 CPU TBS) as it stands, on the host cores."""
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    w = make_workload(args)
    n = w.n
    terms_per_step = 2
    t0 = time.perf_counter()
    m, gh = oracle.plan(n, w.dx, w.f, w.c0)
    plan_s = time.perf_counter() - t0
    c = w.c.astype(np.float64)
    al = None if w.alpha is None else w.alpha.astype(np.float64)

    def step():
        V = oracle.potential(w.f, w.c0, c, al, w.ypow, w.f_ref)
        s = oracle.deposit_points(n, w.dx, w.src_ix, w.src_iy, w.src_amp[0].astype(np.complex128))
        oracle.solve(n, m, gh, V, s, terms_per_step, 0.0)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = n * n * terms_per_step * args.steps / dt
    sample = ("%s; each step = V build + source deposit + the first %d terms (u_0, u_1) of the "
              "series, plan (Green table + its FFT, %.1f s) excluded" % (w.name, terms_per_step, plan_s))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": {"workload": describe(w) % (n, m), "n": n, "m": m,
                       "terms_per_step": terms_per_step, "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(w):
    """Oracle timed on a bounded sample of the same workload (rank 0, N = 1)."""
    import numpy as np
    import oracle
    n = w.n
    terms = 3
    m, gh = oracle.plan(n, w.dx, w.f, w.c0)
    c = w.c.astype(np.float64)
    al = None if w.alpha is None else w.alpha.astype(np.float64)
    t0 = time.perf_counter()
    V = oracle.potential(w.f, w.c0, c, al, w.ypow, w.f_ref)
    s = oracle.deposit_points(n, w.dx, w.src_ix, w.src_iy, w.src_amp[0].astype(np.complex128))
    oracle.solve(n, m, gh, V, s, terms, 0.0)
    dt = time.perf_counter() - t0
    return {"value": n * n * terms / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%s: V build + source deposit + the first %d terms of the series in "
                      "complex128 (%.1f s), Green-table plan excluded" % (w.name, terms, dt)}


def cpu_baseline_configs():
    """The oracle as it stands on every workload, all host cores: per-term and
    per-field seconds for the 256^2 disk, the 2048^2 tissue solve and the
    2048^2 second-harmonic pair (each one RHS, to its stop rule), and for the
    broadband sweep one 24-term solve per padded size, extrapolated to all
    512 solves (the sweep in complex128 would take hours).  Green-table plan
    times are reported apart."""
    import numpy as np
    import oracle
    from paper_2507_13754_gb300 import workloads as W

    def one(w, max_terms=None, tol=None, src=None, **stop):
        t0 = time.perf_counter()
        m, gh = oracle.plan(w.n, w.dx, w.f, w.c0)
        t_plan = time.perf_counter() - t0
        t0 = time.perf_counter()
        V = oracle.potential(w.f, w.c0, w.c.astype(np.float64),
                             None if w.alpha is None else w.alpha.astype(np.float64), w.ypow, w.f_ref)
        if src is None:
            src = oracle.deposit_points(w.n, w.dx, w.src_ix, w.src_iy, w.src_amp[0].astype(np.complex128))
        psi, info, _, _ = oracle.solve(w.n, m, gh, V, src, w.max_terms if max_terms is None else max_terms,
                                       w.tol if tol is None else tol, **stop)
        t = time.perf_counter() - t0
        return psi, {"n": w.n, "m": m, "terms": info["terms"], "plan_s": t_plan, "field_s": t,
                     "term_s": t / info["terms"]}

    out = {"cores": oracle.num_threads(), "kind": "oracle"}
    _, out["cfg1_disk_256"] = one(W.cfg1())
    _, out["cfg2_tissue_2048"] = one(W.cfg2())
    w3 = W.cfg3()
    amp = (w3.src_amp * 2e5).astype(np.complex64)
    w3a = W.Workload(w3.name, w3.n, w3.dx, w3.f, w3.c0, w3.c, w3.alpha, w3.ypow, w3.f, w3.src_ix, w3.src_iy, amp,
                     64, 1e-6)
    psi1, r1 = one(w3a)
    s2 = oracle.harmonic2_source(2 * math.pi * w3.f, w3.extras["beta"].astype(np.float64),
                                 w3.extras["rho"].astype(np.float64), w3.c.astype(np.float64), psi1)
    w3b = W.Workload(w3.name, w3.n, w3.dx, 2 * w3.f, w3.c0, w3.c, W.cfg3_harmonic_alpha(w3), w3.ypow, 2 * w3.f,
                     w3.src_ix, w3.src_iy, amp, 64, 1e-6)
    _, r2 = one(w3b, src=s2)
    out["cfg3_harmonic_2048"] = {"fundamental": r1, "second_harmonic": r2,
                                 "field_s": r1["field_s"] + r2["field_s"]}
    ws = W.cfg4_list()
    buckets = {}
    for w in ws:
        m = oracle.padded_size(w.n)
        buckets.setdefault(m, []).append(w)
    sweep = 0.0
    per = {}
    for m, group in sorted(buckets.items()):
        # every sweep field runs exactly 24 terms (divergence rule off, as on the GPU)
        _, r = one(group[len(group) // 2], max_terms=24, tol=0.0, div_window=1 << 30, div_factor=math.inf)
        per["M=%d" % m] = dict(r, plans=len(group))
        sweep += r["field_s"] * len(group) * group[0].n_rhs
    out["cfg4_sweep"] = {"per_bucket": per, "extrapolated_sweep_s": sweep,
                         "how": "one 24-term solve (the middle frequency of each padded size) x the number of "
                                "solves of that size (plans x 8 angles)"}
    return out


def _timed(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def bench_cufft(w, plan, c_d, a_d, terms, ours_ms_per_term, stream):
    """Same recurrence with full padded cuFFT transforms + elementwise ops."""
    from paper_2507_13754_gb300 import baseline_cufft as B
    base = B.CufftBornSeries(w.n, plan.m, B.full_spectrum(plan.ghat_quadrant(), plan.m))
    V = B.potential(w.f, w.c0, c_d, a_d, w.ypow, w.f_ref)
    S = B.dense_source(w.n, w.dx, w.src_ix, w.src_iy, w.src_amp[0])
    base.solve_fixed(V, S, 3)
    ms = _timed(lambda: base.solve_fixed(V, S, terms), 2, stream)
    return {"ms_per_term": ms / terms, "ours_ms_per_term": ours_ms_per_term,
            "speedup": (ms / terms) / ours_ms_per_term, "terms": terms,
            "what": "torch.fft (cuFFT) full %d^2 C2C forward + inverse per term, separate pad/multiply/"
                    "crop/accumulate/norm ops, same Ghat and V" % plan.m}


def bench_sharded_sweep(stream, rank, world, dev):
    """The broadband sweep's 512 solves split over the ranks (one GPU each) by
    cost (M^2 x terms, longest first to the least-loaded rank): each rank
    builds one plan per frequency it owns, with the angles it owns as RHS,
    and runs them as one batch graph; no data crosses ranks.  The time is the
    slowest rank's (barrier on both sides); fields/s counts all ranks."""
    import torch
    from paper_2507_13754_gb300 import shard, tbs, workloads as W
    ws = W.cfg4_list()
    mine = shard.rank_solves(ws, world, rank, terms=24)
    fixed = dict(max_terms=24, tol=0.0, div_window=1 << 30, div_factor=math.inf)
    plans = []
    for k, rhs in sorted(mine.items()):
        w = ws[k]
        p = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=len(rhs), **fixed)
        p.set_medium(torch.from_numpy(w.c).to(dev), None, w.ypow, w.f_ref)
        p.set_sources(w.src_ix, w.src_iy, w.src_amp[rhs])
        plans.append(p)
    n_mine = sum(len(r) for r in mine.values())
    batch = tbs.Batch(plans) if plans else None
    if batch:
        batch.solve()
    torch.cuda.synchronize()
    torch.distributed.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(2):
        if batch:
            batch.solve()
    b.record(stream)
    torch.cuda.synchronize()
    t_ms = a.elapsed_time(b) / 2
    t_max, n_all = aggregate_ranks(t_ms / 1e3, n_mine, world, dev)
    if batch:
        batch.close()
    for p in plans:
        p.close()
    return {"fields": int(n_all), "fields_this_rank": n_mine, "ms": 1e3 * t_max,
            "fields_per_s": n_all / t_max, "ranks": world,
            "what": "cfg4 sweep (512 solves, 24 terms) partitioned over ranks by M^2 x terms, one batch "
                    "graph per rank, slowest rank's time"}


def bench_batched(stream):
    """Broadband sweep: 64 frequencies x 8 steering angles (N 512..2048, 24 terms each).

    Every field runs exactly 24 terms: the divergence rule is off (above
    ~4 MHz the 7.5 mm disk makes the series grow; kappa = max|u_n| / |psi|
    is reported)."""
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    ws = W.cfg4_list()
    fixed = dict(max_terms=24, tol=0.0, div_window=1 << 30, div_factor=math.inf)
    t0 = time.perf_counter()
    plans_b, plans_1 = [], []
    for w in ws:
        c = torch.from_numpy(w.c).cuda()
        pb = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=w.n_rhs, **fixed)
        pb.set_medium(c, None, w.ypow, w.f_ref)
        pb.set_sources(w.src_ix, w.src_iy, w.src_amp)
        p1 = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=1, **fixed)
        p1.set_medium(c, None, w.ypow, w.f_ref)
        plans_b.append(pb)
        plans_1.append(p1)
    setup_s = time.perf_counter() - t0
    from paper_2507_13754_gb300 import autotune
    choice = {}
    for p in plans_b + plans_1:  # column and row pass shapes per (M, n_rhs, row shapes), timed once each
        key = "M=%d,rhs=%d,row_shapes=%d" % (p.m, p.n_rhs, tbs.tbs_row_variants(p.handle))
        if key not in choice:
            cv, rv = autotune.tune(p, cache_path=None)[0]
            choice[key] = {"col": tbs.tbs_col_variant_name(p.handle, cv),
                           "row": tbs.tbs_row_variant_name(p.handle, rv), "ids": [cv, rv]}
        else:
            tbs.tbs_set_col_variant(p.handle, choice[key]["ids"][0])
            tbs.tbs_set_row_variant(p.handle, choice[key]["ids"][1])
    batch = tbs.Batch(plans_b)
    n_fields = sum(w.n_rhs for w in ws)
    batch.solve()
    torch.cuda.synchronize()
    infos = [i for per_plan in batch.infos() for i in per_plan]
    kappa = [i["term_norm_max"] / i["psi_norm"] if i["psi_norm"] > 0 else math.inf for i in infos]
    terms = sorted({i["terms"] for i in infos})
    ms_b = _timed(batch.solve, 2, stream)
    # the sweep's time signal (tbs_synthesize) on a 512-receiver line at
    # 36 mm depth, one period of the frequency comb in 672 samples
    side = ws[0].n * ws[0].dx
    df = ws[1].f - ws[0].f
    syn = dict(dxs=[w.dx for w in ws], freqs_hz=[w.f for w in ws], weights=[df] * len(ws),
               origin=(0.0, 0.75 * side), step=(side / 511, 0.0), counts=(512, 1), t0=0.0,
               dt=1.0 / df / 672, n_t=672)
    sig = tbs.synthesize(batch.psi, **syn)
    ms_syn = _timed(lambda: tbs.synthesize(batch.psi, out=sig, **syn), 5, stream)
    outs = [torch.empty((1, w.n, w.n), dtype=torch.complex64, device="cuda") for w in ws]

    def loop():
        for w, p, o in zip(ws, plans_1, outs):
            for r in range(w.n_rhs):
                p.set_sources(w.src_ix, w.src_iy, w.src_amp[r:r + 1])
                p.solve(o, sync=False)
    loop()
    ms_l = _timed(loop, 1, stream)
    # the device side of a loop without host submission: each multi-RHS
    # plan's cached graph replayed back to back on the stream
    outs_b = [torch.empty((w.n_rhs, w.n, w.n), dtype=torch.complex64, device="cuda") for w in ws]
    info_b = [torch.empty(w.n_rhs * ctypes.sizeof(tbs.tbs_solve_info), dtype=torch.uint8, device="cuda")
              for w in ws]

    def replay():
        for p, o, i in zip(plans_b, outs_b, info_b):
            p.solve(o, sync=False, info=i)
    replay()
    ms_r = _timed(replay, 2, stream)
    bytes_sweep = sum(92.0 * w.n * w.n * 24 * w.n_rhs for w in ws)  # algorithmic bytes, 92 N^2 per term
    batch.close()
    for p in plans_b + plans_1:
        p.close()
    return {"fields": n_fields, "batched_fields_per_s": n_fields / (ms_b / 1e3),
            "loop_fields_per_s": n_fields / (ms_l / 1e3), "speedup": ms_l / ms_b,
            "replay_fields_per_s": n_fields / (ms_r / 1e3), "speedup_vs_replay": ms_r / ms_b,
            "batched_hbm_gbs": bytes_sweep / (ms_b / 1e3) / 1e9,
            "batched_ms": ms_b, "loop_ms": ms_l, "replay_ms": ms_r, "plan_setup_s": setup_s,
            "autotuned_variants": choice,
            "terms": terms, "kappa_max": max(kappa), "fields_kappa_over_10": sum(k > 10 for k in kappa),
            "synthesis_ms": ms_syn, "synthesis": "time signal of all 8 angles at 512 receivers x 672 "
                                                  "samples from the 64 fields (tbs_synthesize)",
            "what": "64 plans (one per frequency, 8 steering angles as right-hand sides) in one "
                    "graph launch vs 512 single-RHS tbs_solve calls in a loop, and vs the 64 plans' "
                    "own cached graphs replayed back to back (no host submission in between)"}


def bench_harmonic(stream):
    """Second harmonic at full size: the 2 MHz fundamental to 1e-6, the
    -1/2 xi (2 omega)^2 psi1^2 source, then the 4 MHz series (Eqs. 28a-b)."""
    import numpy as np
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.cfg3()
    n = w.n
    amp = (w.src_amp * 2e5).astype(np.complex64)  # ~0.5 MPa at the elements
    c = torch.from_numpy(w.c).cuda()
    a1 = torch.from_numpy(w.alpha).cuda()
    a2 = torch.from_numpy(W.cfg3_harmonic_alpha(w)).cuda()
    beta = torch.from_numpy(w.extras["beta"]).cuda()
    rho = torch.from_numpy(w.extras["rho"]).cuda()
    # the 4 MHz series contracts by ~0.86 per term here (the ellipse is twice
    # as strong in phase at 2 k0): 1e-6 takes ~95 terms, so its cap is 128
    p1 = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=1, max_terms=64, tol=1e-6)
    p2 = tbs.Plan(n, w.dx, 2 * w.f, w.c0, n_rhs=1, max_terms=128, tol=1e-6)
    p1.set_medium(c, a1, w.ypow, w.f)
    p2.set_medium(c, a2, w.ypow, 2 * w.f)
    psi1 = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    psi2 = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    st = {}

    def run():
        p1.set_sources(w.src_ix, w.src_iy, amp)
        st["i1"] = p1.solve(psi1, sync=False)[1]
        p2.set_harmonic2_source(psi1, beta, rho, c, 2 * math.pi * w.f)
        st["i2"] = p2.solve(psi2, sync=False)[1]
    run()
    ms = _timed(run, 3, stream)
    i1, i2 = tbs.Plan.info_dicts(st["i1"])[0], tbs.Plan.info_dicts(st["i2"])[0]
    p1.close()
    p2.close()
    t = i1["terms"] + i2["terms"]
    return {"ms": ms, "terms_fundamental": i1["terms"], "terms_harmonic": i2["terms"],
            "status_fundamental": i1["status_name"], "status_harmonic": i2["status_name"],
            "residual_fundamental": i1["residual"], "residual_harmonic": i2["residual"],
            "grid_pt_terms_per_s": n * n * t / (ms / 1e3),
            "what": "cfg3 2048^2: fundamental at 2 MHz to 1e-6 (<= 64 terms), S2 source, second harmonic "
                    "at 4 MHz to 1e-6 (<= 128 terms), plans prebuilt"}


PAPER_CASES = {
    # name: (Table 2 GPU iterations, seconds on the paper's RTX 4060, plan options, scatterer speed)
    "homogeneous": (135, 5.0, {}, None),
    "absorbing": (133, 8.0, {"kspace_dispersion": False}, None),
    "absorbing_dispersive": (132, 11.0, {"kspace_dispersion": True}, None),
    "inhomogeneous_1350": (134, 7.0, {}, 1350.0),
    "inhomogeneous_1650": (134, 7.0, {}, 1650.0),
    "inhomogeneous_1800": (134, 7.0, {}, 1800.0),
    # Table 3's lower convergence edge, where the plain iteration has an
    # unstable mode, with the convergent Born series preconditioner
    "inhomogeneous_1100_cbs": (None, None, {"cbs": True}, 1100.0),
}


def bench_paper_case(stream, name="homogeneous", use_graph=True):
    """One of the paper's own runs (Section 3.1, Table 2) on the periodic
    4096^2 grid: eps = 0.8 k^2, 450-cell sigmoid layer, 501 sources, Eq. 30
    on row 2049 to 1e-5; 'absorbing*' add the k-space potential of alpha0 =
    5.5e-10, nu = 1.5 (with or without its dispersive term),
    'inhomogeneous_*' a 1 mm cylinder at the given speed 40.2 mm down the
    axis."""
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))
    paper_iters, paper_s, opts, v_s = PAPER_CASES[name]
    case = W.paper_periodic_case(g, scatterer_speed=v_s)
    n = case.n
    kw = dict(stop_mode=tbs.TBS_STOP_L1_ROW, l1_row=case.l1_row, periodic=True, eps_factor=case.eps_factor,
              abl_width=case.abl_width, abl_zeta=case.abl_zeta, div_window=1 << 30, div_factor=math.inf)
    kspace = "kspace_dispersion" in opts
    if kspace:
        kw.update(kspace_alpha0=g["alpha0"]["value"], kspace_nu=g["nu"]["value"], **opts)
    if opts.get("cbs"):  # the library chooses eps = 1.01 max |U| from the medium
        kw.update(cbs=True, eps_factor=0.0)
    t0 = time.perf_counter()
    plan = tbs.Plan(n, case.dx, case.f, case.c0, max_terms=2000, tol=case.tol, use_graph=use_graph, **kw)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    c = torch.from_numpy(case.c).cuda()
    psi = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    st = {}

    def run():
        plan.set_medium(c, None, 1.0, case.f)
        plan.set_sources(case.ix, case.iy, case.amp)
        st["i"] = plan.solve(psi, sync=False)[1]
    run()
    # both passes' kernel shapes chosen by the autotuner on this plan's data
    from paper_2507_13754_gb300 import autotune
    (cv, rv), _ = autotune.tune(plan, cache_path=None)
    shapes = {"col": tbs.tbs_col_variant_name(plan.handle), "row": tbs.tbs_row_variant_name(plan.handle)}
    run()
    ms = _timed(run, 3, stream)
    info = tbs.Plan.info_dicts(st["i"])[0]
    plan.close()
    iters = info["terms"] - 1
    # per-pass device times: the same run with CUDA events around every
    # launch, tol = 0 and exactly as many terms, so that every launch is active
    tplan = tbs.Plan(n, case.dx, case.f, case.c0, max_terms=info["terms"], tol=0.0, **kw)
    tbs.tbs_set_col_variant(tplan.handle, cv)
    tbs.tbs_set_row_variant(tplan.handle, rv)
    tplan.set_medium(c, None, 1.0, case.f)
    tplan.set_sources(case.ix, case.iy, case.amp)
    tplan.set_timing(True)
    tplan.solve(psi)
    row_ms, row_k, col_ms, col_k = tplan.timing()
    tplan.close()
    nn = float(n) * n
    # algorithmic bytes: row = W read + X write + psi read/write + (V and S,
    # or psi^0 with the k-space potential) reads; column = X read + W write
    row_b, col_b = (40.0 if kspace else 48.0) * nn, 16.0 * nn
    row_us, col_us = 1e3 * row_ms / max(1, row_k), 1e3 * col_ms / max(1, col_k)
    return {"ms": ms, "iterations": iters, "status": info["status_name"], "plan_ms": plan_ms,
            "row_pass_us": row_us, "col_pass_us": col_us, "autotuned_shapes": shapes,
            "row_pass_gbs": row_b / row_us / 1e3, "col_pass_gbs": col_b / col_us / 1e3,
            "us_per_iteration": 1e3 * ms / info["terms"],
            "grid_pt_iterations_per_s": nn * info["terms"] / (ms / 1e3),
            "paper_gpu": {"iterations": paper_iters, "seconds": paper_s, "hardware": "RTX 4060 (Table 2)"},
            "what": "Section 3.1 %s case on the periodic 4096^2 grid, medium and 501 sources set and solved "
                    "per run, plan built once" % name}


def bench_paper_nonlinear(stream):
    """The paper's nonlinear run (Section 3.1, Table 2 'Nonlinear'): the
    periodic 4096^2 case above in water with B/A = 5, harmonics 1 .. 5 by
    the sum-term sources, eps_n = 0.8 n^2 k^2, each to Eq. 30 < 1e-5; the
    paper reports 135, 228, 306, 368, 416 iterations (RTX 4060: 5, 9, 12,
    15, 16 s)."""
    import numpy as np
    import torch
    from paper_2507_13754_gb300.solvers import harmonics
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))
    n, dx, v, f = g["grid_n"]["value"], g["dx_m"]["value"], g["v_f"]["value"], g["f_hz"]["value"]
    row = g["source_row_1based"]["value"] - 1
    half = (g["n_elements"]["value"] - 1) // 2
    iy = np.arange(row - half, row + half + 1, dtype=np.int32)
    ix = np.full_like(iy, g["source_column"]["value"])
    amp = np.full((1, iy.size), complex(*g["source_amplitude"]["value"]) * dx * dx, np.complex64)
    beta = torch.full((n, n), 1.0 + g["ba"]["value"] / 2.0, dtype=torch.float32, device="cuda")
    rho = torch.full((n, n), 1000.0, dtype=torch.float32, device="cuda")
    kw = dict(max_terms=2000, tol=g["stop_tol"]["value"], periodic=True, eps_factor=g["eps_factor"]["value"],
              abl_width=g["abl_width_cells"]["value"], abl_zeta=g["abl_zeta_np_per_m"]["value"], stop_mode=1,
              l1_row=row, div_window=1 << 30, div_factor=math.inf)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fields, infos = harmonics(5, n, dx, f, v, None, None, 1.0, beta, rho, ix, iy, amp, **kw)
    torch.cuda.synchronize()
    s = time.perf_counter() - t0
    return {"seconds": s, "iterations": [i[0]["terms"] - 1 for i in infos],
            "status": [i[0]["status_name"] for i in infos],
            "log2_scale": [i[0]["log2_scale"] for i in infos],
            "paper_gpu_iterations": [135, 228, 306, 368, 416],
            "what": "harmonics 1-5 of the Section 3.1 run on the periodic 4096^2 grid, plans built per "
                    "harmonic inside the timed region (host wall clock)"}


def bench_adjoint(stream):
    """1024^2, 16 sources: forward solve vs adjoint (gradients in c and alpha)."""
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.cfg5()
    n = w.n
    plan = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=w.n_rhs, max_terms=64, tol=1e-6, keep_terms=True)
    c = torch.from_numpy(w.c).cuda()
    a = torch.from_numpy(w.alpha).cuda()
    g = torch.zeros((w.n_rhs, n, n), dtype=torch.complex64, device="cuda")
    g[:, w.extras["receiver_row"], :] = 1.0
    gc = torch.empty((n, n), dtype=torch.float32, device="cuda")
    ga = torch.empty((n, n), dtype=torch.float32, device="cuda")
    psi = torch.empty((w.n_rhs, n, n), dtype=torch.complex64, device="cuda")
    state = {}

    def fwd():
        plan.set_medium(c, a, w.ypow, w.f_ref)
        plan.set_sources(w.src_ix, w.src_iy, w.src_amp)
        state["infos"] = plan.solve(psi, sync=False)[1]

    def adj():
        plan.solve_adjoint(g, gc, ga)
    fwd()
    adj()
    ms_f = _timed(fwd, 2, stream)
    terms = [i["terms"] for i in tbs.Plan.info_dicts(state["infos"])]
    ms_a = _timed(adj, 2, stream)
    bytes_stored = tbs.tbs_plan_device_bytes(plan.desc)
    plan.close()
    # checkpointed terms: every K-th term kept, the rest recomputed in the sweep
    plan = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=w.n_rhs, max_terms=64, tol=1e-6, keep_terms=True, checkpoint=True)
    fwd()
    adj()
    ms_fc = _timed(fwd, 2, stream)
    ms_ac = _timed(adj, 2, stream)
    bytes_ckpt = tbs.tbs_plan_device_bytes(plan.desc)
    plan.close()
    return {"forward_ms": ms_f, "adjoint_ms": ms_a, "ratio": ms_a / ms_f,
            "terms": sorted(set(terms)), "n_rhs": w.n_rhs,
            "checkpointed": {"forward_ms": ms_fc, "adjoint_ms": ms_ac, "ratio": ms_ac / ms_fc,
                             "plan_bytes": bytes_ckpt, "plan_bytes_all_terms": bytes_stored},
            "what": "1024^2 at 3 MHz, 16 sources, residual 1e-6 (max 64 terms); adjoint = dL/dc and "
                    "dL/dalpha; checkpointed: every 8th term kept, the rest recomputed"}


def aggregate_ranks(t_seconds, units, world, device):
    """Replicas: every rank solved its own problems.  Returns (max time over
    ranks, units summed over ranks); value = units / time for the whole job."""
    if world <= 1:
        return t_seconds, float(units)
    import torch
    tt = torch.tensor([t_seconds, float(units)], dtype=torch.float64, device=device)
    gathered = [torch.zeros_like(tt) for _ in range(world)]
    torch.distributed.all_gather(gathered, tt)
    return max(float(g[0]) for g in gathered), sum(float(g[1]) for g in gathered)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2507_13754_gb300 import build, tbs

    torch.cuda.set_device(local_rank)
    if build.is_stale():
        build.build()
    tbs.load_library()
    w = make_workload(args)
    n = w.n
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    plan = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=1, max_terms=w.max_terms, tol=w.tol, use_graph=not args.no_graph)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    m = plan.m
    col_variant_name = tbs.tbs_col_variant_name(plan.handle)
    row_variant_name = tbs.tbs_row_variant_name(plan.handle)
    c_d = torch.from_numpy(w.c).to(dev)
    a_d = torch.from_numpy(w.alpha).to(dev) if w.alpha is not None else None
    psi = torch.empty((1, n, n), dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # solve records stay on the device in the timed loop (a host copy would
    # make every step wait for the host), one buffer per step
    info_bytes = ctypes.sizeof(tbs.tbs_solve_info)
    info_d = torch.zeros((max(args.steps, args.warmup), info_bytes), dtype=torch.uint8, device=dev)

    def step(k):
        plan.set_medium(c_d, a_d, w.ypow, w.f_ref)
        plan.set_sources(w.src_ix, w.src_iy, w.src_amp)
        plan.solve(psi, sync=False, info=info_d[k])
        return info_d[k]

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    # ---- timed region: K steps, device events per step, L2 flushed between
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    infos = []
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        infos.append(step(k))
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    terms = [plan.device_info_dicts(i)[0]["terms"] for i in infos]
    status = plan.device_info_dicts(infos[-1])[0]["status_name"]
    t_total = sum(ms) / 1e3
    units = n * n * sum(terms)
    t_max, units_all = aggregate_ranks(t_total, units, world, dev)
    value = units_all / t_max
    # medium, deposit, row(src), (col, row, stop) per term slot, info: the
    # graph's term loop runs bodies of four terms until every RHS has
    # stopped (one RHS here), so max(terms) rounds up to a multiple of four
    launches = sum(2 + 1 + 3 * (4 * -(-t // 4)) + 1 for t in terms)

    if args.kernel_only:
        if rank == 0:
            print(json.dumps({"kernel_only": True, "value": value, "terms": terms}), flush=True)
        return 0

    # ---- live per-kernel timing (CUDA events around each launch), tol = 0 so
    # that every launch of the pass is an active one
    T = int(round(statistics.median(terms)))
    tplan = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=1, max_terms=T, tol=0.0)
    tplan.set_medium(c_d, a_d, w.ypow, w.f_ref)
    tplan.set_sources(w.src_ix, w.src_iy, w.src_amp)
    tplan.solve(psi)  # warm
    tplan.set_timing(True)
    for _ in range(2):
        flush.zero_()
        tplan.solve(psi, sync=False)
    torch.cuda.synchronize()
    row_ms, row_n, col_ms, col_n = tplan.timing()
    tplan.close()
    nn = float(n) * n
    row_bytes = 16.0 * n * m + 24.0 * nn  # W read + X write, V read, psi read+write
    col_bytes = 16.0 * n * m + 4.0 * nn   # X read + W write, Ghat octant
    row_avg = row_ms / max(1, row_n)
    col_avg = col_ms / max(1, col_n)
    peak, peak_kind = measured_peak()
    kernels = {"row_pass": (row_avg, row_bytes), "col_pass": (col_avg, col_bytes)}
    dom = max(kernels, key=lambda k: kernels[k][0])
    d_ms, d_bytes = kernels[dom]
    achieved = d_bytes / (d_ms / 1e3) / 1e9
    term_ms = (row_avg + col_avg)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": ncu_traffic(dom, w.name),
                "algorithmic_bytes_per_launch": d_bytes, "avg_launch_ms": d_ms,
                "row_pass_ms": row_avg, "col_pass_ms": col_avg,
                "term_gbs": (row_bytes + col_bytes) / (term_ms / 1e3) / 1e9,
                "term_frac": (row_bytes + col_bytes) / (term_ms / 1e3) / 1e9 / peak}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        # Double-buffered on two copy streams: step k+1's inputs go up on one
        # while step k solves, and step k's psi and records come down on the
        # other while step k+1 solves; each step still copies its c, alpha,
        # amplitudes in and its psi and records out, all inside the one timed
        # region (with the L2 flushes).
        c_h = torch.from_numpy(w.c).pin_memory()
        a_h = torch.from_numpy(w.alpha).pin_memory() if w.alpha is not None else None
        xin, xout = torch.cuda.Stream(), torch.cuda.Stream()
        c_s = [torch.empty_like(c_d) for _ in range(2)]
        a_s = [torch.empty_like(a_d) if a_d is not None else None for _ in range(2)]
        psi_d = [torch.empty((1, n, n), dtype=torch.complex64, device=dev) for _ in range(2)]
        psi_h = [torch.empty((1, n, n), dtype=torch.complex64).pin_memory() for _ in range(2)]
        isz = ctypes.sizeof(tbs.tbs_solve_info)
        nk = args.steps + 2
        info_d = torch.zeros((nk, isz), dtype=torch.uint8, device=dev)
        info_h = torch.zeros((nk, isz), dtype=torch.uint8).pin_memory()
        ev = {key: [torch.cuda.Event() for _ in range(2)] for key in ("in", "free", "out", "d2h")}

        def e2e_step(k):
            b = k % 2
            with torch.cuda.stream(xin):
                xin.wait_event(ev["free"][b])   # step k-2 has read this staging buffer
                c_s[b].copy_(c_h, non_blocking=True)
                if a_h is not None:
                    a_s[b].copy_(a_h, non_blocking=True)
                ev["in"][b].record(xin)
            stream.wait_event(ev["in"][b])
            stream.wait_event(ev["d2h"][b])    # step k-2's psi has left this buffer
            plan.set_medium(c_s[b], a_s[b], w.ypow, w.f_ref)
            ev["free"][b].record(stream)
            plan.set_sources(w.src_ix, w.src_iy, w.src_amp)
            plan.solve(psi_d[b], sync=False, info=info_d[k])
            ev["out"][b].record(stream)
            with torch.cuda.stream(xout):
                xout.wait_event(ev["out"][b])
                psi_h[b].copy_(psi_d[b], non_blocking=True)
                info_h[k].copy_(info_d[k], non_blocking=True)
                ev["d2h"][b].record(xout)

        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        t_a, t_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_a.record(stream)
        xin.wait_event(t_a)
        xout.wait_event(t_a)
        for k in range(2, nk):
            flush.zero_()
            e2e_step(k)
        stream.wait_event(ev["d2h"][(nk - 1) % 2])
        t_b.record(stream)
        torch.cuda.synchronize()
        t2 = t_a.elapsed_time(t_b) / 1e3
        recs = [(tbs.tbs_solve_info * 1).from_buffer_copy(info_h[k].numpy().tobytes()) for k in range(2, nk)]
        terms2 = sum(tbs.Plan.info_dicts(r)[0]["terms"] for r in recs)
        h2d = w.c.nbytes + (w.alpha.nbytes if w.alpha is not None else 0) + w.src_amp.nbytes + \
            w.src_ix.nbytes + w.src_iy.nbytes
        d2h = psi_h[0].numel() * 8 + isz
        e2e = {"value": n * n * terms2 / t2, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * t2 / args.steps,
               "how": "public API per step (set_medium from pinned host c, alpha; set_sources from host "
                      "amplitudes; solve; psi and records back to pinned host), copies double-buffered on two "
                      "copy streams (in, out), one timed region over all steps including the L2 flushes"}

    extra = {}
    if not args.no_extras:
        extra["cufft_baseline"] = bench_cufft(w, plan, c_d, a_d, T, term_ms, stream)
        extra["batched"] = bench_batched(stream)
        extra["adjoint"] = bench_adjoint(stream)
        extra["harmonic"] = bench_harmonic(stream)
        extra["paper_cases"] = {k: bench_paper_case(stream, k) for k in PAPER_CASES}
        extra["paper_nonlinear"] = bench_paper_nonlinear(stream)
        if world > 1:
            extra["sharded_sweep"] = bench_sharded_sweep(stream, rank, world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    plan.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
                "data": "synthetic",
                "config": {"workload": describe(w) % (n, m), "n": n, "m": m,
                           "terms_per_step": terms, "status": status,
                           "l2": "flushed by a 256 MiB write between timed steps",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "norms": "fp64 (per-warp fp32 partials)",
                           "col_pass_variant": col_variant_name,
                           "row_pass_variant": row_variant_name},
                "born_terms_per_s": sum(terms) / t_total,
                "plan_ms": plan_ms,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "source_hash": source_hash(), **extra}
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.paper_case:
        import torch
        torch.cuda.set_device(local_rank)
        stream = torch.cuda.current_stream()
        print(json.dumps({"paper_case": args.paper_case,
                          **bench_paper_case(stream, args.paper_case, use_graph=not args.no_graph)}), flush=True)
        return 0
    if args.cpu_baseline_configs:
        if rank == 0:
            print(json.dumps({"cpu_baseline_configs": cpu_baseline_configs()}), flush=True)
        return 0
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

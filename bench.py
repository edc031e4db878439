#!/usr/bin/env python3
"""Benchmark of the PC-stable skeleton path on one GB300 (or N replicas).

A step is one whole skeleton: FP64 standardisation, the correlation product,
level 0 and every level until the termination rule, on the medium1000 workload
(p = 1000 variables, n = 10000 samples, random DAG of expected degree 3,
weights +-U[0.1, 1], float32 input, alpha = 0.01), synthetic and seeded.

Metric: CI tests per second, counting the tests the serial algorithm performs
on this input (the canonical lexicographic run's per-level counts, identical to
the CPU oracle's), divided by the skeleton wall time. ``value`` is measured
with the input resident in device memory (CUDA events on the library's
stream, L2 flushed between steps); ``e2e`` through the same public call with a
pinned host input, including the upload and the download of the skeleton (as
an edge list) and the SepSets. The plain form (FP64 for every test) is timed
beside the chosen form.

``--impl reference`` times the CPU oracle as it stands on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "skeleton wall time (s) and CI tests/sec, chosen vs plain form, exact skeleton"
UNIT = "CI tests/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


# FP32 SIMT peak from unit counts and clocks: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 non-tensor rate of GB300 (nominal table of the part).
FP64_TFLOPS = 1.25


LEVEL_SOURCES = ("paper_1812_08491_gb300/csrc/k_level.cu", "paper_1812_08491_gb300/csrc/kernels.cuh",
                 "paper_1812_08491_gb300/csrc/cupc_internal.cuh")


def level_source_hash():
    """sha256 of the level kernel's sources (the ncu traffic figures are tied to it)."""
    import hashlib
    h = hashlib.sha256()
    for rel in LEVEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(workload):
    """DRAM bytes per level-kernel launch from the committed ncu summary of this
    workload, or None when there is none or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", f"k_level_{workload}.md")
    try:
        fields = {}
        for line in open(path):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("source_hash") != level_source_hash():
            return None
        return float(fields["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def cpu_oracle_run(sem_obj, nthreads, keep=None):
    """One full oracle skeleton (correlation + Algorithm 1): (seconds, serial tests).
    The oracle's result is stored in keep["res"] when a dict is given."""
    import oracle
    t0 = time.perf_counter()
    C = oracle.correlation(sem_obj.X, nthreads=nthreads)
    res = oracle.pc_stable(C, sem_obj.n, sem_obj.alpha, max_level=sem_obj.max_level, nthreads=nthreads)
    if keep is not None:
        keep["res"] = res
    return time.perf_counter() - t0, res.total_tests


def orientation_line(ctx, X, s, mode, oracle_res=None, reps=5):
    """The second step of PC-stable (v-structures + Meek's rules) on the device,
    after one skeleton of the workload: device time (CUDA events inside the
    library, median of reps) and edge counts; with the oracle's skeleton, the
    oracle's orientation timed on the host beside it (one run)."""
    r = ctx.skeleton(X, s.alpha, mode=mode, max_level=s.max_level)
    times, st = [], None
    for _ in range(reps + 1):
        _, st = r.orient(marks=False)
        times.append(st["ms"])
    r.free()
    ms = statistics.median(times[1:])
    # algorithmic bytes: the skeleton bitset read for the neighbour lists and the
    # v-structures, per rule round the three bitsets (head, headT, proposals) read
    # and the proposals written, and the p x p marks written
    wbytes = s.p * ((s.p + 31) // 32) * 4
    byts = 3 * wbytes + st["rounds"] * 4 * wbytes + s.p * s.p
    ach = byts / (ms * 1e-3) / 1e9
    hbm = _peaks()["hbm_gbs"]
    out = {"device_ms": ms, "rounds": st["rounds"], "directed": st["directed"],
           "undirected": st["undirected"], "bidirected": st["bidirected"],
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                        "alg_bytes": byts, "note": "latency-bound: rule rounds queued four at a time, one readback each"},
           "note": "second step of PC-stable, outside the timed skeleton step"}
    if oracle_res is not None:
        import oracle
        t0 = time.perf_counter()
        oracle.orient(oracle_res)
        out["oracle_cpu_ms"] = 1e3 * (time.perf_counter() - t0)
    return out


def run_reference(args, workload_name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from synth import sem
    cores = os.cpu_count() or 1
    if workload_name in BATCH_WORKLOADS:
        return run_reference_batch(args, workload_name, cores)
    s = sem.workload(workload_name)
    for _ in range(args.warmup):
        cpu_oracle_run(s, cores)
    secs, units = 0.0, 0
    for _ in range(args.steps):
        t, u = cpu_oracle_run(s, cores)
        secs += t
        units += u
    value = units / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded linear-Gaussian SEM)",
            "config": dict(_config(workload_name, s, "cpu oracle"), l2="not applicable (host cores)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"whole {workload_name} skeleton per step (correlation + all levels)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference_batch(args, name, cores):
    """Oracle on a batch workload: each step runs a bounded sample of its problems
    (the first 16), one after another."""
    from synth import sem
    probs = sem.batch_workload(BATCH_WORKLOADS[name], 0)[:16]
    for _ in range(args.warmup):
        cpu_oracle_run(probs[0], cores)
    secs, units = 0.0, 0
    for _ in range(args.steps):
        for s in probs:
            t, u = cpu_oracle_run(s, cores)
            secs += t
            units += u
    value = units / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded linear-Gaussian SEMs)",
            "config": _batch_config(name, probs, "cpu oracle, first 16 problems per step"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "first 16 of the 64 problems per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _config(name, s, form):
    return {"workload": name, "p": s.p, "n": s.n, "family": s.family,
            "degree": s.meta.get("degree"), "alpha": s.alpha, "input_dtype": s.meta.get("dtype"),
            "form": form, "l2": "flushed between steps (256 MiB write)"}


def kernel_rooflines(st, s, mode, peaks, alu=None):
    """Roofline of each kernel of one skeleton call (stats of that call).

    Durations are CUDA-event times on the library's stream; algorithmic work:
      standardize  read X once; write the two bf16 rows (FP32 mode) or the FP64 rows (plain)
      correlation  3 split-precision bf16 products over the upper triangle, 2 n p(p+1)/2 each
      level0       read C once, write the bitset
      level        per level: the C sub-blocks its tests read, sum over rows of (n'_i+1)^2
                   entries, plus the bitset (read twice, copied once) and the CSR arrays
    """
    n, p = s.n, s.p
    es_in = 4 if s.meta.get("dtype") == "float32" else 8
    cb = 4 if mode == "fp32" else 8
    W = (p + 31) // 32
    out = {}
    km, kc = st["kernel_ms"], st["kernel_count"]
    hbm = peaks["hbm_gbs"]

    def mem(name, ms, launches, byts):
        if ms <= 0 or launches <= 0:
            return
        per = byts / launches
        ach = per / (ms / launches * 1e-3) / 1e9
        out[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "ms": ms, "launches": launches, "alg_bytes_per_launch": per, "traffic": None}

    mem("standardize", km["standardize"], kc["standardize"],
        n * p * es_in + (n * p * 4 if mode == "fp32" else n * p * 8))
    mem("level0", km["level0"], 1, p * p * cb + p * W * 4)
    lv = st["levels"]
    lev_ms = sum(st["level_ms"][1:lv])
    byts = 0
    for l in range(1, lv):
        nnz = 2 * st["edges_start"][l]
        byts += st["ci_block_entries"][l] * cb + 3 * p * W * 4 + nnz * 40
    mem("level", lev_ms, max(1, lv - 1), byts)
    # FP64 rechecks: per performed test the Gram block of its l + 2 variables over
    # n samples (one FMA per pair, one centring subtraction per variable, per sample)
    if alu and km.get("recheck", 0) > 0:
        flops = sum(st["rechecks"][l] * n * (2.0 * (l + 2) * (l + 1) / 2 + (l + 2)) for l in range(1, lv))
        ach = flops / (km["recheck"] * 1e-3) / 1e12
        out["recheck"] = {"bound": "alu", "achieved": ach, "peak": alu["fp64_tflops"], "unit": "TFLOP/s",
                          "frac": ach / alu["fp64_tflops"], "ms": km["recheck"], "launches": max(1, lv - 1),
                          "peak_src": "FP64 FMA, measured by cupc_device_peaks", "traffic": None}
    ms = km["correlation"]
    if ms > 0:
        if mode == "fp32":
            flops = 3 * 2.0 * n * p * (p + 1) / 2
            peak = peaks["bf16_tflops"]
            src = "bf16 dense, measured burst"
        else:
            flops = 2.0 * n * p * (p + 1) / 2
            peak = FP64_TFLOPS
            src = "FP64 nominal"
        ach = flops / (ms * 1e-3) / 1e12
        out["correlation"] = {"bound": "tensor" if mode == "fp32" else "alu", "achieved": ach, "peak": peak,
                              "unit": "TFLOP/s", "frac": ach / peak, "ms": ms, "launches": 1,
                              "peak_src": src, "traffic": None}
    return out


def level_bounds(st, mode, peaks, alu):
    """Bound of the level kernel's CI phase per level (SURVEY-style arithmetic
    intensity): algorithmic bytes = the C sub-block entries the level's tests
    read; FP32 (or FP64) flops = tests x (l^2 + 4 l + 10) (the factor apply, the
    decision; the per-(i, S) factorisations are left out, so this is a lower
    bound). A level whose flops per byte exceed the ridge point (measured ALU
    peak / measured HBM bandwidth) is ALU-bound, else HBM-bound; achieved is over
    the CI phase's device-clock time."""
    cb = 4 if mode == "fp32" else 8
    hbm = peaks["hbm_gbs"]
    alu_peak = (alu["fp32_tflops"] if mode == "fp32" else alu["fp64_tflops"]) if alu else None
    out = []
    for l in range(1, st["levels"]):
        ms = st["phase_ms"][l][1]
        byts = st["ci_block_entries"][l] * cb
        flops = st["tests"][l] * (l * l + 4 * l + 10)
        if ms <= 0 or byts <= 0:
            continue
        ridge = (alu_peak * 1e12) / (hbm * 1e9) if alu_peak else float("inf")
        intensity = flops / byts
        if intensity > ridge:
            ach = flops / (ms * 1e-3) / 1e12
            out.append({"level": l, "bound": "alu", "unit": "TFLOP/s", "achieved": round(ach, 4), "peak": alu_peak,
                        "frac": round(ach / alu_peak, 6), "intensity": round(intensity, 2), "ci_ms": round(ms, 4)})
        else:
            ach = byts / (ms * 1e-3) / 1e9
            out.append({"level": l, "bound": "hbm", "unit": "GB/s", "achieved": round(ach, 3), "peak": hbm,
                        "frac": round(ach / hbm, 6), "intensity": round(intensity, 2), "ci_ms": round(ms, 4)})
    return out


def timed_steps(ctx, X, s, opts, steps, stream, flush):
    """Device time (ms) of `steps` skeleton calls with L2 flushed between them, and
    the last call's stats; CUDA events on the library's stream around each call."""
    import torch
    tot, st = 0.0, None
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = ctx.skeleton(X, s.alpha, opts)
        b.record(stream)
        st = r.stats()
        r.free()
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot, st


def large_leg(ctx, args, peaks_alu, dev, stream, flush, learned_info_cache):
    """The p = 10^4 workload (n = 1000, degree 5, levels up to 6) beside the
    headline one: FP32 bulk + FP64 recheck, the learned ordering on top of it,
    and the plain FP64 form, each timed on device-resident input."""
    import torch

    import paper_1812_08491_gb300 as cupc
    from synth import sem
    s = sem.workload("large10000")
    X = torch.from_numpy(s.Xt).to(dev).T
    ref = ctx.skeleton(X, s.alpha, mode=cupc.MODE_FP32_RECHECK, canonical=True, max_level=s.max_level)
    units = int(sum(ref.stats()["serial_tests"]))
    ref.free()
    opts = ctx.options(mode=cupc.MODE_FP32_RECHECK, canonical=True, max_level=s.max_level)
    timed_steps(ctx, X, s, opts, max(3, args.warmup), stream, flush)
    k = max(3, args.steps // 2)
    ms, st = timed_steps(ctx, X, s, opts, k, stream, flush)
    leg = {"workload": "large10000", "p": s.p, "n": s.n, "degree": 5.0, "alpha": s.alpha, "max_level": s.max_level,
           "input_dtype": "float64", "serial_tests_per_step": units, "steps": k,
           "ms_per_step": ms / k, "value": units * k / (ms * 1e-3), "unit": UNIT,
           "form": "FP32 bulk + FP64 recheck", "l2": "flushed between steps (256 MiB write)"}
    kern = kernel_rooflines(st, s, "fp32", _peaks(), peaks_alu)
    dom = max((q for q in kern if q != "recheck"), key=lambda q: kern[q]["ms"])
    leg["roofline"] = {q: kern[dom][q] for q in ("bound", "achieved", "peak", "unit", "frac")}
    leg["roofline"]["kernel"] = dom
    leg["kernel_rooflines"] = {q: {"frac": round(v["frac"], 5), "achieved": round(v["achieved"], 3),
                                   "unit": v["unit"], "bound": v["bound"], "ms": round(v["ms"], 4)}
                               for q, v in kern.items()}
    leg["level_bounds"] = level_bounds(st, "fp32", _peaks(), peaks_alu)
    leg["kernel_launches_per_step"] = st["kernel_launches"]
    if not args.no_plain:
        popt = ctx.options(mode=cupc.MODE_PLAIN_FP64, canonical=True, max_level=s.max_level)
        timed_steps(ctx, X, s, popt, 1, stream, flush)
        pms, _ = timed_steps(ctx, X, s, popt, 2, stream, flush)
        leg["plain_form"] = {"ms_per_step": pms / 2, "value": units * 2 / (pms * 1e-3), "unit": UNIT}
        leg["speedup_vs_plain"] = (pms / 2) / (ms / k)
    if not args.no_learned_leg:
        from paper_1812_08491_gb300 import learned
        if "weights" not in learned_info_cache:
            t0 = time.perf_counter()
            Xtr, ttr = learned.collect(ctx, [sem.mlp_training_instance(q) for q in range(200)])
            learned.train(ctx, Xtr, ttr, epochs=6, batch=4096, lr=2e-3)
            learned_info_cache["weights"] = ctx.mlp_get_weights()
            learned_info_cache["setup_s"] = round(time.perf_counter() - t0, 1)
        ctx.mlp_set_weights(learned_info_cache["weights"])
        lopt = ctx.options(mode=cupc.MODE_FP32_RECHECK, canonical=True, max_level=s.max_level, learned_order=True)
        timed_steps(ctx, X, s, lopt, 1, stream, flush)
        lms, lst = timed_steps(ctx, X, s, lopt, k, stream, flush)
        lser = int(sum(lst["serial_tests"]))
        leg["learned_form"] = {"ms_per_step": lms / k, "value": units * k / (lms * 1e-3), "unit": UNIT,
                               "serial_tests_learned_order": lser, "serial_tests_lexicographic": units,
                               "network_setup_s": learned_info_cache["setup_s"]}
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        secs, cu = cpu_oracle_run(s, cores)
        leg["cpu_baseline"] = {"value": cu / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"whole large10000 skeleton once (correlation + levels 0-6), {secs:.2f} s"}
    return leg


def sshare_report(ctx, dev, names=("medium1000", "scalefree2500", "large10000"), levels=(1, 2, 3)):
    """The global-sharing diagnostic (Sec. 5.5, Fig. 9) per workload and level:
    one JSON line each with the histogram of rows per conditioning set, what a
    global search finds (distinct sets, factorisations it would save) and its
    device time, beside the level's CI-phase time with row-local sharing."""
    import torch
    from synth import sem
    bins = [1, 2, 3, 5, 9, 17, 33, 41, 65, 129]
    for name in names:
        s = sem.workload(name)
        X = torch.from_numpy(s.Xt).to(dev).T
        r = ctx.skeleton(X, s.alpha, max_level=s.max_level)
        st = r.stats()
        for level in levels:
            if level >= st["levels"]:
                continue
            r.sshare(level, bins)                         # warm-up (buffers sized)
            counts, ss = r.sshare(level, bins)
            red = ss["redundant"]
            sets_le40 = sum(c for b, c in zip(bins, counts) if b <= 40) - counts[0]
            print(json.dumps({"sshare": name, "level": level, "bins": bins, "sets_per_bin": counts,
                              "pairs_row_S": ss["pairs"], "distinct_S": ss["distinct"], "redundant_S": red,
                              "redundant_in_at_most_40_rows": round(sets_le40 / red, 4) if red else None,
                              "max_rows_one_S": ss["max_rows"], "rows": ss["rows"],
                              "factorisations_saved_by_global_sharing": ss["pairs"] - ss["distinct"],
                              "global_search_ms": round(ss["search_ms"], 4),
                              "level_ci_ms_row_local": round(st["phase_ms"][level][1], 4)}))
        r.free()


SWEEP_POINTS = ([(p, 10000, 0.1) for p in (1000, 2000, 3000, 4000)] +
                [(1000, m, 0.1) for m in (2000, 4000, 6000, 8000)] +
                [(1000, 10000, d) for d in (0.2, 0.3, 0.4, 0.5)])
# points whose oracle run (levels 0-2) finishes in well under a minute on 16 cores
SWEEP_PARITY = {(1000, 10000, 0.1), (1000, 2000, 0.1), (1000, 4000, 0.1), (1000, 6000, 0.1), (1000, 8000, 0.1)}


def sweep_report(ctx, dev, graphs, max_level=2, parity=True):
    """The scalability sweep of Sec. 5.6 on its axes (p 1000-4000 at m = 10^4,
    d = 0.1; m 2000-10^4 at p = 1000, d = 0.1; d 0.1-0.5 at p = 1000, m = 10^4),
    `graphs` graphs per point, with the signed-weight, variance-normalised form of
    the paper's generator (synth.sem.paper_density_signed) and levels 0-2 (dense
    graphs make deeper levels' subset counts explode). One JSON line per point:
    device time and host wall time of one skeleton from device-resident data
    (the second call on that shape), serial tests, edges; on graph 0 of the
    points in SWEEP_PARITY, the oracle's run of the same levels and whether the
    skeleton, removal levels, SepSets and serial counts are identical."""
    import numpy as np
    import torch

    import oracle
    import paper_1812_08491_gb300 as cupc
    from synth import sem
    for q, (p, m, d) in enumerate(SWEEP_POINTS):
        dev_ms, wall_ms, tests, edges, match = [], [], [], [], None
        for g in range(graphs):
            s = sem.paper_density_signed(p, m, d, 6000000 + 1000 * q + g, max_level=max_level)
            X = torch.from_numpy(s.Xt).to(dev).T
            opts = ctx.options(mode=cupc.MODE_FP32_RECHECK, canonical=True, max_level=max_level)
            ctx.skeleton(X, s.alpha, opts).free()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = ctx.skeleton(X, s.alpha, opts)
            wall_ms.append(1e3 * (time.perf_counter() - t0))
            st = r.stats()
            dev_ms.append(st["total_ms"])
            tests.append(int(sum(st["serial_tests"])))
            edges.append(int(st["edges_final"]))
            if parity and g == 0 and (p, m, d) in SWEEP_PARITY:
                t1 = time.perf_counter()
                C = oracle.correlation(s.X, nthreads=os.cpu_count() or 1)
                ref = oracle.pc_stable(C, s.n, s.alpha, max_level=max_level, nthreads=os.cpu_count() or 1)
                match = {"identical": bool(np.array_equal(r.adjacency(), ref.adj)
                                            and np.array_equal(r.sep_levels(), ref.sep_level)
                                            and r.sepsets() == ref.sepsets
                                            and st["serial_tests"][:ref.levels_run] == list(ref.tests)),
                          "oracle_s": round(time.perf_counter() - t1, 2)}
            r.free()
            del X
        print(json.dumps({"sweep_point": {"p": p, "m": m, "d": d}, "graphs": graphs, "max_level": max_level,
                          "device_ms_mean": round(float(np.mean(dev_ms)), 3),
                          "device_ms_min_max": [round(min(dev_ms), 3), round(max(dev_ms), 3)],
                          "wall_ms_mean": round(float(np.mean(wall_ms)), 3),
                          "serial_tests_mean": int(np.mean(tests)), "edges_mean": int(np.mean(edges)),
                          "serial_tests_per_s": float(np.sum(tests) / (np.sum(dev_ms) * 1e-3)),
                          "parity_graph0": match if match is not None else "oracle not run at this size",
                          "generator": "paper_density_signed (Sec. 5.6 structure, signed weights, unit variance)"}),
              flush=True)


BATCH_WORKLOADS = {"batch64": 64}
L1_FORMS = {"auto": 0, "pivot": 1, "row": 2}   # cupc_options.level1_form


def _batch_config(name, probs, form):
    ps = [s.p for s in probs]
    ns = [s.n for s in probs]
    return {"workload": name, "problems": len(probs), "p_range": [min(ps), max(ps)], "n_range": [min(ns), max(ns)],
            "sum_p": int(sum(ps)), "family": "random", "degree": "U[2,6]", "alpha": probs[0].alpha,
            "input_dtype": "float32", "form": form, "launch": "one CUDA graph per step",
            "l2": "inputs (%.0f MB) larger than L2; 256 MiB write between steps" %
                  (sum(p * n for p, n in zip(ps, ns)) * 4 / 1e6)}


def batch_rooflines(bst, probs, peaks):
    """Roofline of each stage of one batch step (its stats; CUDA-event stage times).

      standardize  read X (float32), write the two bf16 rows
      correlation  3 bf16 products over each problem's upper triangle, 2 n p (p+1)/2 each
      level0       read every problem's C (FP32) once, write the bitsets; FP64 rechecks of the band
      level        per level: the C sub-blocks its tests read (FP32), the bitsets, the CSR arrays
    """
    km = bst["kernel_ms"]
    hbm = peaks["hbm_gbs"]
    out = {}

    def mem(name, ms, byts):
        if ms <= 0:
            return
        ach = byts / (ms * 1e-3) / 1e9
        out[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "ms": ms,
                     "launches": 1, "alg_bytes_per_launch": byts, "traffic": None}

    words = sum(((s.p + 31) // 32 * 32) ** 2 // 32 for s in probs)
    mem("standardize", km["standardize"], sum(s.n * s.p * (4 + 4) for s in probs))
    mem("level0", km["level0"], sum(s.p * s.p * 4 for s in probs) + words * 4)
    lv = bst["levels"]
    byts = 0
    for l in range(1, lv):
        byts += bst["ci_block_entries"][l] * 4 + 3 * words * 4 + 2 * bst["edges_start"][l] * 40
    mem("level", bst["level_ms"][1] if lv > 1 else 0.0, byts)
    ms = km["correlation"]
    if ms > 0:
        flops = sum(3 * 2.0 * s.n * s.p * (s.p + 1) / 2 for s in probs)
        ach = flops / (ms * 1e-3) / 1e12
        out["correlation"] = {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                              "frac": ach / peaks["bf16_tflops"], "ms": ms, "launches": 1,
                              "peak_src": "bf16 dense, measured burst", "traffic": None}
    return out


def main_batch(args, world, rank, local, dist):
    """The batched workload: a step is one skeleton_batch call over all problems."""
    import numpy as np
    import torch

    import paper_1812_08491_gb300 as cupc
    from synth import sem

    dev = torch.device("cuda", local)
    cupc.build_library()
    probs = sem.batch_workload(BATCH_WORKLOADS[args.workload], 0)
    alphas = [s.alpha for s in probs]
    Xd = [torch.from_numpy(s.Xt.astype(np.float32)).to(dev).T for s in probs]   # variable-major n x p
    ctx = cupc.Context(local, level1_form=L1_FORMS[args.level1])
    if args.once:
        rs, st = ctx.skeleton_batch(Xd, alphas, batch_direct=True)
        for r in rs:
            r.free()
        print(json.dumps({"workload": args.workload, "levels": st["levels"], "total_ms": st["total_ms"],
                          "kernel_launches": st["kernel_launches"], "level_source_hash": level_source_hash()}))
        ctx.close()
        return 0
    tune = {}
    if args.tune:
        table = ctx.autotune_batch(Xd, alphas, reps=2)
        tune = {k: table[0][k] for k in ("chunk", "ctas_per_sm", "corr_kps")}
    res, bst = ctx.skeleton_batch(Xd, alphas, **tune)
    units = int(sum(bst["serial_tests"]))
    edges = int(bst["edges_final"])
    for r in res:
        r.free()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        for r in ctx.skeleton_batch(Xd, alphas, **tune)[0]:
            r.free()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms, launches, stats = 0.0, 0, []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            rs, st = ctx.skeleton_batch(Xd, alphas, **tune)
            for r in rs:
                r.free()
            total_ms += st["total_ms"]
            launches += st["kernel_launches"]
            stats.append(st)
    if dist:
        dist.barrier()
    clocks = clk.summary()
    t = torch.tensor([total_ms], device=dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = units * world * args.steps / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps

    # the same problems one call each (FP32+recheck, and the plain FP64 form):
    # device time of every skeleton summed
    sequential = None
    if not args.no_plain:
        sequential = {}
        for name, m in (("fp32_recheck", cupc.MODE_FP32_RECHECK), ("plain_fp64", cupc.MODE_PLAIN_FP64)):
            for X in Xd[:2]:
                ctx.skeleton(X, probs[0].alpha, mode=m).free()      # warm-up
            tot = 0.0
            for X, s in zip(Xd, probs):
                r = ctx.skeleton(X, s.alpha, mode=m)
                tot += r.stats()["total_ms"]
                r.free()
            sequential[name] = {"ms": round(tot, 3), "value": units / (tot * 1e-3), "unit": UNIT}
        sequential["batched_speedup_vs_fp32_calls"] = round(sequential["fp32_recheck"]["ms"] / ms_per_step, 2)
        sequential["batched_speedup_vs_plain_calls"] = round(sequential["plain_fp64"]["ms"] / ms_per_step, 2)

    e2e = None
    if not args.no_e2e:
        Xh = [torch.from_numpy(s.Xt.astype(np.float32)).pin_memory().T for s in probs]
        for r in ctx.skeleton_batch(Xh, alphas, **tune)[0]:
            r.free()
        secs, h2d, d2h = 0.0, 0, 0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            rs, st = ctx.skeleton_batch(Xh, alphas, **tune)
            for r in rs:
                r.edges()
                r.records_raw()
            secs += time.perf_counter() - t0
            for r in rs:
                r.free()
            h2d += st["h2d_bytes"]
            d2h += st["d2h_bytes"]
        e2e = {"value": units * args.steps / secs, "unit": UNIT, "ms_per_step": 1e3 * secs / args.steps,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    peaks = _peaks()
    kern_all = [batch_rooflines(st, probs, peaks) for st in stats]
    kern = {}
    for nm in kern_all[0]:
        rs = [k[nm] for k in kern_all if nm in k]
        d = dict(rs[0])
        d["ms"] = sum(x["ms"] for x in rs) / len(rs)
        d["achieved"] = sum(x["achieved"] for x in rs) / len(rs)
        d["frac"] = d["achieved"] / d["peak"]
        kern[nm] = d
    dom = max(kern, key=lambda k: kern[k]["ms"])
    roof = {k: kern[dom][k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roof["kernel"] = dom
    roof["ms_per_step"] = kern[dom]["ms"]
    phases = {k: round(sum(st["kernel_ms"][k] for st in stats) / len(stats), 4) for k in stats[0]["kernel_ms"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        secs, cu, used = 0.0, 0, 0
        for s in probs:                       # a bounded sample: problems in order until 15 s
            t_, u_ = cpu_oracle_run(s, cores)
            secs += t_
            cu += u_
            used += 1
            if secs > 15.0:
                break
        cpu = {"value": cu / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {used} of {len(probs)} problems, one by one, {secs:.2f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic (seeded linear-Gaussian SEMs, device-resident input)",
                "config": _batch_config(args.workload, probs, "FP32 bulk + FP64 recheck, batched"),
                "skeleton_wall_s": ms_per_step / 1e3, "serial_tests_per_step": units, "edges": edges,
                "cuda_graph": stats[0]["cuda_graph"], "tuned": tune or None, "sequential_calls": sequential,
                "e2e": e2e, "gpu_launches": launches, "phase_ms_per_step": phases,
                "roofline": roof,
                "kernel_rooflines": {k: {"frac": round(v["frac"], 5), "achieved": round(v["achieved"], 3),
                                         "unit": v["unit"], "bound": v["bound"], "ms": round(v["ms"], 4)}
                                     for k, v in kern.items()},
                "cpu_baseline": cpu, "clocks": clocks}
        print(json.dumps(line))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="medium1000")
    ap.add_argument("--mode", default="fp32", choices=["fp32", "plain"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP64 form")
    ap.add_argument("--tune", action="store_true", help="batch workloads: autotune the launch configuration")
    ap.add_argument("--learned", action="store_true",
                    help="learned subset ordering: train the network on 200 seeded p=500 instances first")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large10000 leg (p = 10^4) of the medium1000 line")
    ap.add_argument("--no-learned-leg", action="store_true",
                    help="skip the learned-ordering form of the large10000 leg")
    ap.add_argument("--sshare", action="store_true",
                    help="print the global-sharing diagnostic (Sec. 5.5) per workload and level, then exit")
    ap.add_argument("--sweep", action="store_true",
                    help="run the scalability sweep of Sec. 5.6 (levels 0-2) and print one line per point, then exit")
    ap.add_argument("--sweep-graphs", type=int, default=3, help="graphs per sweep point (the paper uses 10)")
    ap.add_argument("--sweep-no-parity", action="store_true", help="sweep without the oracle runs")
    ap.add_argument("--level1", default="auto", choices=sorted(L1_FORMS),
                    help="level-1 form: the library's choice, by conditioning variable (pivot) or by row")
    ap.add_argument("--once", action="store_true",
                    help="run one skeleton of the workload and print its per-level stats (the command profiled)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args, args.workload)

    import numpy as np
    import torch

    import paper_1812_08491_gb300 as cupc
    from synth import sem

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload in BATCH_WORKLOADS:
        rc = main_batch(args, world, rank, local, dist)
        if dist:
            dist.destroy_process_group()
        return rc

    cupc.build_library()
    s = sem.workload(args.workload)
    Xd = torch.from_numpy(s.Xt).to(dev)          # p x n rows; X = Xd.T is variable-major n x p
    X = Xd.T
    ctx = cupc.Context(local, level1_form=L1_FORMS[args.level1])
    mode = cupc.MODE_FP32_RECHECK if args.mode == "fp32" else cupc.MODE_PLAIN_FP64
    if args.once:
        r = ctx.skeleton(X, s.alpha, mode=mode, canonical=True, max_level=s.max_level)
        st = r.stats()
        r.free()
        print(json.dumps({"workload": args.workload, "levels": st["levels"], "total_ms": st["total_ms"],
                          "kernel_launches": st["kernel_launches"], "level_source_hash": level_source_hash(),
                          "ci_block_entries": st["ci_block_entries"], "edges_start": st["edges_start"]}))
        ctx.close()
        return 0
    if args.sshare:
        sshare_report(ctx, dev)
        ctx.close()
        return 0
    if args.sweep:
        sweep_report(ctx, dev, args.sweep_graphs, parity=not args.sweep_no_parity)
        ctx.close()
        return 0
    peaks_alu = ctx.device_peaks()
    learned_info = None
    if args.learned:
        # the ordering network, trained on the GPU from the plain method's SepSets
        from paper_1812_08491_gb300 import learned
        t0 = time.perf_counter()
        train_probs = [sem.mlp_training_instance(k) for k in range(200)]
        Xtr, ttr = learned.collect(ctx, train_probs)
        losses = learned.train(ctx, Xtr, ttr, epochs=6, batch=4096, lr=2e-3)
        learned_info = {"train_instances": 200, "train_examples": int(Xtr.shape[0]),
                        "positive_rate": round(float(ttr.mean()), 4),
                        "loss_first_last": [round(float(losses[0]), 4), round(float(losses[-1]), 4)],
                        "setup_s": round(time.perf_counter() - t0, 1)}
    stream = torch.cuda.current_stream(dev)

    # the unit count: serial-order tests of the canonical run (equal to the oracle's)
    ref = ctx.skeleton(X, s.alpha, mode=mode, canonical=True, max_level=s.max_level)
    ref_serial = list(ref.stats()["serial_tests"])
    units = int(sum(ref_serial))
    edges = int(ref.stats()["edges_final"])
    ref.free()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # the options of each form, built once (the public call takes them as given)
    form_opts = {m: ctx.options(mode=m, canonical=True, max_level=s.max_level,
                                learned_order=bool(args.learned) and m == cupc.MODE_FP32_RECHECK)
                 for m in (cupc.MODE_FP32_RECHECK, cupc.MODE_PLAIN_FP64)}
    # FP32 form in lexicographic order (compared with the learned order)
    form_opts["lex32"] = ctx.options(mode=cupc.MODE_FP32_RECHECK, canonical=True, max_level=s.max_level)

    def step(m, done=None):
        """One skeleton call; `done` (a CUDA event) is recorded as soon as the call
        returns, before the result's statistics are read and its memory freed."""
        res = ctx.skeleton(X, s.alpha, form_opts[m])
        if done is not None:
            done.record(stream)
        st = res.stats()
        res.free()
        return st

    if args.learned:
        st_l = step(mode)
        learned_info["serial_tests_learned"] = int(sum(st_l["serial_tests"]))
        learned_info["serial_tests_lexicographic"] = units
        learned_info["serial_tests_saved_levels_ge1"] = int(sum(ref_serial[1:]) - sum(st_l["serial_tests"][1:]))
        learned_info["serial_tests_per_level_learned"] = [int(v) for v in st_l["serial_tests"]]
        learned_info["serial_tests_per_level_lexicographic"] = [int(v) for v in ref_serial]

    for _ in range(args.warmup):
        step(mode)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = 0.0
    roofs = []
    launches = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = step(mode, b)
            torch.cuda.synchronize()
            total_ms += a.elapsed_time(b)
            launches += st["kernel_launches"]
            roofs.append((st, kernel_rooflines(st, s, args.mode, _peaks(), peaks_alu)))
    if dist:
        dist.barrier()
    clocks = clk.summary()
    t = torch.tensor([total_ms], device=dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = units * world * args.steps / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps

    # plain form (FP64 for every test) on the same input
    plain = None
    if args.mode == "fp32" and not args.no_plain:
        k2 = max(2, args.steps // 2)
        step(cupc.MODE_PLAIN_FP64)
        pm = 0.0
        for _ in range(k2):
            flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(cupc.MODE_PLAIN_FP64, b)
            torch.cuda.synchronize()
            pm += a.elapsed_time(b)
        plain = {"value": units * k2 / (pm * 1e-3), "unit": UNIT, "ms_per_step": pm / k2, "steps": k2}
    if learned_info is not None and args.mode == "fp32":
        # the same FP32 form in lexicographic order, timed the same way
        step("lex32")
        lm_ = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step("lex32", b)
            torch.cuda.synchronize()
            lm_ += a.elapsed_time(b)
        learned_info["fp32_lexicographic_ms_per_step"] = lm_ / args.steps
        learned_info["fp32_learned_ms_per_step"] = ms_per_step

    # end to end through the public call with a pinned host input: the skeleton
    # with its host lists (edge list and SepSet records, built on the device and
    # downloaded with the call's final readback), then both read on the host
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(s.Xt).pin_memory()
        Xhv = Xh.T
        e2e_opts = ctx.options(mode=mode, canonical=True, max_level=s.max_level, host_lists=True,
                               learned_order=bool(args.learned) and mode == cupc.MODE_FP32_RECHECK)
        r = ctx.skeleton(Xhv, s.alpha, e2e_opts)
        r.edges(); r.records_raw(); r.free()
        secs, h2d, d2h = 0.0, 0, 0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            r = ctx.skeleton(Xhv, s.alpha, e2e_opts)
            r.edges()
            r.records_raw()
            secs += time.perf_counter() - t0
            st = r.stats()
            h2d += st["h2d_bytes"]
            d2h += st["d2h_bytes"]
            r.free()
        e2e = {"value": units * args.steps / secs, "unit": UNIT, "ms_per_step": 1e3 * secs / args.steps,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    # per-kernel rooflines averaged over the timed steps; the dominant kernel is
    # the one with the largest device time
    names = set().union(*[r.keys() for _, r in roofs])
    kern = {}
    for nm in names:
        rs = [r[nm] for _, r in roofs if nm in r]
        ms = sum(x["ms"] for x in rs) / len(rs)
        first = dict(rs[0])
        first["ms"] = ms
        first["achieved"] = sum(x["achieved"] for x in rs) / len(rs)
        first["frac"] = first["achieved"] / first["peak"]
        kern[nm] = first
    dom = max((k for k in kern if k != "recheck"), key=lambda k: kern[k]["ms"])
    if "level" in kern:
        kern["level"]["traffic"] = committed_traffic(args.workload)
    roof = {k: kern[dom][k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roof["kernel"] = dom
    roof["ms_per_step"] = kern[dom]["ms"]
    roof["peak_src"] = "measured (MEASURED_PEAKS.json)" if _peaks()["src"] == "measured" else "fallback"
    roof["alg_bytes_per_launch"] = kern[dom].get("alg_bytes_per_launch")
    kernels = {k: round(v["ms"], 4) for k, v in kern.items()}
    phases = {k: round(sum(st["kernel_ms"][k] for st, _ in roofs) / len(roofs), 4)
              for k in roofs[0][0]["kernel_ms"]}

    cpu = None
    keep = {}
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        secs, cu = cpu_oracle_run(s, cores, keep)
        cpu = {"value": cu / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"whole {args.workload} skeleton once (correlation + all levels), {secs:.2f} s"}
        # the oracle on one core (the serial analogue), when that stays within ~30 s
        if secs * cores <= 30.0:
            s1, cu1 = cpu_oracle_run(s, 1)
            cpu["serial_1core"] = {"value": cu1 / s1, "unit": UNIT, "seconds": round(s1, 3)}
    orient = orientation_line(ctx, X, s, mode, keep.get("res")) if rank == 0 else None
    large = None
    if rank == 0 and args.workload == "medium1000" and args.mode == "fp32" and not args.no_large:
        with ClockSampler(local) as clk2:
            large = large_leg(ctx, args, peaks_alu, dev, stream, flush, {})
        large["clocks"] = clk2.summary()
    lbounds = level_bounds(roofs[-1][0], args.mode, _peaks(), peaks_alu)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if args.mode == "fp32" else "f64",
                "data": "synthetic (seeded linear-Gaussian SEM, device-resident input)",
                "config": _config(args.workload, s, ("FP32 bulk + FP64 recheck" +
                                                     (" + learned ordering" if args.learned else ""))
                                  if args.mode == "fp32" else "plain FP64"),
                "learned": learned_info,
                "skeleton_wall_s": ms_per_step / 1e3, "serial_tests_per_step": units, "edges": edges,
                "plain_form": plain,
                "speedup_vs_plain": (plain["ms_per_step"] / ms_per_step) if plain else None,
                "e2e": e2e, "gpu_launches": launches, "kernel_ms_per_step": kernels,
                "phase_ms_per_step": phases,
                "roofline": roof,
                "kernel_rooflines": {k: {"frac": round(v["frac"], 5), "achieved": round(v["achieved"], 3),
                                         "unit": v["unit"], "bound": v["bound"]} for k, v in kern.items()},
                "cpu_baseline": cpu, "clocks": clocks, "orientation": orient,
                "level_bounds": lbounds, "large10000": large,
                "alu_peaks_measured": {k: round(v, 2) for k, v in peaks_alu.items()},
                "level_source_hash": level_source_hash()}
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark of the FP64 hot path on one synthetic coronal grid (128 x 192 x 384 cells).

One step = one pass over every step of the path, through the C ABI:
  conduction: set_coeffs (+ Gershgorin dt_exp); RKL2 super-steps at dt/dt_exp = 100,
              1000, 10000 (s = 20, 63, 200); BE+PCG to rtol 1e-10 at the same three
              dt with point Jacobi and with 8x8x8 block ILU0;
  viscosity:  set_coeffs; RKL2 at dt/dt_exp = 500 (s = 45) and BE+PCG (Jacobi, block
              ILU0) at the same dt, on the three Cartesian velocity components.
Metric: cell-updates/s = cells x (RKL2 stages + PCG iterations, per component) / time.

Timing: W untimed warm-up steps, then K steps between barriers and device syncs, CUDA
events on the library's stream, max over ranks, on the library's default path (the
RKL2 super-steps and the PCG loops run as CUDA graphs).  The per-kernel times of the
roofline come from one more step run right after, with the library's event profiler on
(every launch bracketed by events, graphs off), so that the timed steps carry no
instrumentation.  The working set of every stage pass (~1.2 GB) is far larger than the
129 MB L2, so no flush is needed between steps.  Several GPUs (torchrun) run independent
replicas (one grid per GPU, no exchange).  `--impl reference` times the FP64 CPU oracle
instead (bounded sample, host cores).

The line's `detail` also times, once, the other configurations of the comparison:
32 x 32 x 64 (RKL2 and BE + PCG-Jacobi, FP64, next to the oracle's full run of the same on
the host cores), 256 x 384 x 768 (mixed precision against FP64) and 192 x 288 x 576
(viscosity, FP64 against FP32 mixed precision, RKL2 against BE + PCG-Jacobi).
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = (128, 192, 384)
RATIOS = (100.0, 1000.0, 10000.0)
VISC_RATIO = 500.0
RTOL = 1e-10
MAXIT = 20000
BLOCK = (8, 8, 8)
BETA_TCUT = True  # kappa0 T^{5/2} times the printed factor (T / 5e5 K)^{5/2} below 5e5 K (Sec. 4.1 beta_Tcut)
FP64_PEAK_TFLOPS = 1.25  # nominal FP64 rate of the GB300 (2 DFMA/clk/SM x 152 SMs x 2.07 GHz)
# Algorithmic cost per cell of one launch of each kernel family (one field component):
# (flop, bytes, binding unit, ncu summary, sources the summary was taken on).
#  rkl2_stage cond: 19 stencil FMA + 1/W scaling + 5 recurrence terms = 48 flop;
#                   10 coefficients + 1/W + Y_{j-1}, Y_{j-2}, Y_0, M_0 read, Y_j written = 128 B
#  rkl2_stage visc: 7 FMA + 1 + 9 = 24 flop; 4 coefficients + 1/W + 5 fields = 80 B
#  spmv cond: y = A p with A = W + dt S assembled once per solve: 19 FMA + p.y = 40 flop;
#             10 coefficients of A + p + y = 96 B
#  spmv visc: 7 FMA + p.y = 16 flop; 4 coefficients + p + y = 48 B
#  bilu_apply cond: 9 + 9 FMA + 1/U_ii + r.z = 39 flop; 19 factors + r + z = 168 B
#                   (r.r is formed by the x, r update that precedes it)
#  bilu_apply visc: 3 + 3 FMA + 1 + 2 = 15 flop; 7 factors + r + z = 72 B
KERNEL_COST = {
    ("conduction", "rkl2_stage"): (48.0, 128.0, "alu", "rkl2_stage_128x192x384.md",
                                   ("rkl2.cu:k_rkl2_stage", "stencil.cuh")),
    ("viscosity", "rkl2_stage"): (24.0, 80.0, "alu", "rkl2_stage_visc_128x192x384.md",
                                  ("rkl2.cu:k_rkl2_stage", "stencil.cuh")),
    ("conduction", "spmv"): (40.0, 96.0, "alu", "spmv_128x192x384.md", ("pcg.cu:k_spmv_a", "stencil.cuh")),
    ("viscosity", "spmv"): (16.0, 48.0, "alu", "spmv_visc_128x192x384.md", ("pcg.cu:k_spmv_a", "stencil.cuh")),
    ("conduction", "bilu_apply"): (39.0, 168.0, "alu", "bilu_apply_128x192x384.md", ("pcg.cu:k_bilu_apply",)),
    ("viscosity", "bilu_apply"): (15.0, 72.0, "alu", "bilu_apply_visc_128x192x384.md", ("pcg.cu:k_bilu_apply",)),
}
# part of the demangled ncu kernel name of each family (for --summarize-ncu)
FAMILY_KERNEL = {
    ("conduction", "rkl2_stage"): "k_rkl2_stage<0>", ("viscosity", "rkl2_stage"): "k_rkl2_stage<1>",
    ("conduction", "spmv"): "k_spmv_a<0>", ("viscosity", "spmv"): "k_spmv_a<1>",
    ("conduction", "bilu_apply"): "k_bilu_apply<0, double>", ("viscosity", "bilu_apply"): "k_bilu_apply<1, double>",
}
WORKLOAD = "coronal FP64 conduction+viscosity, 128x192x384 spherical grid"


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-accuracy", action="store_true")
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--mixed-large", action="store_true",
                   help="run the mixed-precision comparison at 256x384x768 (75.5 M cells) instead of the step")
    p.add_argument("--warmstart", action="store_true",
                   help="run the learned-initial-guess study (200 BE steps with heating) instead of the step")
    p.add_argument("--profile", choices=("stage", "apply", "pcg-jacobi", "pcg-bilu0", "setup", "stage-mix",
                                         "pcg-jacobi-mix", "pcg-bilu0-mix", "ws-forward", "ws-train",
                                         "visc-stage", "visc-pcg-jacobi", "visc-pcg-bilu0"),
                   help="run only a minimal case of one kernel family for an ncu capture (no timing)")
    p.add_argument("--profile-grid", type=int, nargs=3, metavar=("NR", "NTH", "NPH"), default=list(GRID),
                   help="grid of the --profile case (default the bench grid); a smaller grid keeps an ncu "
                        "capture of many passes small")
    p.add_argument("--plain-launches", action="store_true",
                   help="run every step with the library's event profiler on (plain launches, no graphs), so "
                        "that an ncu launch list sees every kernel; not a bench number")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the 32x32x64, 256x384x768 and 192x288x576 lines of detail")
    p.add_argument("--summarize-ncu", nargs=3, metavar=("REPORT", "FAMILY", "OUT"),
                   help="write a profile summary (metrics, traffic, source hash, capture date) of the kernel of "
                        "FAMILY (e.g. conduction/spmv) from an ncu report, then exit")
    p.add_argument("--summary-command", default="", help="command line recorded in the --summarize-ncu summary")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def base_config():
    return {
        "workload": WORKLOAD,
        "grid_nr_nth_nph": list(GRID),
        "cells": GRID[0] * GRID[1] * GRID[2],
        "rkl2_dt_over_dt_exp": list(RATIOS),
        "be_dt_over_dt_exp": list(RATIOS),
        "pcg": ["jacobi", "bilu0-8x8x8"],
        "rtol": RTOL,
        "beta_tcut": BETA_TCUT,
        "viscosity_dt_over_dt_exp": VISC_RATIO,
        "l2": "no flush: every stage pass streams ~1.2 GB, far above the 129 MB L2",
        "graphs": "library default: RKL2 super-steps and PCG loops replayed as CUDA graphs in the timed steps",
    }


# ------------------------------------------------------------------ CPU oracle sample
# PCG iteration counts of the timed step at this configuration (the oracle's, which the GPU
# path matches to within one: tests/golden/bench_config_iters.json); RKL2 stage counts
# follow from Eq. 5
STEP_ITERS = {"jacobi": (72, 238, 733), "bilu0": (31, 126, 422),
              "visc_jacobi": (143, 142, 126), "visc_bilu0": (52, 52, 47)}
# stages / iterations of each part timed per CPU sample (viscosity on one component)
CPU_PARTS = {"rkl2_c": 4, "jacobi_c": 6, "bilu0_c": 4, "rkl2_v": 2, "jacobi_v": 4, "bilu0_v": 2}


def step_mix():
    """Work of one timed step in cell passes per part (RKL2 stages, PCG iterations; viscosity
    summed over its three components) and its one-off parts."""
    import oracle as O

    return {"rkl2_c": sum(O.rkl2_stages(r) for r in RATIOS), "jacobi_c": sum(STEP_ITERS["jacobi"]),
            "bilu0_c": sum(STEP_ITERS["bilu0"]), "rkl2_v": 3 * O.rkl2_stages(VISC_RATIO),
            "jacobi_v": sum(STEP_ITERS["visc_jacobi"]), "bilu0_v": sum(STEP_ITERS["visc_bilu0"]),
            "factor_c": len(RATIOS), "factor_v": 1, "assembly": 2}


def cpu_sample(seed: int):
    """The FP64 CPU oracle (host cores) on one timed step's work mix, on the full grid: each
    part (conduction RKL2 stages, PCG-Jacobi and PCG-block-ILU0 iterations; the same for
    viscosity, one component) is timed on CPU_PARTS stages or iterations and weighted by its
    count in the step; the step's block-ILU0 factorisations and operator assemblies are
    timed once at set-up and counted at their per-step number.  run() returns the time the
    sample's cell passes take at that mix, so units / run() is the oracle's rate on the
    step's mix."""
    import oracle as O

    from paper_1610_01265_gb300 import synth

    nr, nth, nph = GRID
    c = synth.conduction_case(nr, nth, nph, seed)
    v = synth.viscosity_case(nr, nth, nph, seed)
    g = O.Grid(c["rf"], nth, nph)
    t0 = time.perf_counter()
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=BETA_TCUT)
    dte, _ = O.gershgorin_dt(g, S, W)
    t1 = time.perf_counter()
    Sv, Wv = O.assemble_viscosity(g, v["rho"], v["nu"])
    dtv, _ = O.gershgorin_dt(g, Sv, Wv)
    t2 = time.perf_counter()
    O.bilu0_factor(g, O.build_A(S, W, 1000.0 * dte), BLOCK)
    t3 = time.perf_counter()
    O.bilu0_factor(g, O.build_A(Sv, Wv, VISC_RATIO * dtv), BLOCK, pattern=7)
    t4 = time.perf_counter()
    once = {"assembly": (t2 - t0) / 2, "factor_c": t3 - t2, "factor_v": t4 - t3}
    mix = step_mix()
    n = CPU_PARTS
    vv = v["v"][0]

    def timed(f):
        ta = time.perf_counter()
        f()
        return time.perf_counter() - ta

    def run():
        per = {
            "rkl2_c": timed(lambda: O.rkl2_superstep(g, S, W, c["T"], n["rkl2_c"] * dte, n["rkl2_c"])) / n["rkl2_c"],
            "jacobi_c": timed(lambda: O.be_pcg(g, S, W, c["T"], 1000.0 * dte, pc=O.PC_JACOBI,
                                               fixed_iters=n["jacobi_c"])) / n["jacobi_c"],
            "bilu0_c": (timed(lambda: O.be_pcg(g, S, W, c["T"], 1000.0 * dte, pc=O.PC_BILU0, block=BLOCK,
                                               fixed_iters=n["bilu0_c"])) - once["factor_c"]) / n["bilu0_c"],
            "rkl2_v": timed(lambda: O.rkl2_superstep(g, Sv, Wv, vv, n["rkl2_v"] * dtv, n["rkl2_v"])) / n["rkl2_v"],
            "jacobi_v": timed(lambda: O.be_pcg(g, Sv, Wv, vv, VISC_RATIO * dtv, pc=O.PC_JACOBI,
                                               fixed_iters=n["jacobi_v"], pattern=7)) / n["jacobi_v"],
            "bilu0_v": (timed(lambda: O.be_pcg(g, Sv, Wv, vv, VISC_RATIO * dtv, pc=O.PC_BILU0, block=BLOCK,
                                               fixed_iters=n["bilu0_v"], pattern=7)) - once["factor_v"])
            / n["bilu0_v"],
        }
        t_step = sum(mix[k] * per[k] for k in per) + sum(mix[k] * once[k] for k in once)
        return sum(n.values()) * t_step / sum(mix[k] for k in per)

    return run, g.N * sum(n.values()), O.num_threads()


def cpu_sample_text():
    import oracle as O

    m = step_mix()
    return (f"the oracle on one bench step's work mix, full 128x192x384 grid: conduction RKL2 "
            f"stages, PCG-Jacobi and PCG-block-ILU0(8^3) iterations (timed on {CPU_PARTS['rkl2_c']}, "
            f"{CPU_PARTS['jacobi_c']} and {CPU_PARTS['bilu0_c']}) and the same for viscosity on one "
            f"component (timed on {CPU_PARTS['rkl2_v']}, {CPU_PARTS['jacobi_v']} and {CPU_PARTS['bilu0_v']}), "
            f"weighted by their counts in the step ({m['rkl2_c']}, {m['jacobi_c']}, {m['bilu0_c']}; "
            f"{m['rkl2_v']}, {m['jacobi_v']}, {m['bilu0_v']} over three components), plus the step's "
            f"{m['factor_c'] + m['factor_v']} block-ILU0 factorisations and 2 operator assemblies (timed "
            f"once); cell-updates = cells x {sum(CPU_PARTS.values())} per sample at the step's mix "
            f"(threads: {O.num_threads()})")


C1_GRID = (32, 32, 64)
C1_RATIO = 100.0


def cpu_model():
    """Host CPU model and core count (lscpu, else /proc/cpuinfo)."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    name = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform

    return {"model": name or platform.processor() or platform.machine(), "machine": platform.machine(),
            "logical_cpus": os.cpu_count()}


def cpu_c1_full(seed: int, threads: int | None = None):
    """The oracle's full run of the 32 x 32 x 64 configuration on the host cores: conduction
    with beta_Tcut, one RKL2 super-step at 100 dt_exp (s = 20) and one BE step by PCG-Jacobi
    to rtol 1e-10 at the same dt; operator assembly and Gershgorin timed separately."""
    import oracle as O

    from paper_1610_01265_gb300 import synth

    nr, nth, nph = C1_GRID
    c = synth.conduction_case(nr, nth, nph, seed)
    g = O.Grid(c["rf"], nth, nph)
    prev = O.num_threads()
    if threads:
        O.set_num_threads(threads)
    try:
        used = O.num_threads()
        t0 = time.perf_counter()
        S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=BETA_TCUT)
        dte, _ = O.gershgorin_dt(g, S, W)
        t1 = time.perf_counter()
        s = O.rkl2_stages(C1_RATIO)
        O.rkl2_superstep(g, S, W, c["T"], C1_RATIO * dte, s)
        t2 = time.perf_counter()
        _, its, rel, st = O.be_pcg(g, S, W, c["T"], C1_RATIO * dte, pc=O.PC_JACOBI, rtol=RTOL, maxit=MAXIT)
        t3 = time.perf_counter()
    finally:
        O.set_num_threads(prev)
    units = g.N * (s + its)
    return {"threads": used, "setup_ms": 1e3 * (t1 - t0), "rkl2_ms": 1e3 * (t2 - t1), "s": s,
            "be_jacobi_ms": 1e3 * (t3 - t2), "be_jacobi_iters": its, "be_converged": st == 0,
            "cell_updates_per_s": units / (t3 - t1)}


def cpu_baseline_leg(seed: int):
    """cpu_baseline of the bench line: the bounded sample of the timed workload on all host
    cores (value), plus a single-thread rate and the oracle's full 32 x 32 x 64 run."""
    run, units, cores = cpu_sample(seed)
    t = run()
    out = {"value": units / t, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
           "sample": cpu_sample_text(), "seconds": t, "host": cpu_model()}
    one = cpu_c1_full(seed, threads=1)
    out["single_thread"] = {"value": one["cell_updates_per_s"], "unit": "cell-updates/s", "cores": 1,
                            "sample": "the oracle's full 32x32x64 run (RKL2 s=20 + BE-Jacobi to 1e-10 at "
                                      "100 dt_exp), one thread", "detail": one}
    out["c1_full_all_cores"] = cpu_c1_full(seed)
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    run, units, cores = cpu_sample(args.seed)
    for _ in range(max(args.warmup, 0)):
        run()
    times = [run() for _ in range(args.steps)]
    total = sum(times)
    value = units * args.steps / total
    line = {
        "metric": "cell-updates/s",
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": base_config(),
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": cpu_sample_text()},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _function_text(text, func):
    """Source of the __global__ function `func` (with its template line), or the whole text."""
    m = re.search(r"__global__[^;{]*?\b" + re.escape(func) + r"\s*\(", text)
    if not m:
        return text
    start = text.rfind("\n", 0, m.start()) + 1
    prev = text.rfind("\n", 0, start - 1) + 1
    if text[prev:start].lstrip().startswith("template"):
        start = prev
    depth, pos = 0, text.index("{", m.end())
    for q in range(pos, len(text)):
        if text[q] == "{":
            depth += 1
        elif text[q] == "}":
            depth -= 1
            if depth == 0:
                return text[start:q + 1]
    return text[start:]


def kernel_source_hash(names=("rkl2.cu:k_rkl2_stage", "stencil.cuh")):
    """Hash of the source a kernel is built from: 'file:function' hashes that function's
    text, 'file' the whole file (headers the kernel includes)."""
    h = hashlib.sha256()
    for name in names:
        fname, _, func = name.partition(":")
        with open(os.path.join(ROOT, "paper_1610_01265_gb300", "csrc", fname)) as f:
            text = f.read()
        h.update((_function_text(text, func) if func else text).encode())
    return h.hexdigest()[:16]


def profiled_traffic(summary, sources):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, if that summary
    was taken on the current source of the kernel (else None)."""
    if not summary:
        return None
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != kernel_source_hash(sources):
        return None
    return float(m.group(1))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class Workload:
    def __init__(self, R, torch, seed: int, host: bool = False):
        from paper_1610_01265_gb300 import synth

        self.R, self.torch = R, torch
        nr, nth, nph = GRID
        self.N = nr * nth * nph
        c = synth.conduction_case(nr, nth, nph, seed)
        v = synth.viscosity_case(nr, nth, nph, seed)
        self.host = host
        if host:
            pin = lambda a: torch.from_numpy(np.array(a, dtype=np.float64).reshape(-1)).pin_memory().numpy()  # noqa: E731
            self.T, self.b, self.n = pin(c["T"]), pin(c["bhat"]), pin(c["n"])
            self.rho, self.nu, self.v = pin(v["rho"]), pin(v["nu"]), pin(v["v"])
            self.u = pin(np.empty(self.N))
            self.uv = pin(np.empty(3 * self.N))
        else:
            dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda()  # noqa: E731
            self.T, self.b, self.n = dev(c["T"]).view(-1), dev(c["bhat"]).view(-1), dev(c["n"]).view(-1)
            self.rho, self.nu, self.v = dev(v["rho"]).view(-1), dev(v["nu"]).view(-1), dev(v["v"]).view(-1)
            self.u = torch.empty_like(self.T)
            self.uv = torch.empty_like(self.v)
        self.ctx_c = R.Context(c["rf"], nth, nph)
        self.ctx_v = R.Context(v["rf"], nth, nph)
        self.h2d = 0
        self.d2h = 0

    def _load(self, dst, src):
        if self.host:
            np.copyto(dst, src)
        else:
            dst.copy_(src)

    def launches(self):
        return self.ctx_c.kernel_launches + self.ctx_v.kernel_launches

    def step(self):
        """One pass over the hot path; returns (cell-updates, per-path details)."""
        R, N = self.R, self.N
        units = 0
        info = {"rkl2": {}, "be": {}, "visc": {}}
        self.h2d = self.d2h = 0
        dte = self.ctx_c.set_conduction(self.T, self.b, self.n, beta_tcut=BETA_TCUT)
        self.h2d += 5 * N * 8
        for ratio in RATIOS:
            self._load(self.u, self.T)
            s = self.ctx_c.rkl2_superstep(self.u, ratio * dte, dte)
            units += N * s
            info["rkl2"][str(int(ratio))] = {"s": s}
            self.h2d += N * 8
            self.d2h += N * 8
        for pc, name in ((R.RKL_PC_JACOBI, "jacobi"), (R.RKL_PC_BILU0, "bilu0")):
            for ratio in RATIOS:
                self._load(self.u, self.T)
                code, its, rel = self.ctx_c.be_pcg_solve(self.u, ratio * dte, pc=pc, block=BLOCK, rtol=RTOL,
                                                         maxit=MAXIT)
                if code != R.RKL_OK:
                    raise RuntimeError(f"BE+PCG({name}) at {ratio} did not converge: {R.strerror(code)}")
                units += N * its[0]
                info["be"][f"{name}_{int(ratio)}"] = {"iters": its[0], "relres": rel[0]}
                self.h2d += N * 8
                self.d2h += N * 8
        dtv = self.ctx_v.set_viscosity(self.rho, self.nu)
        self.h2d += 2 * N * 8
        self._load(self.uv, self.v)
        s = self.ctx_v.rkl2_superstep(self.uv, VISC_RATIO * dtv, dtv, ncomp=3)
        units += 3 * N * s
        info["visc"]["rkl2"] = {"s": s}
        self.h2d += 3 * N * 8
        self.d2h += 3 * N * 8
        for pc, name in ((R.RKL_PC_JACOBI, "jacobi"), (R.RKL_PC_BILU0, "bilu0")):
            self._load(self.uv, self.v)
            code, its, rel = self.ctx_v.be_pcg_solve(self.uv, VISC_RATIO * dtv, pc=pc, block=BLOCK, rtol=RTOL,
                                                     maxit=MAXIT, ncomp=3)
            if code != R.RKL_OK:
                raise RuntimeError(f"viscosity BE+PCG({name}) did not converge: {R.strerror(code)}")
            units += N * sum(its)
            info["visc"][f"be_{name}"] = {"iters": its, "relres": max(rel)}
            self.h2d += 3 * N * 8
            self.d2h += 3 * N * 8
        info["dt_exp_conduction_s"] = dte
        info["dt_exp_viscosity_s"] = dtv
        return units, info


def path_timings(wl, torch):
    """ms per large step of each path (after the timed region, device-resident)."""
    R = wl.R
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dte = wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
    e0.record()
    wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
    e1.record()
    torch.cuda.synchronize()
    out["set_coeffs_conduction_ms"] = e0.elapsed_time(e1)
    for ratio in RATIOS:
        wl.u.copy_(wl.T)
        e0.record()
        s = wl.ctx_c.rkl2_superstep(wl.u, ratio * dte, dte)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[f"rkl2_{int(ratio)}"] = {"s": s, "ms": ms, "cell_updates_per_s": wl.N * s / ms * 1e3}
        for pc, name in ((R.RKL_PC_JACOBI, "jacobi"), (R.RKL_PC_BILU0, "bilu0")):
            wl.u.copy_(wl.T)
            e0.record()
            code, its, rel = wl.ctx_c.be_pcg_solve(wl.u, ratio * dte, pc=pc, block=BLOCK, rtol=RTOL, maxit=MAXIT)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[f"be_{name}_{int(ratio)}"] = {"iters": its[0], "ms": ms,
                                              "cell_updates_per_s": wl.N * its[0] / ms * 1e3}
    return out


def mixed_report(wl, R, torch):
    """Mixed precision (FP32 stages / FP32 PCG with FP64 refinement) against the FP64 GPU
    path on the same inputs: ms per large step and error relative to the step's change."""
    nr, nth, nph = GRID
    out = {}
    mix = R.Context(wl.ctx_c._rf, nth, nph, prec=R.RKL_F32MIX)
    try:
        dte = mix.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
        wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ref = torch.empty_like(wl.T)
        for ratio in RATIOS:
            ref.copy_(wl.T)
            wl.ctx_c.rkl2_superstep(ref, ratio * dte, dte)
            wl.u.copy_(wl.T)
            mix.rkl2_superstep(wl.u, ratio * dte, dte)  # warm
            wl.u.copy_(wl.T)
            e0.record()
            s = mix.rkl2_superstep(wl.u, ratio * dte, dte)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            err = (torch.linalg.vector_norm(wl.u - ref) / torch.linalg.vector_norm(ref - wl.T)).item()
            err_u = (torch.linalg.vector_norm(wl.u - ref) / torch.linalg.vector_norm(ref)).item()
            out[f"rkl2_{int(ratio)}"] = {"s": s, "ms": ms, "cell_updates_per_s": wl.N * s / ms * 1e3,
                                         "err_rel_change": err, "err_rel_u": err_u}
            for pc, name in ((R.RKL_PC_JACOBI, "jacobi"), (R.RKL_PC_BILU0, "bilu0")):
                wl.u.copy_(wl.T)
                e0.record()
                code, its, rel = mix.be_pcg_solve(wl.u, ratio * dte, pc=pc, block=BLOCK, rtol=RTOL, maxit=MAXIT)
                e1.record()
                torch.cuda.synchronize()
                out[f"be_{name}_{int(ratio)}"] = {"fp32_iters": its[0], "relres_fp64": rel[0],
                                                  "ms": e0.elapsed_time(e1), "converged": code == R.RKL_OK}
    finally:
        mix.close()
    return out


def flux_report(wl, torch):
    """The non-symmetric flux form of conduction (RKL_FLUX_FORM) next to the symmetric form
    on the same inputs: ms per large step and PCG iterations (RKL2 and block-ILU0 PCG at
    dt = 1000 dt_exp, Jacobi PCG at 30 and, capped, at 1000 dt_exp)."""
    R = wl.R
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, flux in (("symmetric", False), ("flux_form", True)):
        e0.record()
        dte = wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT, flux_form=flux)
        e1.record()
        torch.cuda.synchronize()
        r = {"set_coeffs_ms": e0.elapsed_time(e1), "dt_exp_s": dte}
        wl.u.copy_(wl.T)
        e0.record()
        s = wl.ctx_c.rkl2_superstep(wl.u, 1000 * dte, dte)
        e1.record()
        torch.cuda.synchronize()
        r["rkl2_1000"] = {"s": s, "ms": e0.elapsed_time(e1)}
        # point Jacobi stalls on the flux form at large dt: capped at 2000 iterations there
        for pc, pname, ratio, maxit in ((R.RKL_PC_JACOBI, "jacobi", 30, MAXIT), (R.RKL_PC_JACOBI, "jacobi", 1000, 2000),
                                        (R.RKL_PC_BILU0, "bilu0", 1000, MAXIT)):
            wl.u.copy_(wl.T)
            e0.record()
            code, its, rel = wl.ctx_c.be_pcg_solve(wl.u, ratio * dte, pc=pc, block=BLOCK, rtol=RTOL, maxit=maxit)
            e1.record()
            torch.cuda.synchronize()
            r[f"be_{pname}_{ratio}"] = {"iters": its[0], "ms": e0.elapsed_time(e1), "relres": rel[0],
                                        "converged": code == R.RKL_OK}
        out[name] = r
    wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
    return out


def variants_report(wl, torch):
    """Sec. 6 remedies at dt = 1000 dt_exp: cost of 10 RKL2 sub-cycles and of an explicit
    Euler prefix over a quarter of the step, next to one RKL2 super-step."""
    dte = wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, kw in (("rkl2", {}), ("rkl2_10_cycles", {"cycles": 10}), ("euler_prefix_0.25", {"euler_fraction": 0.25}),
                     ("rkl1_plus_2", {"scheme": 1, "extra_stages": 2})):
        wl.u.copy_(wl.T)
        e0.record()
        n = wl.ctx_c.sts_advance(wl.u, 1000 * dte, dte, **kw)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"operator_applications": n, "ms": e0.elapsed_time(e1)}
    return out


def accuracy_report(wl, torch, ratios=RATIOS):
    """Relative L2 error of one large step of each method against the semi-discrete
    solution exp(dt M) T, approximated by 64 RKL2 sub-steps of dt/64 (FP64 GPU path)."""
    R = wl.R
    dte = wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
    out = {}
    for ratio in ratios:
        ref = wl.T.clone()
        for _ in range(64):
            wl.ctx_c.rkl2_superstep(ref, ratio * dte / 64, dte)
        nref = torch.linalg.vector_norm(ref - wl.T).item()
        wl.u.copy_(wl.T)
        wl.ctx_c.rkl2_superstep(wl.u, ratio * dte, dte)
        e_rkl = torch.linalg.vector_norm(wl.u - ref).item() / torch.linalg.vector_norm(ref).item()
        wl.u.copy_(wl.T)
        wl.ctx_c.be_pcg_solve(wl.u, ratio * dte, pc=R.RKL_PC_BILU0, block=BLOCK, rtol=RTOL, maxit=MAXIT)
        e_be = torch.linalg.vector_norm(wl.u - ref).item() / torch.linalg.vector_norm(ref).item()
        out[str(int(ratio))] = {"rkl2_rel_l2": e_rkl, "be_rel_l2": e_be,
                                "change_rel_l2": nref / torch.linalg.vector_norm(ref).item()}
    return out


def seeds_report(wl, torch, seeds=(2, 3)):
    """The same conduction paths on the other seeded inputs (the headline uses seed 1):
    stage counts, PCG iterations, ms per large step and accuracy at 1000 dt_exp."""
    from paper_1610_01265_gb300 import synth

    R = wl.R
    nr, nth, nph = GRID
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    T0, b0, n0 = wl.T.clone(), wl.b.clone(), wl.n.clone()
    try:
        for seed in seeds:
            c = synth.conduction_case(nr, nth, nph, seed)
            wl.T.copy_(torch.from_numpy(c["T"].reshape(-1)))
            wl.b.copy_(torch.from_numpy(c["bhat"].reshape(-1)))
            wl.n.copy_(torch.from_numpy(np.array(c["n"]).reshape(-1)))
            r = {"accuracy_1000": accuracy_report(wl, torch, ratios=(1000.0,))["1000"]}
            dte = wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
            wl.u.copy_(wl.T)
            e0.record()
            s = wl.ctx_c.rkl2_superstep(wl.u, 1000 * dte, dte)
            e1.record()
            torch.cuda.synchronize()
            r["rkl2_1000"] = {"s": s, "ms": e0.elapsed_time(e1)}
            for pc, name in ((R.RKL_PC_JACOBI, "jacobi"), (R.RKL_PC_BILU0, "bilu0")):
                wl.u.copy_(wl.T)
                e0.record()
                code, its, rel = wl.ctx_c.be_pcg_solve(wl.u, 1000 * dte, pc=pc, block=BLOCK, rtol=RTOL, maxit=MAXIT)
                e1.record()
                torch.cuda.synchronize()
                r[f"be_{name}_1000"] = {"iters": its[0], "ms": e0.elapsed_time(e1), "converged": code == R.RKL_OK}
            out[str(seed)] = r
    finally:
        wl.T.copy_(T0)
        wl.b.copy_(b0)
        wl.n.copy_(n0)
        wl.ctx_c.set_conduction(wl.T, wl.b, wl.n, beta_tcut=BETA_TCUT)
    return out


def _timed(torch, fn, reps=1):
    """(result of the last call, median ms) of fn() on the current stream, CUDA events."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, r = [], None
    for _ in range(reps):
        torch.cuda.synchronize()
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return r, statistics.median(ms)


def c1_report(R, torch, seed: int):
    """32 x 32 x 64 (the configuration the oracle runs in full): conduction with beta_Tcut,
    RKL2 at 100 dt_exp and BE + PCG-Jacobi to rtol 1e-10 at the same dt, FP64, ms per large
    step (median of 5 after a warm-up, default path), with the difference from the oracle."""
    import oracle as O

    from paper_1610_01265_gb300 import synth

    nr, nth, nph = C1_GRID
    N = nr * nth * nph
    c = synth.conduction_case(nr, nth, nph, seed)
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64).ravel()).cuda()  # noqa: E731
    T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
    out = {"grid_nr_nth_nph": list(C1_GRID), "cells": N, "dt_over_dt_exp": C1_RATIO, "rtol": RTOL,
           "beta_tcut": BETA_TCUT}
    with R.Context(c["rf"], nth, nph) as ctx:
        dte, out["set_coeffs_ms"] = _timed(torch, lambda: ctx.set_conduction(T, b, n, beta_tcut=BETA_TCUT), 5)
        u = torch.empty_like(T)

        def rk():
            u.copy_(T)
            return ctx.rkl2_superstep(u, C1_RATIO * dte, dte)

        rk()
        s, ms = _timed(torch, rk, 5)
        g = O.Grid(c["rf"], nth, nph)
        S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=BETA_TCUT)
        ref = O.rkl2_superstep(g, S, W, c["T"], C1_RATIO * dte, s)
        err = float(np.linalg.norm(u.cpu().numpy() - ref.ravel()) / np.linalg.norm(ref))
        out["rkl2"] = {"s": s, "ms": ms, "cell_updates_per_s": N * s / ms * 1e3, "rel_l2_vs_oracle": err}

        def be():
            u.copy_(T)
            return ctx.be_pcg_solve(u, C1_RATIO * dte, pc=R.RKL_PC_JACOBI, rtol=RTOL, maxit=MAXIT)

        be()
        (code, its, rel), ms = _timed(torch, be, 5)
        x_o, it_o, _, _ = O.be_pcg(g, S, W, c["T"], C1_RATIO * dte, pc=O.PC_JACOBI, rtol=RTOL, maxit=MAXIT)
        out["be_jacobi"] = {"iters": its[0], "oracle_iters": it_o, "ms": ms, "relres": rel[0],
                            "converged": code == R.RKL_OK, "cell_updates_per_s": N * its[0] / ms * 1e3,
                            "rel_l2_vs_oracle": float(np.linalg.norm(u.cpu().numpy() - x_o.ravel())
                                                      / np.linalg.norm(x_o))}
    return out


C4_GRID = (192, 288, 576)


def c4_report(R, torch, seed: int):
    """192 x 288 x 576 viscosity on the three Cartesian components at 500 dt_exp: FP64 against
    FP32 mixed precision, RKL2 (s = 45) against BE + PCG-Jacobi to rtol 1e-10; ms per large
    step, and the difference of each result from the FP64 one relative to the step's
    change."""
    from paper_1610_01265_gb300 import synth

    nr, nth, nph = C4_GRID
    N = nr * nth * nph
    v = synth.viscosity_case(nr, nth, nph, seed)
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64).ravel()).cuda()  # noqa: E731
    rho, nu, V = dev(v["rho"]), dev(v["nu"]), dev(v["v"])
    rf = v["rf"]
    del v
    out = {"grid_nr_nth_nph": list(C4_GRID), "cells": N, "components": 3, "dt_over_dt_exp": VISC_RATIO,
           "rtol": RTOL}
    res = {}
    u = torch.empty_like(V)
    for prec, pname in ((R.RKL_F64, "fp64"), (R.RKL_F32MIX, "fp32_mixed")):
        with R.Context(rf, nth, nph, prec=prec) as ctx:
            dte, set_ms = _timed(torch, lambda: ctx.set_viscosity(rho, nu))
            dt = VISC_RATIO * dte

            def rk():
                u.copy_(V)
                return ctx.rkl2_superstep(u, dt, dte, ncomp=3)

            rk()
            s, ms_rk = _timed(torch, rk, 3)
            y_rk = u.clone()

            def be():
                u.copy_(V)
                return ctx.be_pcg_solve(u, dt, pc=R.RKL_PC_JACOBI, rtol=RTOL, maxit=MAXIT, ncomp=3)

            be()
            (code, its, rel), ms_be = _timed(torch, be, 3)
            res[pname] = {"rkl2": y_rk, "be": u.clone()}
            out[pname] = {"set_coeffs_ms": set_ms, "dt_exp_s": dte,
                          "rkl2": {"s": s, "ms": ms_rk, "cell_updates_per_s": 3 * N * s / ms_rk * 1e3},
                          "be_jacobi": {"iters": its, "ms": ms_be, "relres": max(rel), "converged": code == R.RKL_OK,
                                        "cell_updates_per_s": N * sum(its) / ms_be * 1e3}}
    for path in ("rkl2", "be"):
        ref = res["fp64"][path]
        chg = torch.linalg.vector_norm(ref - V).item()
        key = path if path == "rkl2" else "be_jacobi"
        out["fp32_mixed"][key]["err_rel_change_vs_fp64"] = torch.linalg.vector_norm(
            res["fp32_mixed"][path] - ref).item() / chg
    out["rkl2_vs_be_fp64_rel_change"] = (torch.linalg.vector_norm(res["fp64"]["rkl2"] - res["fp64"]["be"]).item()
                                         / torch.linalg.vector_norm(res["fp64"]["be"] - V).item())
    return out


def aggregate(ms: float, units: float, dist=None, device=None):
    """Whole-job figures of independent replicas: the slowest rank's time and the sum of
    the cell-updates of all ranks (value = units / time).  dist None = one process."""
    if dist is None:
        return ms, units
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.item(), u.item()


def nvtx(name=None):
    """Push (name) or pop (None) an NVTX range so that an ncu launch list can be limited
    to the timed region; a no-op where NVTX is unavailable."""
    try:
        import torch

        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def profile_case(args):
    """Minimal device work of one kernel family on the full grid (a few GB), for ncu."""
    import torch

    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg as R
    from paper_1610_01265_gb300 import synth

    B.build()
    nr, nth, nph = args.profile_grid
    c = synth.conduction_case(nr, nth, nph, args.seed)
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda().view(-1)  # noqa: E731
    T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
    if args.profile in ("ws-forward", "ws-train"):
        from paper_1610_01265_gb300 import warmstart as W

        net = W.Net(args.seed)
        N = nr * nth * nph
        if args.profile == "ws-forward":
            x0 = torch.empty_like(T)
            for _ in range(2):
                net.guess((nph, nth, nr), T, b, 50.0, WS_UNIT, x0)
        else:
            feat = torch.empty(5 * N, dtype=torch.float32, device="cuda")
            tgt = torch.zeros(N, dtype=torch.float32, device="cuda")
            net.features((nph, nth, nr), T, b, 50.0, feat)
            for _ in range(2):
                net.loss_grad((nr, nth, nph), feat, tgt, want_loss=False)
                net.adam(1e-3)
        net.check()
        net.close()
        print(f"profile case {args.profile} done")
        return 0
    mixed = args.profile.endswith("-mix")
    ctx = R.Context(c["rf"], nth, nph, prec=R.RKL_F32MIX if mixed else R.RKL_F64)
    if args.profile.startswith("visc-"):
        v = synth.viscosity_case(nr, nth, nph, args.seed)
        dte = ctx.set_viscosity(dev(v["rho"]), dev(v["nu"]))
        V = dev(v["v"])
        ctx.profile_enable(True)  # plain launches (see below)
        if args.profile == "visc-stage":
            ctx.rkl2_superstep(V, 10 * dte, dte, s=4, ncomp=3)
        else:
            pc = R.RKL_PC_JACOBI if args.profile == "visc-pcg-jacobi" else R.RKL_PC_BILU0
            ctx.be_pcg_solve(V, 100 * dte, pc=pc, block=BLOCK, rtol=0.0, maxit=3, ncomp=3)
        torch.cuda.synchronize()
        ctx.close()
        print(f"profile case {args.profile} done")
        return 0
    dte = ctx.set_conduction(T, b, n, beta_tcut=BETA_TCUT)
    # the library's own profiler runs the solver loops as plain launches: ncu cannot
    # profile the kernel nodes of a graph that holds a conditional (while) node
    ctx.profile_enable(True)
    u = T.clone()
    if args.profile in ("stage", "stage-mix"):
        ctx.rkl2_superstep(u, 10 * dte, dte, s=4)
    elif args.profile == "apply":
        F = torch.empty_like(T)
        for _ in range(3):
            ctx.apply_F(T, F)
    elif args.profile in ("pcg-jacobi", "pcg-jacobi-mix"):
        ctx.be_pcg_solve(u, 100 * dte, pc=R.RKL_PC_JACOBI, rtol=0.0, maxit=3)
    elif args.profile in ("pcg-bilu0", "pcg-bilu0-mix"):
        ctx.be_pcg_solve(u, 100 * dte, pc=R.RKL_PC_BILU0, block=BLOCK, rtol=0.0, maxit=3)
    elif args.profile == "setup":
        ctx.set_conduction(T, b, n, beta_tcut=BETA_TCUT)
    torch.cuda.synchronize()
    ctx.close()
    print(f"profile case {args.profile} done")
    return 0


# ------------------------------------------------------------------ ncu summaries
NCU_METRICS = (
    ("gpu__time_duration.sum", "gpu__time_duration.sum"),
    ("sm__cycles_elapsed.avg.per_second", "sm__cycles_elapsed.avg.per_second"),
    ("dram__bytes_read.sum", "dram__bytes_read.sum"),
    ("dram__bytes_write.sum", "dram__bytes_write.sum"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "gpu__dram_throughput (pct of peak, elapsed)"),
    ("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_elapsed",
     "sm__pipe_fp64_cycles_active (pct of peak, elapsed)"),
    ("sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active", "FP64 pipe instructions (pct of peak, active)"),
    ("sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_elapsed",
     "sm__pipe_tensor_cycles_active (pct of peak, elapsed)"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "sm__warps_active (pct of peak, active)"),
    ("lts__t_sector_hit_rate.pct", "L2 hit rate (pct)"),
    ("l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum", "shared-memory bank conflicts"),
    ("launch__registers_per_thread", "launch__registers_per_thread"),
    ("launch__grid_size", "launch__grid_size"),
    ("launch__block_size", "launch__block_size"),
)
BYTE_UNITS = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}


def summarize_ncu(report: str, family: str, out: str, command: str) -> int:
    """Profile summary of the first launch of FAMILY's kernel in an ncu report: the metrics
    above, the per-launch DRAM traffic and the hash of the kernel's current source (the
    bench takes roofline.traffic from it only while that hash matches), capture date."""
    import csv
    import io

    key = tuple(family.split("/"))
    pat = FAMILY_KERNEL[key]
    txt = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(io.StringIO(txt)))
    head, units = rows[0], rows[1]
    col = {h: q for q, h in enumerate(head)}
    sel = [r for r in rows[2:] if pat in r[col["Kernel Name"]]]
    if not sel:
        raise SystemExit(f"no launch of {pat} in {report}")
    r = sel[0]
    lines = []
    vals = {}
    for metric, label in NCU_METRICS:
        if metric in col:
            q = col[metric]
            lines.append(f"| {label} | {r[q]} {units[q]} |")
            vals[metric] = (r[q], units[q])
    stalls = []
    for h, q in col.items():
        if h.startswith("smsp__average_warps_issue_stalled_") and h.endswith("_per_issue_active.ratio"):
            try:
                stalls.append((float(r[q].replace(",", "")), h[len("smsp__average_warps_issue_stalled_"):-len(
                    "_per_issue_active.ratio")]))
            except ValueError:
                pass
    stalls.sort(reverse=True)
    if stalls:
        lines.append("| top stalls (cycles per issue) | " + ", ".join(f"{n} {v:.2f}" for v, n in stalls[:4]) + " |")

    def nbytes(m):
        v, u = vals[m]
        return float(v.replace(",", "")) * BYTE_UNITS.get(u, 1.0)

    traffic = nbytes("dram__bytes_read.sum") + nbytes("dram__bytes_write.sum")
    flop, alg_bytes, _, _, sources = KERNEL_COST[key]
    cells = GRID[0] * GRID[1] * GRID[2]
    with open(out, "w") as f:
        f.write(f"# {r[col['Kernel Name']].split('(')[0]} ({family}) — one launch, "
                f"{GRID[0]} x {GRID[1]} x {GRID[2]} cells\n\n")
        f.write("Command (on one GB300; the same command first exited 0 without ncu):\n\n")
        for cl in command.split(" ;; "):
            f.write(f"    {cl}\n")
        f.write(f"    python bench.py --summarize-ncu {report} {family} {out}\n\n")
        f.write(f"Kernel: `{r[col['Kernel Name']]}`\n\n| metric | value |\n|---|---|\n")
        f.write("\n".join(lines) + "\n\n")
        f.write(f"Algorithmic traffic: {alg_bytes:.0f} B/cell x {cells} cells = {alg_bytes * cells / 1e9:.4f} GB; "
                f"DRAM {traffic / 1e9:.4f} GB ({traffic / (alg_bytes * cells):.3f} of algorithmic); "
                f"{flop:.0f} flop/cell.\n\n")
        f.write(f"captured: {time.strftime('%Y-%m-%d', time.gmtime(os.path.getmtime(report)))}\n")
        f.write(f"traffic_bytes_per_launch: {traffic:.0f}\n")
        f.write(f"kernel_source_sha256_16: {kernel_source_hash(sources)}\n")
    print(out)
    return 0


# ------------------------------------------------------------------ mixed precision, 75.5 M cells
MIXED_GRID = (256, 384, 768)


def mixed_large_report(seed=1, dims=MIXED_GRID, ratios=RATIOS, log=None):
    """FP32-stage / FP32-PCG path against the FP64 path at 256 x 384 x 768: ms per large
    step, cell-updates/s and the relative L2 difference per large step, plus the live
    roofline of the FP32 stage kernel (60 B per cell: 10 FP32 coefficients, 1/W, three
    increments read, one written)."""
    import torch

    from paper_1610_01265_gb300 import rklpcg as R
    from paper_1610_01265_gb300 import synth

    nr, nth, nph = dims
    N = nr * nth * nph
    c = synth.conduction_case(nr, nth, nph, seed)
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64).ravel()).cuda()  # noqa: E731
    T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
    del c
    ctx64 = R.Context(synth.r_faces(nr), nth, nph)
    mix = R.Context(synth.r_faces(nr), nth, nph, prec=R.RKL_F32MIX)
    dte = ctx64.set_conduction(T, b, n, beta_tcut=BETA_TCUT)
    mix.set_conduction(T, b, n, beta_tcut=BETA_TCUT)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    out = {"grid_nr_nth_nph": list(dims), "cells": N, "beta_tcut": BETA_TCUT, "rtol": RTOL}
    ref = torch.empty_like(T)
    u = torch.empty_like(T)
    for ratio in ratios:
        dt = ratio * dte
        ref.copy_(T)
        s, ms64 = timed(lambda: ctx64.rkl2_superstep(ref, dt, dte))
        u.copy_(T)
        mix.rkl2_superstep(u, dt, dte)  # warm
        u.copy_(T)
        mix.profile_enable(True)
        _, msm = timed(lambda: mix.rkl2_superstep(u, dt, dte))
        prof = mix.profile()
        mix.profile_enable(False)
        chg = torch.linalg.vector_norm(ref - T).item()
        r = {"s": s, "fp64_ms": ms64, "mixed_ms": msm, "fp64_cell_updates_per_s": N * s / ms64 * 1e3,
             "mixed_cell_updates_per_s": N * s / msm * 1e3,
             "err_rel_change": torch.linalg.vector_norm(u - ref).item() / chg,
             "err_rel_u": torch.linalg.vector_norm(u - ref).item() / torch.linalg.vector_norm(ref).item()}
        st_ms, st_n = prof.get("rkl2_stage", (0.0, 0))
        if st_n:
            t = st_ms / st_n * 1e-3
            r["stage_kernel"] = {"launch_ms": t * 1e3, "hbm_gbs": 60.0 * N / t / 1e9,
                                 "hbm_frac": 60.0 * N / t / 1e9 / measured_peaks().get("hbm_gbs", 6800.0)}
        for pc, name in ((R.RKL_PC_JACOBI, "jacobi"), (R.RKL_PC_BILU0, "bilu0")):
            ref.copy_(T)
            (code64, its64, _), b64 = timed(lambda: ctx64.be_pcg_solve(ref, dt, pc=pc, block=BLOCK, rtol=RTOL,
                                                                        maxit=MAXIT))
            u.copy_(T)
            mix.profile_enable(True)
            (codem, itsm, relm), bm = timed(lambda: mix.be_pcg_solve(u, dt, pc=pc, block=BLOCK, rtol=RTOL,
                                                                     maxit=MAXIT))
            sp_ms, sp_n = mix.profile().get("spmv", (0.0, 0))
            mix.profile_enable(False)
            r[f"be_{name}"] = {"fp64_iters": its64[0], "fp64_ms": b64, "mixed_fp32_iters": itsm[0], "mixed_ms": bm,
                               "mixed_relres_fp64": relm[0], "converged": code64 == R.RKL_OK and codem == R.RKL_OK,
                               "err_rel_change": torch.linalg.vector_norm(u - ref).item()
                               / torch.linalg.vector_norm(ref - T).item()}
            if sp_n:  # FP32 y = A p: 10 coefficients + W + p + y = 52 B per cell
                t = sp_ms / sp_n * 1e-3
                r[f"be_{name}"]["fp32_spmv_kernel"] = {
                    "launch_ms": t * 1e3, "hbm_gbs": 52.0 * N / t / 1e9,
                    "hbm_frac": 52.0 * N / t / 1e9 / measured_peaks().get("hbm_gbs", 6800.0)}
        out[str(int(ratio))] = r
        if log:
            log(f"ratio {ratio}: {r}")
    ctx64.close()
    mix.close()
    return out


# ------------------------------------------------------------------ learned initial guess
WS_STEPS, WS_TRAIN, WS_RATIO, WS_UNIT = 200, 100, 1000.0, 1e4
WS_GUESSES = ("zero", "previous", "no_change", "extrapolated", "learned")
# algorithmic FLOP per cell of one forward pass (3x3x3 taps, 5-32-32-32-1 channels)
WS_FWD_FLOP = 2 * 27 * (5 * 32 + 32 * 32 + 32 * 32 + 32 * 1)


def warmstart_study(seed=1, dims=GRID, n_steps=WS_STEPS, n_train=WS_TRAIN, ratio=WS_RATIO, epochs=4, lr=1e-3,
                    pcs=(1, 2), log=None):
    """Backward-Euler conduction steps with an explicit seeded heating source, the first
    n_train from the no-change guess (their solutions train the net), the rest solved from
    each guess in WS_GUESSES to the same rtol; returns iterations, times and errors."""
    import torch

    from paper_1610_01265_gb300 import rklpcg as R
    from paper_1610_01265_gb300 import synth
    from paper_1610_01265_gb300 import warmstart as W

    nr, nth, nph = dims
    shape, N, box = (nph, nth, nr), nr * nth * nph, (nr, nth, nph)
    c = synth.conduction_case(nr, nth, nph, seed)
    hc = synth.heating_case(nr, nth, nph, seed)
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64).ravel()).cuda()  # noqa: E731
    T, b, n, h = dev(c["T"]), dev(c["bhat"]), dev(c["n"]), dev(hc["h"])
    ctx = R.Context(c["rf"], nth, nph)
    dt = ratio * ctx.set_conduction(T, b, n, beta_tcut=BETA_TCUT)
    net = W.Net(seed)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def heated(Tn, step):
        # workload input: u* = T^n + dt q(x, n), q0 dt = WS_UNIT (seeded pattern h, modulation)
        return torch.add(Tn, h, alpha=WS_UNIT * synth.heating_modulation(step, hc["psi"]))

    ustars, targets = [], []
    train_iters = []
    for step in range(n_train):
        ctx.set_conduction(T, b, n, beta_tcut=BETA_TCUT)
        us = heated(T, step)
        x = us.clone()
        code, its, _ = ctx.be_pcg_solve(x, dt, pc=R.RKL_PC_JACOBI, rtol=RTOL, maxit=MAXIT)
        if code != R.RKL_OK:
            raise RuntimeError(f"training-phase solve {step} did not converge ({code})")
        tgt = torch.empty(N, dtype=torch.float32, device="cuda")
        net.target(x, us, WS_UNIT, tgt)
        ustars.append(us)
        targets.append(tgt)
        train_iters.append(its[0])
        T = x
    dT_prev = T - ustars[-1]

    # training: full-grid samples, Adam, learning rate decaying tenfold over the run
    feat = torch.empty(5 * N, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    losses = []
    t0, t1 = ev(), ev()
    torch.cuda.synchronize()
    t0.record()
    nopt = 0
    for e in range(epochs):
        el = []
        for k in rng.permutation(n_train):
            net.features(shape, ustars[k], b, dt, feat)
            el.append(net.loss_grad(box, feat, targets[k]))
            net.adam(lr * 0.1 ** (nopt / max(1, epochs * n_train - 1)))
            nopt += 1
        losses.append(float(np.mean(el)))
        if log:
            log(f"epoch {e}: mean loss {losses[-1]:.4e}")
    t1.record()
    torch.cuda.synchronize()
    train_ms = t0.elapsed_time(t1)
    del ustars, targets

    res = {pc: {g: {"iters": [], "ms": [], "guess_ms": [], "init_err": []} for g in WS_GUESSES} for pc in pcs}
    spread = 0.0
    x0 = torch.empty_like(T)
    test_loss = []
    for step in range(n_train, n_steps):
        ctx.set_conduction(T, b, n, beta_tcut=BETA_TCUT)
        us = heated(T, step)
        sols = {}
        for pc in pcs:
            if pc == R.RKL_PC_BILU0:  # factor outside the timed solves (cached per step)
                scratch = us.clone()
                ctx.be_pcg_solve(scratch, dt, pc=pc, block=BLOCK, rtol=0.0, maxit=1)
            for g in WS_GUESSES:
                x = us.clone()
                torch.cuda.synchronize()
                e0, e1, e2 = ev(), ev(), ev()
                e0.record()
                if g == "zero":
                    x0.zero_()
                elif g == "previous":
                    x0.copy_(T)
                elif g == "no_change":
                    x0.copy_(us)
                elif g == "extrapolated":
                    torch.add(us, dT_prev, out=x0)
                else:
                    net.guess(shape, us, b, dt, WS_UNIT, x0)
                e1.record()
                code, its, _ = ctx.be_pcg_solve(x, dt, pc=pc, block=BLOCK, rtol=RTOL, maxit=MAXIT, x0=x0)
                e2.record()
                torch.cuda.synchronize()
                if code != R.RKL_OK:
                    raise RuntimeError(f"test-phase solve {step} ({g}, pc {pc}) did not converge ({code})")
                r = res[pc][g]
                r["iters"].append(its[0])
                r["ms"].append(e0.elapsed_time(e2))
                r["guess_ms"].append(e0.elapsed_time(e1))
                d = float(torch.linalg.norm(x - us))
                r["init_err"].append(float(torch.linalg.norm(x0 - x)) / d)
                sols[(pc, g)] = x
        ref = sols[(pcs[0], "learned")]
        dref = float(torch.linalg.norm(ref - us))
        for x in sols.values():
            spread = max(spread, float(torch.linalg.norm(x - ref)) / dref)
        tgt = torch.empty(N, dtype=torch.float32, device="cuda")
        net.target(ref, us, WS_UNIT, tgt)
        net.features(shape, us, b, dt, feat)
        yv = torch.empty(N, dtype=torch.float32, device="cuda")
        net.forward(box, feat, yv)
        test_loss.append(float(torch.mean((yv - tgt) ** 2)))
        dT_prev = ref - us
        T = ref
        if log and (step - n_train) % 20 == 0:
            log(f"step {step}: " + ", ".join(f"{g} {res[pcs[0]][g]['iters'][-1]}" for g in WS_GUESSES))

    # cost of the guess alone at this size: full forward pass, tensor-core rate
    fwd_ms = []
    for _ in range(5):
        e0, e1 = ev(), ev()
        e0.record()
        net.guess(shape, T, b, dt, WS_UNIT, x0)
        e1.record()
        torch.cuda.synchronize()
        fwd_ms.append(e0.elapsed_time(e1))
    net.check()  # every tensor-core convolution of the study finished
    g_ms = statistics.median(fwd_ms)
    bf16_peak = measured_peaks().get("bf16_tflops", 1900.0)
    out = {
        "study": "learned PCG initial guess",
        "grid_nr_nth_nph": list(dims),
        "steps": n_steps,
        "train_steps": n_train,
        "dt_over_dt_exp0": ratio,
        "dt_s": dt,
        "heating_K_per_step_at_h1": WS_UNIT,
        "rtol": RTOL,
        "train": {"epochs": epochs, "optimizer_steps": nopt, "ms_total": train_ms, "ms_per_step": train_ms / nopt,
                  "epoch_mean_loss": losses, "train_phase_iters_mean": float(np.mean(train_iters))},
        "test_mse_mean": float(np.mean(test_loss)),
        "solution_spread_rel": spread,
        "guess_forward": {"ms": g_ms, "tflops_algorithmic": WS_FWD_FLOP * N / (g_ms * 1e-3) / 1e12,
                          "bf16_peak_tflops": bf16_peak,
                          "frac": WS_FWD_FLOP * N / (g_ms * 1e-3) / 1e12 / bf16_peak},
        "test": {},
    }
    for pc in pcs:
        name = {1: "jacobi", 2: "bilu0-8x8x8"}[pc]
        out["test"][name] = {g: {"iters_mean": float(np.mean(r["iters"])), "ms_mean": float(np.mean(r["ms"])),
                                 "guess_ms_mean": float(np.mean(r["guess_ms"])),
                                 "init_err_mean": float(np.mean(r["init_err"]))}
                             for g, r in res[pc].items()}
    net.close()
    ctx.close()
    return out


def roofline_of(prof, N, ms_step, fp64_peak, fp64_peak_note, hbm_peak):
    """Roofline of the dominant kernel family (largest total time in the profiled step) and
    the per-kernel table."""
    per_kernel = {}
    for opn, table in prof.items():
        for kname, (tms, nl) in table.items():
            if nl:
                per_kernel[f"{opn}/{kname}"] = {"ms": tms, "launches": nl, "ms_per_launch": tms / nl}
    cands = [(v["ms"], key) for key, v in per_kernel.items() if tuple(key.split("/")) in KERNEL_COST]
    _, dom = max(cands)
    opn, kname = dom.split("/")
    flop, nbytes, bound, summary, sources = KERNEL_COST[(opn, kname)]
    t_launch = per_kernel[dom]["ms_per_launch"] * 1e-3
    achieved_tf = flop * N / t_launch / 1e12
    total = sum(v["ms"] for v in per_kernel.values())
    roof = {
        "kernel": f"{kname} ({opn}, FP64)",
        "bound": bound,
        "achieved": achieved_tf,
        "peak": fp64_peak,
        "unit": "TFLOP/s",
        "frac": achieved_tf / fp64_peak,
        "traffic": profiled_traffic(summary, sources),
        "traffic_source": f"profiles/{summary}" if summary else None,
        "launch_ms": t_launch * 1e3,
        "launches": per_kernel[dom]["launches"],
        "share_of_step": per_kernel[dom]["ms"] / ms_step,
        "share_of_kernel_time": per_kernel[dom]["ms"] / total,
        "flop_per_cell": flop,
        "bytes_per_cell": nbytes,
        "hbm_achieved_gbs": nbytes * N / t_launch / 1e9,
        "hbm_peak_gbs": hbm_peak,
        "hbm_frac": nbytes * N / t_launch / 1e9 / hbm_peak,
        "peak_note": fp64_peak_note,
    }
    for v in per_kernel.values():
        v["share"] = v["ms"] / total
    return roof, per_kernel


def main():
    args = parse_args()
    if args.summarize_ncu:
        return summarize_ncu(*args.summarize_ncu, args.summary_command)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return profile_case(args)
    if args.mixed_large:
        import torch

        from paper_1610_01265_gb300 import build as B

        B.build()
        if not torch.cuda.is_available():
            raise SystemExit("bench.py needs a CUDA GPU")
        print(json.dumps(mixed_large_report(args.seed, log=lambda m: print(m, file=sys.stderr, flush=True))),
              flush=True)
        return 0
    if args.warmstart:
        import torch

        from paper_1610_01265_gb300 import build as B

        B.build()
        if not torch.cuda.is_available():
            raise SystemExit("bench.py needs a CUDA GPU")
        out = warmstart_study(args.seed, log=lambda m: print(m, file=sys.stderr, flush=True))
        print(json.dumps(out), flush=True)
        return 0
    world, rank, local = dist_env()
    import torch

    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg as R

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    B.build()
    R.load()

    # CPU oracle baseline first (rank 0, one GPU only), before any device work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(args.seed)

    wl = Workload(R, torch, args.seed + rank)
    if args.plain_launches:
        wl.ctx_c.profile_enable(True)
        wl.ctx_v.profile_enable(True)
    for _ in range(max(args.warmup, 3)):
        wl.step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = wl.launches()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        nvtx("timed")
        t_start.record()
        units = 0
        info = None
        for _ in range(args.steps):
            u, info = wl.step()
            units += u
        t_end.record()
        torch.cuda.synchronize()
        nvtx()
    if world > 1:
        dist.barrier()
    launches = wl.launches() - launches0
    ms = t_start.elapsed_time(t_end)
    ms, units_all = aggregate(ms, float(units), dist if world > 1 else None, "cuda")
    value = units_all / (ms * 1e-3)

    # per-kernel times: one more step with the library's event profiler on (plain launches)
    wl.ctx_c.profile_enable(True)
    wl.ctx_v.profile_enable(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    units_p, _ = wl.step()
    p1.record()
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    prof = {"conduction": wl.ctx_c.profile(), "viscosity": wl.ctx_v.profile()}
    if not args.plain_launches:
        wl.ctx_c.profile_enable(False)
        wl.ctx_v.profile_enable(False)

    # FP64 roof: the device's measured FMA throughput
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    try:
        fp64_peak = R.fp64_peak()
        fp64_note = ("FP64 peak measured in this run (rkl_fp64_peak: 8 independent FMA chains per thread, 8 CTAs "
                     "of 256 threads per SM, best of 3); HBM peak = measured copy (MEASURED_PEAKS.json)")
    except R.RklError:
        fp64_peak = FP64_PEAK_TFLOPS
        fp64_note = "FP64 peak = nominal 1.25 TFLOP/s (measurement failed); HBM peak = measured copy"
    roofline, per_kernel = roofline_of(prof, wl.N, ms_prof, fp64_peak, fp64_note, hbm_peak)
    roofline["profiled_step_ms"] = ms_prof
    roofline["timed_step_ms"] = ms / args.steps
    # the fused RKL2 stage kernel, whatever its share
    st = per_kernel.get("conduction/rkl2_stage")
    stage_roof = None
    if st:
        t_st = st["ms_per_launch"] * 1e-3
        stage_roof = {"launch_ms": t_st * 1e3, "tflops": 48.0 * wl.N / t_st / 1e12,
                      "frac_fp64": 48.0 * wl.N / t_st / 1e12 / fp64_peak,
                      "hbm_frac": 128.0 * wl.N / t_st / 1e9 / hbm_peak}

    detail = {"last_step": info, "kernels": per_kernel, "rkl2_stage_kernel": stage_roof,
              "fp64_peak_tflops_measured": fp64_peak, "profiled_step_units": units_p}
    if rank == 0:
        detail["paths"] = path_timings(wl, torch)
        if not args.no_accuracy:
            detail["accuracy_vs_semidiscrete"] = accuracy_report(wl, torch)
            detail["mixed_precision"] = mixed_report(wl, R, torch)
            detail["sec6_variants"] = variants_report(wl, torch)
            detail["flux_form"] = flux_report(wl, torch)
            detail["other_seeds"] = seeds_report(wl, torch)
        if not args.no_configs:
            detail["c1_32x32x64"] = c1_report(R, torch, args.seed)
            if cpu:
                detail["c1_32x32x64"]["oracle_host_all_cores"] = cpu["c1_full_all_cores"]
                detail["c1_32x32x64"]["oracle_host_one_thread"] = cpu["single_thread"]["detail"]
            detail["c3_mixed_256x384x768"] = mixed_large_report(args.seed, ratios=(1000.0,))
            torch.cuda.empty_cache()
            detail["c4_viscosity_192x288x576"] = c4_report(R, torch, args.seed)
            torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        hw = Workload(R, torch, args.seed + rank, host=True)
        hw.step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        eu = 0
        for _ in range(args.steps):
            u, _ = hw.step()
            eu += u
        torch.cuda.synchronize()
        et = time.perf_counter() - t0
        et, eu = aggregate(et, float(eu), dist if world > 1 else None, "cuda")
        e2e = {"value": eu / et, "unit": "cell-updates/s", "h2d_bytes_per_step": hw.h2d,
               "d2h_bytes_per_step": hw.d2h}

    if rank == 0:
        line = {
            "metric": "cell-updates/s",
            "value": value,
            "unit": "cell-updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": max(args.warmup, 3),
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": base_config(),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "detail": detail,
        }
        if args.plain_launches:
            line["note"] = "--plain-launches: every step ran with the event profiler on (not a bench number)"
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

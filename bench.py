#!/usr/bin/env python
"""Throughput of MRCM-OS on one GB300: fine cells per second for the whole
method (basis build + interface solve + smoothing), mixed precision against
plain FP64, with the flux L2 error against the CPU oracle stated.

Workload: 512x512 unit square, 32x32 subdomains of 16x16 cells oversampled by
4, piecewise-linear interface spaces, channelised K (sinusoidal channels of
width 4-8 cells, contrast 1e4, log-normal background of variance 1), p = 1 / 0
on x = 0 / 1, 8 smoothing steps.  A step is one full pass:
mrcm_build_basis + mrcm_solve_interface + mrcm_smooth(8).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own copy of
the problem (replicas: the single problem's interface solve couples every
subdomain, so it is not sharded); value = cells of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "2d_512x512_channel_P1_l4_Ns8"
METRIC = "MRCM fine-cells/sec at fixed flux L2 error vs oracle; mixed vs FP64 batched"
N_SMOOTH = 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle check and CPU baseline")
    ap.add_argument("--space", type=int, default=None, choices=[0, 1],
                    help="layered3d only: interface spaces, 0 = P0 (the default workload), 1 = P1 = {1, s, t} "
                         "(up to 18 basis right-hand sides per box)")
    ap.add_argument("--grid", default=None,
                    help="layered3d only: cells per axis as nx,ny,nz (default 60,220,85; the layer split "
                         "keeps its share of the z extent)")
    ap.add_argument("--particular", default="omega", choices=["omega", "hat"],
                    help="small, layered3d, ensemble: the particular problem of Step 4 on Omega_i (the paper) "
                         "or on hat-Omega_i (the variant)")
    ap.add_argument("--workload", default="channel2d",
                    choices=["channel2d", "small", "layered3d", "ensemble", "adjoint", "variant"],
                    help="channel2d: the benchmark line; the others print a timing line for another "
                         "workload (64x64 quarter five-spot, 60x220x85 layered 3D, 256-member ensemble, "
                         "256x256 gradient, the 512x512 channel with the particular problem on Omega_i "
                         "and on hat-Omega_i)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
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
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work (counting rule: factor n b^2, solve 4 n b per right-hand side)
# ---------------------------------------------------------------------------
def _band(sides):
    """Band half-width of a box in natural order with the short axes fastest:
    the smallest side in 2D, the product of the two smallest in 3D."""
    s = sorted(sides)
    return s[0] if len(s) == 2 else s[0] * s[1]


def algorithmic_work(cases, particular="omega"):
    """Arithmetic the method needs on these problems (one factorisation per
    operator, one solve per right-hand side, 2 n^3 per slab inverse):
    flops of the basis build (basis boxes, particular problems), of one
    smoothing step, of the slab inverses, and the local right-hand sides.
    particular="hat": the particular problem is one more solve with the
    basis box's factor instead of an Omega_i factor and solve."""
    basis = smooth = slab = 0.0
    rhs = 0
    for case in cases:
        prob, part, pm = case.problem, case.partition, case.params
        d, n, sub, l = prob.dim, prob.n, part.sub, part.overlap
        M = [n[a] // sub[a] for a in range(d)]
        npsi = 1 if pm.space == 0 else (2 if d == 2 else 3)
        extra = pm.alpha_basis != pm.alpha_smooth   # a second factor of every box for the smoothing
        ni = int(np.prod(sub))
        bi = _band(sub)
        layer = {}
        for idx in np.ndindex(*M[::-1]):
            mi = idx[::-1]
            lo = [mi[a] * sub[a] for a in range(d)]
            hi = [lo[a] + sub[a] for a in range(d)]
            sides = [min(n[a], hi[a] + l) - max(0, lo[a] - l) for a in range(d)]
            nh, bh = int(np.prod(sides)), _band(sides)
            ns = sum((mi[a] > 0) + (mi[a] < M[a] - 1) for a in range(d))
            N = ns * npsi
            part_flops = 4 * nh * bh if particular == "hat" else ni * bi * bi + 4 * ni * bi
            basis += nh * bh * bh * (2 if extra else 1) + N * 4 * nh * bh + part_flops
            smooth += 4 * nh * bh
            rhs += N + 1
            layer[mi[-1]] = layer.get(mi[-1], 0) + N
        slab += sum(2.0 * float(k) ** 3 for k in layer.values())
    return {"local_basis": basis, "smooth_per_step": smooth, "interface_lu": slab, "basis_rhs": rhs}


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu measurement
    (profiles/roofline_traffic.json), or None when the kernel's source has
    changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh).get(kernel)
    if not rec:
        return None
    hsh = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as fh:
            hsh.update(fh.read())
    return rec["bytes_per_launch"] if hsh.hexdigest() == rec["sha256"] else None


SLAB_KERNEL = {"gauss-jordan-registers": "k_gjr_inverse", "gauss-jordan": "k_gj_inverse", "lu": "k_lu_inverse"}
LIMITER = {
    "local_basis": "latency: the dependent chain of line factorisations and solves of each box (one box per CTA)",
    "smooth": "latency: one box per CTA, a chain of line solves per sweep, 2^d dependent colour launches",
    "interface_lu": "latency: the pivot chain (one panel owner at a time) of the slabs of a reduction level",
}


def kernel_rooflines(work, tm, n_smooth, peaks, precision, slab_inverse, dim):
    """Per kernel group: algorithmic flops per launch / device time per launch
    against the measured FMA peak of the form's local arithmetic (FP32 for the
    mixed form, FP64 for the FP64 form; the slab inverses are FP32 in both)."""
    local_kind = "fp32" if precision == "mixed" else "fp64"
    tag = "3d" if dim == 3 else "2d"
    names = {"local_basis": f"k_local{tag}<{'float' if local_kind == 'fp32' else 'double'}>",
             "smooth": f"k_smooth{tag}<{'float' if local_kind == 'fp32' else 'double'}>",
             "interface_lu": SLAB_KERNEL.get(slab_inverse, slab_inverse)}
    total = {"local_basis": work["local_basis"], "smooth": work["smooth_per_step"] * n_smooth,
             "interface_lu": work["interface_lu"]}
    out = {}
    for ph in ("local_basis", "smooth", "interface_lu"):
        ms, nl = tm.get(ph, (0.0, 0))
        if ms <= 0 or nl <= 0:
            continue
        kind = "fp32" if ph == "interface_lu" else local_kind
        peak = peaks[kind]
        per_launch_ms = ms / nl
        wl = total[ph] / nl
        ach = wl / (per_launch_ms * 1e-3) / 1e12
        out[ph] = {"kernel": names[ph], "bound": "alu", "pipe": kind, "achieved": ach, "peak": peak,
                   "unit": "TFLOP/s", "frac": ach / peak, "ms_per_step": ms, "launches_per_step": nl,
                   "launch_ms": per_launch_ms, "work_per_launch_flop": wl,
                   "traffic": measured_traffic(names[ph]), "limiter": LIMITER[ph]}
    return out


def local_solves_per_step(case):
    """Local right-hand sides per step: N_i basis + 1 particular + N_s smoothing per subdomain."""
    w = algorithmic_work([case])
    n, sub = case.problem.n, case.partition.sub
    nsub = int(np.prod([n[a] // sub[a] for a in range(case.problem.dim)]))
    return w["basis_rhs"] + nsub * N_SMOOTH


def sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def measured_peaks(stream):
    """FP32 / FP64 FMA throughput of this GPU (the library's FMA probe) and
    the measured figures, if present."""
    from paper_2404_13811_gb300 import _lib as L
    f32, f64 = L.mrcm_measure_fma_peaks(stream.cuda_stream)
    out = {"fp32": f32, "fp64": f64, "unit": "TFLOP/s",
           "source": "mrcm_measure_fma_peaks: independent FMA chains on every SM, CUDA events, median of 3"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as fh:
                mp = json.load(fh)
            out["measured_peaks_json"] = {k: mp[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained") if k in mp}
        except Exception:
            pass
    return out


class Timer:
    """Device time of K steps after W warm-up steps, L2 flushed (512 MB write)
    before every timed step, CUDA events on the launching stream."""

    def __init__(self, stream):
        import torch
        self.stream = stream
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def __call__(self, fn, K, W, nvtx=None):
        import torch
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        ms = []
        if nvtx:
            torch.cuda.nvtx.range_push(nvtx)   # lets a profiler keep to the timed steps
        for k in range(K):
            self.flush.fill_(float(k))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        if nvtx:
            torch.cuda.nvtx.range_pop()
        return float(np.sum(ms)), ms


def phase_times(s, step_eager, reps=2):
    """Per-phase device time and kernel counts per step from eager steps (the
    kernels the captured graph replays), outside the timed region."""
    s.profile(True)
    for _ in range(reps):
        step_eager(s)
    tm = {k: (v[0] / reps, v[1] / reps) for k, v in s.timings().items()}
    s.profile(False)
    return tm


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, rank, world):
    import torch
    from paper_2404_13811_gb300 import _lib as L
    from paper_2404_13811_gb300 import build as B
    from paper_2404_13811_gb300 import inputs as I
    from paper_2404_13811_gb300.solver import MRCM

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    # the slab-inverse choice is measured once per shape class and tolerance
    # and then read from the cache, as a long-running user would have it (a
    # cache named by MRCM_TUNE_CACHE is used as it is)
    if not os.environ.get("MRCM_TUNE_CACHE"):
        fd, cache = tempfile.mkstemp(suffix=".json")
        os.close(fd)
        os.unlink(cache)
        os.environ["MRCM_TUNE_CACHE"] = cache
    case = I.config_channel2d()
    prob, part, pm = case.problem, case.partition, case.params
    ncell = prob.ncells
    stream = torch.cuda.current_stream()
    timer = Timer(stream)
    peaks = measured_peaks(stream)

    def make(precision, tol=1e-12):
        return MRCM(prob, part, space=pm.space, alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth,
                    precision=precision, ir_tol=tol, max_ir=30, stream=stream, device_inputs=True)

    def step(s):
        # the whole step (basis, interface, smoothing) as one captured CUDA
        # graph (mrcm_run); the first call runs eagerly and captures
        s.run(N_SMOOTH, graph=True)

    def step_eager(s):
        s.build_basis()
        s.solve_interface()
        s.smooth(N_SMOOTH)

    ref = None
    cpu = None
    use_oracle = rank == 0 and not args.no_oracle
    if use_oracle:
        from oracle import mrcm_oracle as O
        t0 = time.perf_counter()
        ref = O.mrcm_os(prob, part.sub, part.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth, N_SMOOTH)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": ncell / t_cpu, "unit": "cells/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one full pass of the oracle on the whole {WORKLOAD} workload "
                         f"({t_cpu:.1f} s; numpy/scipy, LAPACK threads = host cores)"}

    def errors(s):
        if ref is None:
            return None
        p, u = s.fluxes()
        ep, eu = O.rel_errors(prob, p, u, ref.p, ref.u)
        return {"flux_rel_l2": eu, "pressure_rel_l2": ep}

    solvers = {"mixed": make("mixed"), "fp64": make("fp64")}
    errs = {}
    for name, s in solvers.items():
        step(s)
        errs[name] = errors(s)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(dev)
    clk.start()
    ms_mixed, _ = timer(lambda: step(solvers["mixed"]), args.steps, args.warmup, nvtx="mrcm_timed_steps")
    k64 = max(3, args.steps // 4)
    ms_fp64, _ = timer(lambda: step(solvers["fp64"]), k64, 1)

    # the fixed-error comparison: both forms over a range of ir_tol (the
    # interface refinement of both and the local refinement of the mixed
    # form stop there); at the tightest flux error both reach, and at 1e-10,
    # each form at its fastest setting that meets the target
    sweep = {"mixed": [], "fp64": []}
    tols = {"mixed": (1e-10, 1e-11, 1e-12, 1e-13), "fp64": (1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-13)}
    ks = max(3, args.steps // 4)
    for form in (("mixed", "fp64") if use_oracle else ()):   # the sweep is there for its errors
        for tol in tols[form]:
            rec = {"ir_tol": tol}
            s = None
            try:
                s = make(form, tol)
                step(s)
                rec.update(errors(s) or {})
                t, _ = timer(lambda: step(s), ks, 1)
                rec["ms_per_step"] = t / ks
            except L.MrcmError as exc:
                rec["error"] = str(exc)
            if s is not None:
                s.close()
            sweep[form].append(rec)
    clocks = clk.stop()
    clocks["window"] = "sampled over the timed steps of both forms (and of the ir_tol sweep with the oracle)"

    fixed = None
    if use_oracle:
        ok = {f: [r for r in sweep[f] if "ms_per_step" in r and "flux_rel_l2" in r] for f in sweep}
        if ok["mixed"] and ok["fp64"]:
            tight = max(min(r["flux_rel_l2"] for r in ok[f]) for f in ok)
            fixed = []
            for target in sorted({tight, 1e-10}):
                entry = {"target_flux_rel_l2": target}
                for f in ok:
                    meet = [r for r in ok[f] if r["flux_rel_l2"] <= target * (1 + 1e-9)]
                    if meet:
                        b = min(meet, key=lambda r: r["ms_per_step"])
                        entry[f] = dict(b, value=ncell / (b["ms_per_step"] * 1e-3), unit="cells/s")
                if "mixed" in entry and "fp64" in entry:
                    entry["speedup_mixed_over_fp64"] = entry["fp64"]["ms_per_step"] / entry["mixed"]["ms_per_step"]
                fixed.append(entry)

    torch.cuda.synchronize()
    ms_mixed = max_over_ranks(ms_mixed, world, "cuda")
    ms_step = ms_mixed / args.steps
    value = ncell * world / (ms_step * 1e-3)
    fp64_ms = ms_fp64 / k64

    # per-kernel rooflines (phase device times from eager steps of the same
    # kernels), and the dominant kernel of the mixed form as the headline
    tm = phase_times(solvers["mixed"], step_eager)
    tm64 = phase_times(solvers["fp64"], step_eager)
    st = solvers["mixed"].stats()
    st64 = solvers["fp64"].stats()
    work = algorithmic_work([case])
    kr = kernel_rooflines(work, tm, N_SMOOTH, peaks, "mixed", st["slab_inverse"], 2)
    kr64 = kernel_rooflines(work, tm64, N_SMOOTH, peaks, "fp64", st64["slab_inverse"], 2)
    dom = max(kr, key=lambda k: kr[k]["ms_per_step"])
    roof = {k: kr[dom][k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel", "pipe",
                                    "launch_ms", "work_per_launch_flop", "limiter")}
    roof["peak_basis"] = "of measured: FMA probe (mrcm_measure_fma_peaks) on this GPU"
    roof["work_rule"] = "factor n b^2 and 4 n b per right-hand side (local kernels); 2 n^3 per slab inverse"

    # end to end through the C ABI, host buffers: every step a new K from
    # pinned host memory (mrcm_set_permeability copies it), the whole method
    # (mrcm_run, eager: a new operator), and p, u read back to pinned memory
    Kh = torch.from_numpy(np.ascontiguousarray(prob.K).reshape(-1)).pin_memory()
    pout = torch.empty(ncell, dtype=torch.float64).pin_memory()
    uout = torch.empty((ncell, 4), dtype=torch.float64).pin_memory()
    s_e = make("mixed")
    e2e_ms = 0.0
    ke = max(3, args.steps // 4)
    for k in range(ke + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.mrcm_set_permeability(s_e.h, Kh.numpy(), 0)
        L.mrcm_run(s_e.h, N_SMOOTH, 0)
        L.mrcm_fluxes(s_e.h, 0, uout.numpy(), pout.numpy())
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_ms += dt * 1e3
    s_e.close()
    e2e = {"value": ncell / (e2e_ms / ke * 1e-3), "unit": "cells/s",
           "h2d_bytes_per_step": int(ncell * 8), "d2h_bytes_per_step": int(5 * ncell * 8),
           "includes": "mrcm_set_permeability (H2D of K, face coefficients) + mrcm_run eager (basis, interface "
                       "with the cached slab-inverse choice, 8 smoothing steps) + mrcm_fluxes (D2H of p, u)"}

    gpu_launches = int(round(sum(v[1] for k, v in tm.items() if k not in ("graph", "interface_lu"))))
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [512, 512], "subdomains": [32, 32], "sub": [16, 16],
                   "overlap": 4, "space": "P1", "n_smooth": N_SMOOTH, "alpha": 1.0,
                   "contrast": 1e4, "precision": "mixed (FP32 local factor/solves, FP64 residuals), ir_tol 1e-12",
                   "l2": "flushed (512 MB write) between timed steps", "parallelism": f"replicas{world}",
                   "step": "mrcm_run: the whole step replayed as one captured CUDA graph"},
        "fp64_form": {"value": ncell / (fp64_ms * 1e-3), "unit": "cells/s", "ms_per_step": fp64_ms,
                      "form": "FP64 local factorisations and solves; the interface solve is the same in both "
                              "forms (FP32 block-cyclic-reduction factors, FP64 residuals and refinement)"},
        "fixed_error_comparison": fixed, "ir_tol_sweep": sweep,
        "errors_vs_oracle": errs, "phase_ms_per_step": {k: v[0] for k, v in tm.items()},
        "launches_per_step": {k: v[1] for k, v in tm.items()},
        "fp64_phase_ms_per_step": {k: v[0] for k, v in tm64.items()},
        "roofline": roof, "kernel_rooflines": {"mixed": kr, "fp64": kr64}, "peaks": peaks,
        "stats": {"mixed": st, "fp64": st64},
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": gpu_launches,
        "subdomain_solves_per_s": local_solves_per_step(case) * world / (ms_step * 1e-3),
    }
    for s in solvers.values():
        s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# lines of the other workloads (not the benchmark line)
# ---------------------------------------------------------------------------
def run_other(args):
    import torch
    from paper_2404_13811_gb300 import build as B
    from paper_2404_13811_gb300 import inputs as I
    from paper_2404_13811_gb300.solver import MRCM

    B.build()
    if not os.environ.get("MRCM_TUNE_CACHE"):
        fd, cache = tempfile.mkstemp(suffix=".json")
        os.close(fd)
        os.unlink(cache)
        os.environ["MRCM_TUNE_CACHE"] = cache
    stream = torch.cuda.current_stream()
    timer = Timer(stream)
    peaks = measured_peaks(stream)
    dev = torch.cuda.current_device()

    w = args.workload
    line = {"workload": w, "unit": "cells/s", "steps": args.steps, "warmup": args.warmup,
            "l2": "flushed (512 MB write) between timed steps", "data": "synthetic", "peaks": peaks}
    if w in ("small", "layered3d", "ensemble"):
        if w == "layered3d" and (args.grid or args.space is not None):
            n3 = tuple(int(v) for v in args.grid.split(",")) if args.grid else (60, 220, 85)
            cases = [I.config_layered3d(n=n3, n_upper=max(1, round(35 * n3[2] / 85)),
                                        space=args.space if args.space is not None else 0)]
            line["grid"] = list(n3)
            line["space"] = "P1" if cases[0].params.space == 1 else "P0"
        else:
            cases = I.config_ensemble() if w == "ensemble" else [I.config_small() if w == "small" else I.config_layered3d()]
        probs = [c.problem for c in cases]
        parts = [c.partition for c in cases]
        pm = cases[0].params
        cells = sum(p.ncells for p in probs)
        dim = probs[0].dim
        line.update({"members": len(cases), "cells": cells, "n_smooth": pm.n_smooth, "particular": args.particular,
                     "step": "mrcm_run: the whole step replayed as one captured CUDA graph"})
        # oracle check: every member of the small and 3D workloads; a seeded
        # subset of 4 members of the ensemble
        check = list(range(len(cases)))
        if w == "ensemble":
            check = sorted(np.random.default_rng(4040).choice(len(cases), 4, replace=False).tolist())
        refs = {}
        if not args.no_oracle:
            from oracle import mrcm_oracle as O
            t0 = time.perf_counter()
            for m in check:
                c = cases[m]
                refs[m] = O.mrcm_os(c.problem, c.partition.sub, c.partition.overlap, c.params.space,
                                    c.params.alpha_basis, c.params.alpha_smooth, c.params.n_smooth,
                                    particular=args.particular)
            line["oracle"] = {"members_checked": check, "seconds": time.perf_counter() - t0,
                              "subset": "seeded subset of 4 members" if w == "ensemble" else "all members"}
        work = algorithmic_work(cases, particular=args.particular)
        clk = Clocks(dev)
        clk.start()
        for precision in ("mixed", "fp64"):
            s = MRCM(probs if len(probs) > 1 else probs[0], parts if len(parts) > 1 else parts[0], space=pm.space,
                     alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth, precision=precision, stream=stream,
                     particular=args.particular)
            s.run(pm.n_smooth, graph=True)
            tot, _ = timer(lambda: s.run(pm.n_smooth, graph=True), args.steps, args.warmup)
            ms = tot / args.steps
            errs = {}
            if refs:
                worst = [0.0, 0.0]
                for m in check:
                    p, u = s.fluxes(member=m)
                    ep, eu = O.rel_errors(cases[m].problem, p, u, refs[m].p, refs[m].u)
                    worst = [max(worst[0], eu), max(worst[1], ep)]
                errs = {"flux_rel_l2_max": worst[0], "pressure_rel_l2_max": worst[1]}

            def eager(sv):
                sv.build_basis()
                sv.solve_interface()
                sv.smooth(pm.n_smooth)

            tm = phase_times(s, eager, reps=1)
            st = s.stats()
            kr = kernel_rooflines(work, tm, pm.n_smooth, peaks, precision, st["slab_inverse"], dim)
            dom = max(kr, key=lambda k: kr[k]["ms_per_step"])
            line[precision] = {"ms_per_step": ms, "value": cells / (ms * 1e-3), "errors_vs_oracle": errs,
                               "phase_ms_eager": {k: round(v[0], 3) for k, v in tm.items() if v[0] > 0},
                               "roofline": kr[dom], "kernel_rooflines": kr, "stats": st}
            s.close()
        line["clocks"] = clk.stop()
    elif w == "variant":
        # Step 4 as in the paper (particular problem on Omega_i) and the
        # variant on hat-Omega_i, on the 512x512 channel workload, mixed form:
        # time, the oracle of each form, and both against the fine solution
        case = I.config_channel2d()
        prob, part, pm = case.problem, case.partition, case.params
        line.update({"cells": prob.ncells, "n_smooth": pm.n_smooth, "grid": list(prob.n), "sub": list(part.sub),
                     "overlap": part.overlap, "space": "P1" if pm.space == 1 else "P0", "precision": "mixed",
                     "step": "mrcm_run: the whole step replayed as one captured CUDA graph"})
        refs, fine = {}, None
        if not args.no_oracle:
            from oracle import mrcm_oracle as O
            t0 = time.perf_counter()
            fine = O.fine_solve(prob)
            for v in ("omega", "hat"):
                refs[v] = O.mrcm_os(prob, part.sub, part.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth,
                                    pm.n_smooth, keep_stages=True, particular=v)
            line["oracle"] = {"seconds": time.perf_counter() - t0,
                              "what": "the fine solution and MRCM-OS with each particular form"}
        clk = Clocks(dev)
        clk.start()
        for v in ("omega", "hat"):
            s = MRCM(prob, part, space=pm.space, alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth,
                     precision="mixed", stream=stream, particular=v)
            rec = {}
            if refs:
                s.run(0)
                p, u = s.fluxes()
                rp, ru = refs[v].stages["mrcm_o"]
                ep, eu = O.rel_errors(prob, p, u, rp, ru)
                fp, fu = O.rel_errors(prob, p, u, *fine)
                rec["mrcm_o"] = {"vs_oracle": {"flux_rel_l2": eu, "pressure_rel_l2": ep},
                                 "vs_fine": {"flux_rel_l2": fu, "pressure_rel_l2": fp}}
            s.run(pm.n_smooth, graph=True)
            tot, _ = timer(lambda: s.run(pm.n_smooth, graph=True), args.steps, args.warmup)
            ms = tot / args.steps
            if refs:
                p, u = s.fluxes()
                ep, eu = O.rel_errors(prob, p, u, refs[v].p, refs[v].u)
                fp, fu = O.rel_errors(prob, p, u, *fine)
                rec[f"smooth{pm.n_smooth}"] = {"vs_oracle": {"flux_rel_l2": eu, "pressure_rel_l2": ep},
                                               "vs_fine": {"flux_rel_l2": fu, "pressure_rel_l2": fp}}

            def eager(sv):
                sv.build_basis()
                sv.solve_interface()
                sv.smooth(pm.n_smooth)

            tm = phase_times(s, eager, reps=1)
            st = s.stats()
            kr = kernel_rooflines(algorithmic_work([case], particular=v), tm, pm.n_smooth, peaks, "mixed",
                                  st["slab_inverse"], 2)
            rec.update({"ms_per_step": ms, "value": prob.ncells / (ms * 1e-3),
                        "phase_ms_eager": {k: round(x[0], 3) for k, x in tm.items() if x[0] > 0},
                        "launches_eager": {k: x[1] for k, x in tm.items() if x[1] > 0},
                        "roofline_local_basis": kr.get("local_basis"), "stats": st})
            line[v] = rec
            s.close()
        line["clocks"] = clk.stop()
    else:
        case = I.config_adjoint()
        prob, part, pm = case.problem, case.partition, case.params
        sinks = np.array([ix + prob.n[0] * iy for (ix, iy) in case.extra["sinks"]])
        # the loss target: the forward solution for the second K (an input of the timing)
        t = MRCM(case.extra["target_problem"], part, space=pm.space, precision="fp64", stream=stream)
        t.run(pm.n_smooth)
        ut = t.state()[1][torch.as_tensor(sinks, device="cuda")]
        t.close()
        line.update({"cells": prob.ncells, "n_smooth": pm.n_smooth,
                     "loss": "sum over the 4 faces of 8 sink cells of (u - u_target)^2"})
        gref = None
        if not args.no_oracle:
            from oracle import mrcm_adjoint as OA
            from oracle import mrcm_oracle as O
            t0 = time.perf_counter()
            ref = O.mrcm_os(prob, part.sub, part.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth, pm.n_smooth)
            gu = np.zeros_like(ref.u)
            gu[sinks] = 2.0 * (ref.u[sinks] - ut.cpu().numpy())
            _, gref = OA.mrcm_os_adjoint(prob, part.sub, part.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth,
                                         pm.n_smooth, np.zeros(prob.ncells), gu)
            line["oracle"] = {"seconds": time.perf_counter() - t0, "what": "forward pass and adjoint gradient"}
        clk = Clocks(dev)
        clk.start()
        for precision in ("mixed", "fp64"):
            s = MRCM(prob, part, space=pm.space, alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth,
                     precision=precision, stream=stream)
            rows = torch.as_tensor(sinks, device="cuda")

            def fwd():
                s.run(pm.n_smooth)

            def grad():
                u = s.state()[1]
                gu = torch.zeros_like(u)
                gu[rows] = 2.0 * (u[rows] - ut)
                return s.adjoint(None, gu)

            fwd()
            ms_f, _ = timer(fwd, args.steps, args.warmup)
            ms_g, _ = timer(grad, args.steps, args.warmup)
            ms_f /= args.steps
            ms_g /= args.steps
            rec = {"forward_ms": ms_f, "adjoint_ms": ms_g, "adjoint_over_forward": ms_g / ms_f,
                   "value": prob.ncells / ((ms_f + ms_g) * 1e-3)}
            if gref is not None:
                fwd()
                g = grad().cpu().numpy()
                rec["gradient_rel_l2_vs_oracle"] = float(np.linalg.norm(g - gref) / np.linalg.norm(gref))
            line[precision] = rec
            s.close()
        line["clocks"] = clk.stop()
    print(json.dumps(line), flush=True)


def max_over_ranks(x, world, device):
    """The largest of the ranks' values: a replicated job takes as long as its
    slowest rank.  device: "cuda" under NCCL, "cpu" under gloo."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import mrcm_oracle as O
    from paper_2404_13811_gb300 import inputs as I
    case = I.config_channel2d(n=128)
    prob, part, pm = case.problem, case.partition, case.params
    for _ in range(min(args.warmup, 1)):
        O.mrcm_os(prob, part.sub, part.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth, N_SMOOTH)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.mrcm_os(prob, part.sub, part.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth, N_SMOOTH)
    dt = time.perf_counter() - t0
    value = prob.ncells * args.steps / dt
    sample = ("each step: the oracle's full pipeline on a 128x128 sample of the same recipe "
              "(8x8 subdomains of 16x16, overlap 4, P1, contrast 1e4, 8 smoothing steps)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "host cores"},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "sample": sample, "value": value,
                             "unit": "cells/s"},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "gpu" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload != "channel2d":
        run_other(args)
    else:
        run_gpu(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

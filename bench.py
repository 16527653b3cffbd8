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
    ap.add_argument("--workload", default="channel2d",
                    choices=["channel2d", "small", "layered3d", "ensemble", "adjoint"],
                    help="channel2d: the benchmark line; the others print a timing line for another "
                         "workload (64x64 quarter five-spot, 60x220x85 layered 3D, 256-member ensemble, "
                         "256x256 gradient)")
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
def algorithmic_flops(case):
    """Per phase: FP32/FP64 arithmetic the method needs on this workload (one
    factorisation per operator, one solve per right-hand side)."""
    prob, part = case.problem, case.partition
    n, sub, l = prob.n, part.sub, part.overlap
    M = [n[a] // sub[a] for a in range(2)]
    npsi = 2 if case.params.space == 1 else 1
    basis = 0.0
    smooth = 0.0
    for iy in range(M[1]):
        for ix in range(M[0]):
            lo = [ix * sub[0], iy * sub[1]]
            hi = [lo[0] + sub[0], lo[1] + sub[1]]
            loh = [max(0, lo[a] - l) for a in range(2)]
            hih = [min(n[a], hi[a] + l) for a in range(2)]
            bx, by = hih[0] - loh[0], hih[1] - loh[1]
            nh = bx * by
            nsides = (ix > 0) + (ix < M[0] - 1) + (iy > 0) + (iy < M[1] - 1)
            N = nsides * npsi
            ni = sub[0] * sub[1]
            basis += nh * bx * bx + N * 4 * nh * bx + ni * sub[0] ** 2 + 4 * ni * sub[0]
            smooth += 4 * nh * bx
    # interface: every slab (one layer of subdomains along the last axis) is
    # inverted once per factorisation, 2 n^3 flops for n unknowns
    lu = 0.0
    for iy in range(M[1]):
        ns = sum(((ix > 0) + (ix < M[0] - 1) + (iy > 0) + (iy < M[1] - 1)) * npsi for ix in range(M[0]))
        lu += 2.0 * ns ** 3
    return {"local_basis": basis, "smooth_per_step": smooth, "interface_lu": lu}


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


def local_solves_per_step(case):
    """Local right-hand sides per step: N_i basis + 1 particular + N_s smoothing per subdomain."""
    n, sub = case.problem.n, case.partition.sub
    M = [n[a] // sub[a] for a in range(2)]
    npsi = 2 if case.params.space == 1 else 1
    tot = 0
    for iy in range(M[1]):
        for ix in range(M[0]):
            nsides = (ix > 0) + (ix < M[0] - 1) + (iy > 0) + (iy < M[1] - 1)
            tot += nsides * npsi + 1 + N_SMOOTH
    return tot


def sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, rank, world):
    import torch
    from paper_2404_13811_gb300 import build as B
    from paper_2404_13811_gb300 import inputs as I
    from paper_2404_13811_gb300.solver import MRCM

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    case = I.config_channel2d()
    prob, part, pm = case.problem, case.partition, case.params
    ncell = prob.ncells
    stream = torch.cuda.current_stream()

    def make(precision, device_inputs=True, tol=1e-12):
        return MRCM(prob, part, space=pm.space, alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth,
                    precision=precision, ir_tol=tol, max_ir=30, stream=stream, device_inputs=device_inputs)

    def step(s):
        # the whole step (basis, interface, smoothing) as one captured CUDA
        # graph (mrcm_run); the first call runs eagerly and captures
        s.run(N_SMOOTH, graph=True)

    def step_eager(s):
        s.build_basis()
        s.solve_interface()
        s.smooth(N_SMOOTH)

    # correctness against the oracle (and the CPU baseline timing) on rank 0
    cpu = None
    errs = {}
    solvers = {"mixed": make("mixed"), "fp64": make("fp64")}
    if rank == 0 and not args.no_oracle:
        from oracle import mrcm_oracle as O
        t0 = time.perf_counter()
        ref = O.mrcm_os(prob, part.sub, part.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth, N_SMOOTH)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": ncell / t_cpu, "unit": "cells/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one full pass of the oracle on the whole {WORKLOAD} workload "
                         f"({t_cpu:.1f} s; numpy/scipy, LAPACK threads = host cores)"}
        for name, s in solvers.items():
            step(s)
            p, u = s.fluxes()
            ep, eu = O.rel_errors(prob, p, u, ref.p, ref.u)
            errs[name] = {"flux_rel_l2": eu, "pressure_rel_l2": ep}
    # the equal-error comparison: the mixed form with the refinement tolerance
    # tightened towards the FP64 form's flux error (the first tolerance whose
    # local and interface refinements converge)
    from paper_2404_13811_gb300 import _lib as L
    eq = {"note": "mixed form with ir_tol tightened towards the FP64 form's flux error"}
    for tol in (1e-14, 1e-13):
        s_eq = None
        try:
            s_eq = make("mixed", tol=tol)
            step(s_eq)
            eq["ir_tol"] = tol
            if rank == 0 and not args.no_oracle:
                p, u = s_eq.fluxes()
                ep, eu = O.rel_errors(prob, p, u, ref.p, ref.u)
                eq["flux_rel_l2"], eq["pressure_rel_l2"] = eu, ep
            solvers["mixed_eq"] = s_eq
            break
        except L.MrcmError as exc:
            eq["unconverged_at_" + f"{tol:.0e}"] = str(exc)
            if s_eq is not None:
                s_eq.close()

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 512 MB > L2

    def timed(s, K, W, profile=False):
        for _ in range(W):
            step(s)
        torch.cuda.synchronize()
        if profile:
            s.profile(True)
        tot = 0.0
        for k in range(K):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(s)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        tm = None
        if profile:
            # per-phase device time and kernel counts from eager steps (the
            # same kernels the graph replays), outside the timed region
            s.profile(True)
            for _ in range(2):
                step_eager(s)
            tm = {k: (v[0] / 2, v[1] / 2) for k, v in s.timings().items()}
            s.profile(False)
        return tot, tm

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(dev)
    clk.start()
    ms_mixed, tm = timed(solvers["mixed"], args.steps, args.warmup, profile=True)
    clocks = clk.stop()
    ms_fp64, _ = timed(solvers["fp64"], max(2, args.steps // 4), 1)
    if "mixed_eq" in solvers:
        ms_eq, _ = timed(solvers["mixed_eq"], max(2, args.steps // 4), 1)
        eq["ms_per_step"] = ms_eq / max(2, args.steps // 4)
        eq["value"] = ncell / (eq["ms_per_step"] * 1e-3)
        eq["unit"] = "cells/s"
    torch.cuda.synchronize()
    ms_mixed = max_over_ranks(ms_mixed, world, "cuda")
    ms_step = ms_mixed / args.steps
    value = ncell * world / (ms_step * 1e-3)
    fp64_value = ncell / (ms_fp64 / max(2, args.steps // 4) * 1e-3)

    # end to end through the C ABI from pinned host memory, result read back
    Kh = torch.from_numpy(np.ascontiguousarray(prob.K)).pin_memory()
    fh = torch.from_numpy(np.ascontiguousarray(prob.f)).pin_memory()
    pout = torch.empty(ncell, dtype=torch.float64).pin_memory()
    uout = torch.empty((ncell, 4), dtype=torch.float64).pin_memory()
    from paper_2404_13811_gb300 import _lib as L
    g, b, pt = L.make_structs(2, prob.n, prob.h, prob.bc_kind, prob.bc_value, part.sub, part.overlap)
    prm = L.make_params(pm.space, pm.alpha_basis, pm.alpha_smooth, L.MRCM_MIXED, 1e-12, 8)
    ke = max(2, args.steps // 4)
    e2e_ms = 0.0
    for k in range(ke + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = L.mrcm_create(g, Kh.data_ptr(), fh.data_ptr(), b, pt, prm, 0, stream.cuda_stream)
        L.mrcm_build_basis(h)
        L.mrcm_solve_interface(h)
        L.mrcm_smooth(h, N_SMOOTH)
        L.mrcm_fluxes(h, 0, uout.numpy(), pout.numpy())
        dt = time.perf_counter() - t0
        L.mrcm_destroy(h)
        if k > 0:
            e2e_ms += dt * 1e3
    e2e = {"value": ncell / (e2e_ms / ke * 1e-3), "unit": "cells/s",
           "h2d_bytes_per_step": int(2 * ncell * 8), "d2h_bytes_per_step": int(5 * ncell * 8),
           "includes": "create (plan, allocation, H2D of K and f) + build + interface + 8 smoothing steps + D2H of p, u"}

    # roofline of the dominant kernel: the one with the most device time per
    # step among the local basis kernels, the smoothing kernel and the slab LU
    flops = algorithmic_flops(case)
    nsm = sm_count()
    mhz = clocks.get("sm_mhz") or 1485.0
    peak32 = nsm * 128 * 2 * mhz * 1e6 / 1e12
    phase_ms = {k: v[0] for k, v in tm.items()}
    launches = {k: v[1] for k, v in tm.items()}
    dom = max(("local_basis", "smooth", "interface_lu"), key=lambda k: phase_ms[k])
    total = {"local_basis": flops["local_basis"], "smooth": flops["smooth_per_step"] * N_SMOOTH,
             "interface_lu": flops["interface_lu"]}[dom]
    kname = {"local_basis": "k_local2d<float>", "smooth": "k_smooth2d<float>", "interface_lu": "k_lu_inverse"}[dom]
    work = total / max(launches[dom], 1)
    per_launch_ms = phase_ms[dom] / max(launches[dom], 1)
    achieved = work / (per_launch_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": kname,
            "achieved": achieved, "peak": peak32, "unit": "TFLOP/s", "frac": achieved / peak32,
            "traffic": measured_traffic(kname),
            "peak_basis": f"{nsm} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (median sampled SM clock; "
                          "MEASURED_PEAKS.json holds no FP32 SIMT figure)",
            "work_per_launch_flop": work, "launch_ms": per_launch_ms,
            "work_rule": "factor n b^2 and 4 n b per solve (local kernels); 2 n^3 per slab inverse"}
    # kernels of one step (the captured graph replays the eager sequence; the
    # slab-LU phase is a part of interface_factor)
    gpu_launches = int(round(sum(v[1] for k, v in tm.items() if k not in ("graph", "interface_lu"))))
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [512, 512], "subdomains": [32, 32], "sub": [16, 16],
                   "overlap": 4, "space": "P1", "n_smooth": N_SMOOTH, "alpha": 1.0,
                   "contrast": 1e4, "precision": "mixed (FP32 local factor/solves, FP64 residuals)",
                   "l2": "flushed (512 MB write) between timed steps", "parallelism": f"replicas{world}",
                   "step": "mrcm_run: the whole step replayed as one captured CUDA graph"},
        "fp64_form": {"value": fp64_value, "unit": "cells/s", "ms_per_step": 1e3 * ncell / fp64_value},
        "mixed_equal_error": eq,
        "errors_vs_oracle": errs, "phase_ms_per_step": phase_ms, "launches_per_step": launches,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": gpu_launches,
        "subdomain_solves_per_s": local_solves_per_step(case) * world / (ms_step * 1e-3),
    }
    for s in solvers.values():
        s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# timing lines of the other workloads (not the benchmark line)
# ---------------------------------------------------------------------------
def run_other(args):
    import torch
    from paper_2404_13811_gb300 import build as B
    from paper_2404_13811_gb300 import inputs as I
    from paper_2404_13811_gb300.solver import MRCM

    B.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 512 MB > L2

    def timeit(fn, K, W):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for k in range(K):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / K

    def phases(s, ns):
        s.profile(True)
        s.build_basis()
        s.solve_interface()
        s.smooth(ns)
        tm = s.timings()
        s.profile(False)
        return {k: round(v[0], 3) for k, v in tm.items() if v[0] > 0}

    w = args.workload
    line = {"workload": w, "unit": "cells/s", "steps": args.steps, "warmup": args.warmup,
            "l2": "flushed (512 MB write) between timed steps", "data": "synthetic"}
    if w in ("small", "layered3d", "ensemble"):
        cases = I.config_ensemble() if w == "ensemble" else [I.config_small() if w == "small" else I.config_layered3d()]
        probs = [c.problem for c in cases]
        parts = [c.partition for c in cases]
        pm = cases[0].params
        cells = sum(p.ncells for p in probs)
        line.update({"members": len(cases), "cells": cells, "n_smooth": pm.n_smooth,
                     "step": "mrcm_run: the whole step replayed as one captured CUDA graph"})
        for precision in ("mixed", "fp64"):
            s = MRCM(probs if len(probs) > 1 else probs[0], parts if len(parts) > 1 else parts[0], space=pm.space,
                     alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth, precision=precision, stream=stream)
            ms = timeit(lambda: s.run(pm.n_smooth, graph=True), args.steps, args.warmup)
            line[precision] = {"ms_per_step": ms, "value": cells / (ms * 1e-3), "phase_ms_eager": phases(s, pm.n_smooth),
                               "subdomains": s.stats()["subdomains"]}
            s.close()
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
            ms_f = timeit(fwd, args.steps, args.warmup)
            ms_g = timeit(grad, args.steps, args.warmup)
            line[precision] = {"forward_ms": ms_f, "adjoint_ms": ms_g, "adjoint_over_forward": ms_g / ms_f,
                               "value": prob.ncells / ((ms_f + ms_g) * 1e-3)}
            s.close()
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

#!/usr/bin/env python3
"""sn-K K-build throughput on GB300.

One step = one full K build of the 96-atom workload (992 Cartesian functions up
to d, 768,000 grid points, 200 occupied orbitals, FP64): snk_set_density (P
upload, symmetry check, F-tilde and sn-LinK pair screen, task lists) followed
by snk_build_K (collocation, F = X P, 3c-CP integrals contracted into G,
K-tilde = G^T X, symmetrisation).  Inputs are resident in HBM when the timed
region starts (`value`); `e2e` repeats the measurement through the C ABI with
host buffers, the P upload and the K download inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (the build does not shard);
the value is the total builds of all ranks over the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of grid points of the same workload and extrapolates to builds/s.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sn-K K-builds/s at stated max|ΔK|: chosen form vs plain FP64, same GB300"
WORKLOAD = "cluster96"
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 (2 DFMA/clk/SM x 152 SMs x ~2.06 GHz)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(p, name=WORKLOAD):
    n_heavy = int((p.mol.Z == 8).sum())
    return {"workload": f"{name}: {p.mol.Z.shape[0]} atoms ({n_heavy} O-like, {p.mol.Z.shape[0] - n_heavy} H-like), "
                        f"{p.basis.n_functions} Cartesian functions up to d, {p.grid.n_points} grid points "
                        f"(50 MK radial x 8 GL theta x 20 phi per atom, Becke), {p.meta['n_occ']} occupied orbitals",
            "precision": "fp64", "screen": "sn-LinK eps_E = eps_K = eps_B = 1e-12", "batch_max": 4096,
            "l2": "no flush: each step rewrites a >10 GB workspace (X, F, G), far above the 126 MB L2"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
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
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


GOLDEN = os.path.join(ROOT, "tests", "golden", "cluster96_K_entries.txt")


def sampled_parity(K):
    """max |K - K_oracle| over the stored oracle entries of the 96-atom workload."""
    if not os.path.exists(GOLDEN):
        return {"value": None, "note": "oracle entries file missing"}
    d = np.loadtxt(GOLDEN)
    mu, nu, ref = d[:, 0].astype(int), d[:, 1].astype(int), d[:, 2]
    err = float(np.max(np.abs(K[mu, nu] - ref)))
    return {"value": err, "vs": f"{len(ref)} entries of the unscreened FP64 CPU oracle (tests/golden)",
            "tolerance": 1e-10}


def cpu_oracle_rate(p, target_s: float = 12.0):
    """The oracle on a bounded random sample of grid points; returns
    (builds/s extrapolated, threads, sample description)."""
    import oracle
    import synth
    rng = np.random.default_rng(0)
    n_total = p.grid.n_points
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def run(n):
        idx = np.sort(rng.choice(n_total, size=n, replace=False))
        g = synth.Grid(xyz=p.grid.xyz[idx], w=p.grid.w[idx], atom=p.grid.atom[idx])
        t = time.perf_counter()
        oracle.snk_K(p.basis, g, p.P, nthreads=cores)
        return time.perf_counter() - t

    n0 = max(cores * 4, 64)
    t0 = run(n0)
    n = int(min(n_total, max(n0, n0 * target_s / max(t0, 1e-3))))
    t = run(n)
    rate = (n / n_total) / t
    return rate, cores, f"{n} of {n_total} grid points drawn at random (seed 0), {t:.1f} s; builds/s = (n/N_g)/t"


def run_reference(args, rank, world):
    import synth
    if rank != 0:
        return 0
    p = synth.cluster96()
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    rng = np.random.default_rng(1)
    per_step = max(cores * 8, 64)
    times = []
    for step in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(p.grid.n_points, size=per_step, replace=False))
        g = synth.Grid(xyz=p.grid.xyz[idx], w=p.grid.w[idx], atom=p.grid.atom[idx])
        t = time.perf_counter()
        oracle.snk_K(p.basis, g, p.P, nthreads=cores)
        if step >= args.warmup:
            times.append(time.perf_counter() - t)
    t = float(np.sum(times))
    builds = args.steps * per_step / p.grid.n_points
    value = builds / t
    sample = (f"each step: the FP64 CPU oracle (plain C, OpenMP) on {per_step} of {p.grid.n_points} grid points; "
              f"builds/s = steps * sample / N_g / time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "K-builds/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(p),
            "cpu_baseline": {"value": value, "unit": "K-builds/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "K-builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD)
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import synth
    import paper_2303_14280_gb300 as snk

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    snk.lib()
    dev = torch.device("cuda", local)
    p = synth.cluster96(device=dev) if args.workload == WORKLOAD else getattr(synth, args.workload)(device=dev)
    t_create = time.perf_counter()
    eng = snk.Engine(p.basis, p.grid)
    t_create = time.perf_counter() - t_create
    stream = torch.cuda.current_stream()
    eng.set_stream(stream)
    nf = eng.nf
    Pd = torch.from_numpy(p.P).to(dev)
    Kd = torch.empty_like(Pd)

    def step():
        eng.set_density(Pd)
        eng.build_K(out=Kd)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = eng.stats()

    # device-resident timing: K steps between events on the engine's stream
    k_ms_int, flops_int = 0.0, 0.0
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
            s = eng.stats()       # integral-kernel time from the library's events on the same stream
            k_ms_int += s["ms_integrals"]
            flops_int += s["integral_flops"]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    st = eng.stats()
    ms_t = torch.tensor([ms], device=dev)
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms = float(ms_t.item())
    value = world * args.steps / (ms * 1e-3)

    # end to end through the C ABI with host buffers
    Ph = np.ascontiguousarray(p.P)
    Kh = np.empty_like(Ph)
    barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        eng.set_density(Ph)
        eng.build_K(out=Kh)
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t
    e2e_t = torch.tensor([e2e_s], device=dev)
    if dist is not None:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = world * args.steps / float(e2e_t.item())
    kdiff = float(np.max(np.abs(Kh - Kd.cpu().numpy())))

    achieved = flops_int / (k_ms_int * 1e-3) / 1e12 if k_ms_int > 0 else None
    dK = sampled_parity(Kh) if args.workload == WORKLOAD else None
    line = {
        "metric": METRIC, "value": value, "unit": "K-builds/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(p, args.workload),
        "form": "plain FP64", "max_abs_dK": dK,
        "integrals_per_s": st["integrals"] / (ms / args.steps * 1e-3),
        "phases_ms": {k: st[k] for k in ("ms_screen", "ms_collocation", "ms_fgemm", "ms_integrals", "ms_kgemm",
                                         "ms_finish", "ms_build")},
        "integral_ms_by_class": dict(zip(["ss", "ps", "pp", "ds", "dp", "dd"], st["ms_integrals_class"])),
        "pairs_kept": st["pairs_kept"], "n_batches": st["n_batches"], "integrals_per_build": st["integrals"],
        "create_s": t_create,
        "roofline": {"bound": "alu", "kernel": "integral_kernel<la,lb> (FP64 VRR/HRR + contraction)",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
                     "peak_source": "nominal FP64 of the recipe (not in MEASURED_PEAKS.json); a DFMA microbenchmark "
                                    "measured 1.19 TFLOP/s"},
        "clocks": clocks,
        "gpu_launches": int(st["kernel_launches"]) * args.steps,
        "e2e": {"value": e2e_value, "unit": "K-builds/s", "h2d_bytes_per_step": nf * nf * 8,
                "d2h_bytes_per_step": nf * nf * 8, "host_vs_device_K_max_abs_diff": kdiff},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate(p)
        line["cpu_baseline"] = {"value": rate, "unit": "K-builds/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
    eng.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

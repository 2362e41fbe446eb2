#!/usr/bin/env python3
"""sn-K K-build throughput on GB300: the chosen form against plain FP64.

One step = one full K build: snk_set_density (P upload, symmetry check,
F-tilde, sn-LinK screen, learned screen, task lists) followed by snk_build_K
(collocation, F = X P, 3c-CP integrals contracted into G, K-tilde = G^T X,
symmetrisation).  Inputs are resident in HBM when the timed region starts
(`value`); `e2e` repeats the chosen form through the C ABI with host buffers,
the P upload and the K download inside the timed region.

Forms:
  plain   FP64 everywhere, rigorous sn-LinK screen at 1e-12 (eps_B = eps_E = eps_K)
  chosen  rigorous screen at 1e-10, then the learned block screen (shipped
          weights and calibrated thresholds: skip, and move high-tier blocks
          with a small predicted contribution to FP32); pairs whose sn-LinK estimate is
          below 3e-4 run their integrals in FP32, the rest in double-FP32 (hi +
          lo float pairs, ~1e-14 relative); F = X P and Kt = G^T X on the
          tcgen05 tensor cores as bf16 fixed-point slice products (5 slices
          for the columns of shells in double-FP32 pairs, 4 for the rest);
          G and K accumulated in FP64
  (batch64: the 64 molecules in one handle, one launch per phase, CUDA graph,
   autotuned tiles, every pair and GEMM in double-FP32 for the 1e-10 target,
   against 64 separate plain FP64 builds)

Default workload: the 512-atom cluster (5,280 functions, 4,096,000 points).
Its plain FP64 build (~23 minutes) cannot run beside the chosen form's steps,
so the plain arm is timed on the grid points of every 16th atom (a stated,
cost-stratified subset whose batches are those of the full build) and scaled
to the full build phase by phase with the full build's own screened work.
Other workloads: --workload cluster96 | cluster256 | batch64 | batch64_small
(their plain arm runs in full).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (the build does not shard);
the value is the total builds of all ranks over the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of grid points of the same workload and scales to builds/s.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sn-K K-builds/s at stated max|ΔK|: chosen form vs plain FP64, same GB300"
WORKLOAD = "cluster512"
# ALU peaks of GB300 (152 SMs at the 2070 MHz maximum SM clock): FP64 as the
# recipe's nominal 1.25 TFLOP/s; FP32 = 152 x 128 lanes x 2 flop x 2.07 GHz.
# A DFMA / FFMA microbenchmark on this pool measured 1.19 and 73.2 TFLOP/s.
FP64_PEAK = 1.25
FP32_PEAK = 152 * 128 * 2 * 2.07e9 / 1e12
DF32_OPS_PER_MAC = 12      # FP32 instructions per double-FP32 multiply-add (GEMM tiles)
DS_OPS_PER_FLOP = 7.5      # ds fused multiply-add: 15 FP32 instructions for 2 flops
FP32_INSTR_RATE = 152 * 128 * 2.07e9 / 1e12   # T FP32 lane-instructions/s
FP64_DFMA_MEASURED = 1.19  # TFLOP/s, a DFMA microbenchmark on one GB300 of this machine


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


HBM_MEASURED = _measured_peaks().get("hbm_gbs")
HBM_PEAK = float(HBM_MEASURED or 6800.0)
BF16_MEASURED = _measured_peaks().get("bf16_tflops")
BF16_PEAK = float(BF16_MEASURED or 1900.0)
PLAIN = dict()
CHOSEN = dict(eps=1e-10, precision="mixed", fp32_bound=3e-4, gemm="split", tc_slices_hi=5, tc_slices_lo=4,
              ds_integrals=1, eps_tile=1e-11)
GOLDEN = {n: os.path.join(ROOT, "tests", "golden", f"{n}_K_entries.txt")
          for n in ("cluster96", "cluster256", "cluster512")}
# workloads whose plain FP64 build is too slow to repeat beside the chosen
# form: the plain arm runs on every k-th atom's grid points (see plain_subset)
PLAIN_SUBSET = {"cluster512": 16}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of every rank's x (the slowest replica sets the job time)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms_max, steps, world, units_per_step=1):
    """Whole-job rate: the units every replica processed over the slowest
    replica's time (replicas only: each rank runs its own full builds)."""
    return world * steps * units_per_step / (ms_max * 1e-3)


def make_problems(name, device=None):
    import synth
    if name == "batch64":
        return [synth.multi_molecule(m, device=device) for m in range(64)]
    if name == "batch64_small":
        return [synth.small_molecule(m, device=device) for m in range(64)]
    return [getattr(synth, name)(device=device)]


def workload_config(name, probs):
    nat = sum(p.mol.Z.shape[0] for p in probs)
    nh = sum(int((p.mol.Z == 8).sum()) for p in probs)
    nf = sum(p.basis.n_functions for p in probs)
    npts = sum(p.grid.n_points for p in probs)
    if name == "batch64":
        desc = (f"batch64: 64 molecules of 6-60 atoms ({nat} atoms, {nf} Cartesian functions up to d, {npts} grid "
                f"points, 40-50 MK radial x 75-160 angular points per atom, Becke), 20% occupied columns")
    elif name == "batch64_small":
        desc = (f"batch64_small: 64 molecules of 4-12 atoms ({nat} atoms, {nf} Cartesian functions up to d, {npts} "
                f"grid points, 40 MK radial x 75 angular points per atom, Becke), 20% occupied columns")
    else:
        p = probs[0]
        desc = (f"{name}: {nat} atoms ({nh} O-like, {nat - nh} H-like), {nf} Cartesian functions up to d, "
                f"{npts} grid points (50 MK radial x 8 GL theta x 20 phi per atom, Becke), "
                f"{p.meta.get('n_occ')} occupied orbitals")
    return {"workload": desc, "batch_max": 4096,
            "l2": "no flush: each step rewrites a workspace of several GB (X, F, G), far above the 126 MB L2"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"snk_bench_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
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


def golden_err(name, K):
    """max |K - K_oracle| over the stored oracle entries of the workload, if any."""
    path = GOLDEN.get(name)
    if path is None or not os.path.exists(path):
        return None
    d = np.loadtxt(path)
    mu, nu, ref = d[:, 0].astype(int), d[:, 1].astype(int), d[:, 2]
    return float(np.max(np.abs(K[mu, nu] - ref)))


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the oracle timings."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_oracle_rate(p, target_s: float = 12.0, seed: int = 0):
    """The oracle on a bounded random sample of grid points; returns
    (builds/s scaled to the full grid, threads, sample description)."""
    import oracle
    import synth
    rng = np.random.default_rng(seed)
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
    return rate, cores, f"{n} of {n_total} grid points drawn at random (seed {seed}), {t:.1f} s; " \
                        f"builds/s = (n / N_g) / t"


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    # the inputs are made on the GPU when there is one (the Becke partition of
    # millions of points; not timed), the oracle alone runs on the host cores
    dev = None
    try:
        import torch
        if torch.cuda.is_available():
            dev = torch.device("cuda", 0)
    except ImportError:
        pass
    probs = make_problems(args.workload, device=dev)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    rng = np.random.default_rng(1)
    n_total = sum(p.grid.n_points for p in probs)
    per_step = max(cores * 8, 64)
    times, done = [], 0.0
    for step in range(args.warmup + args.steps):
        # a bounded sample of the workload's grid points (all molecules of a batch share the sample)
        t = time.perf_counter()
        frac = 0.0
        for p in probs:
            n = max(1, int(round(per_step * p.grid.n_points / n_total)))
            idx = np.sort(rng.choice(p.grid.n_points, size=min(n, p.grid.n_points), replace=False))
            g = synth.Grid(xyz=p.grid.xyz[idx], w=p.grid.w[idx], atom=p.grid.atom[idx])
            oracle.snk_K(p.basis, g, p.P, nthreads=cores)
            frac += idx.shape[0] / p.grid.n_points / len(probs)
        if step >= args.warmup:
            times.append(time.perf_counter() - t)
            done += frac
    t = float(np.sum(times))
    value = done / t
    sample = (f"each step: the FP64 CPU oracle (plain C, OpenMP) on ~{per_step} of the workload's {n_total} grid "
              f"points; builds/s = (sampled fraction of the grid, summed over steps) / time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "K-builds/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.workload, probs),
            "cpu_baseline": {"value": value, "unit": "K-builds/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "K-builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class Runner:
    """One form on one workload: engine(s), a device step and a host (C ABI) step."""

    def __init__(self, snk, probs, opts, batched, dev, stream, learned=None):
        import torch
        self.snk, self.probs, self.batched, self.dev = snk, probs, batched, dev
        t = time.perf_counter()
        if batched:
            self.engs = [snk.Engine([p.basis for p in probs], [p.grid for p in probs], **opts)]
        elif len(probs) == 1:
            self.engs = [snk.Engine(probs[0].basis, probs[0].grid, **opts)]
        else:                                 # one plain engine per molecule
            self.engs = [snk.Engine(p.basis, p.grid, **opts) for p in probs]
        self.create_s = time.perf_counter() - t
        for e in self.engs:
            e.set_stream(stream)
            if learned is not None:
                e.screen_load(learned)
        if batched:
            Pd = np.concatenate([p.P.reshape(-1) for p in probs])
            self.P = [torch.from_numpy(Pd).to(dev)]
        else:
            self.P = [torch.from_numpy(p.P).to(dev) for p in probs] if len(self.engs) > 1 else \
                [torch.from_numpy(probs[0].P).to(dev)]
        self.K = [torch.empty_like(x) for x in self.P]
        self.runs = None
        if batched:                           # the autotuner times builds of the loaded density
            self.engs[0].set_density(self.P[0])
            self.runs = self.engs[0].autotune()

    def step(self):
        for e, P, K in zip(self.engs, self.P, self.K):
            e.set_density(P)
            e.build_K(out=K)

    def host_step(self, Ph, Kh):
        for e, P, K in zip(self.engs, Ph, Kh):
            e.set_density(P)
            e.build_K(out=K)

    def host_buffers(self):
        if self.batched:
            return [[np.ascontiguousarray(p.P) for p in self.probs]], [None]
        return [np.ascontiguousarray(p.P) for p in self.probs], [np.empty_like(p.P) for p in self.probs]

    def Ks(self):
        """Per-molecule host copies of the last device K."""
        if self.batched:
            flat = self.K[0].cpu().numpy()
            out, off = [], 0
            for p in self.probs:
                n = p.basis.n_functions
                out.append(flat[off:off + n * n].reshape(n, n))
                off += n * n
            return out
        return [k.cpu().numpy() for k in self.K]

    def stats(self):
        return [e.stats() for e in self.engs]

    def close(self):
        for e in self.engs:
            e.close()


def timed(runner, steps, warmup, stream, barrier):
    import torch
    for _ in range(warmup):
        runner.step()
    torch.cuda.synchronize()
    acc = {}
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        runner.step()
        for s in runner.stats():        # per-phase times from the library's events on the same stream
            for k in ("ms_integrals", "ms_integrals_fp32", "ms_fgemm", "ms_kgemm", "ms_screen", "ms_collocation",
                      "ms_finish", "integral_flops", "flops_fp32", "gemm_flops", "kernel_launches", "integrals",
                      "colloc_bytes", "ms_gemm_split", "ms_gemm_hi", "ms_gemm_lo", "gemm_tc_flops",
                      "gemm_flops_hi", "pair_points_fp32", "pair_points_fp32_listed"):
                acc[k] = acc.get(k, 0.0) + float(s[k])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1), acc


def measure_vxc(eng, P, stream, reps=2):
    """V^xc (Sec. II.C) of the loaded density on the same handle: PBE builds
    timed with CUDA events on the library stream (one warm-up), the library's
    phase times, and the Slater homogeneity check tr(V P) = 4/3 E_x."""
    import torch
    dV = torch.empty((eng.nf, eng.nf), dtype=torch.float64, device=P.device)
    pbe = 3
    eng.build_Vxc(pbe, out=dV)                         # warm-up (plans the batches once)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ph = dict(ms_xc_collocation=0.0, ms_xc_fgemm=0.0, ms_xc_point=0.0, ms_xc_vgemm=0.0)
    e0.record(stream)
    for _ in range(reps):
        _, Exc = eng.build_Vxc(pbe, out=dV)
        st = eng.stats()
        for k in ph:
            ph[k] += st[k] / reps
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    V, Ex = eng.build_Vxc(1)
    Pn = P.cpu().numpy()
    hom = abs(float(np.sum(V * Pn)) - 4.0 / 3.0 * Ex) / abs(Ex)
    gms = ph["ms_xc_fgemm"] + ph["ms_xc_vgemm"]
    out = {"functional": "PBE (exchange + PW92/PBE correlation), spin-restricted", "ms_per_build": ms,
           "builds_per_s": 1e3 / ms, "E_xc": Exc, "phases_ms": ph,
           "slater_homogeneity_rel_err": hom, "gemm_flops": st["xc_gemm_flops"]}
    if gms > 0:
        a = st["xc_gemm_flops"] / (gms * 1e-3) / 1e12
        out["products"] = {"achieved": a, "unit": "TFLOP/s (FP64-equivalent)", "bound": "alu"}
    if ph["ms_xc_collocation"] > 0:
        out["collocation_gbs"] = st["xc_colloc_bytes"] / (ph["ms_xc_collocation"] * 1e-3) / 1e9
    return out


def subset_atoms(p, k):
    """Every k-th atom of the molecule in a cost-stratified order (heavy atoms
    first, each kind by distance from the centre), starting at k // 2."""
    xyz, Z = p.mol.xyz, p.mol.Z
    r = np.linalg.norm(xyz - xyz.mean(axis=0), axis=1)
    order = sorted(range(Z.shape[0]), key=lambda a: (-int(Z[a]), float(r[a]), a))
    return sorted(order[k // 2::k])


def plain_subset(snk, p, k, stream, barrier, warmup, dev):
    """The plain FP64 build on the grid points of every k-th atom (its own
    octree batches, basis screen and pair lists are those of the full build:
    batching is per atom), scaled to the full grid phase by phase with the
    full build's own screened work: integrals by FP64 integral flops, the two
    products by their flops, collocation by points, the screen measured on the
    full grid.  Returns (ms per full build estimated, details, K of the
    subset, the subset problem)."""
    import synth
    import torch
    full = snk.Engine(p.basis, p.grid, **PLAIN)
    full.set_stream(stream)
    Pd = torch.from_numpy(p.P).to(dev)
    full.set_density(Pd)
    torch.cuda.synchronize()
    sf = full.stats()
    full.close()
    atoms = subset_atoms(p, k)
    mask = np.isin(p.grid.atom, atoms)
    sub = synth.Problem(p.name + f"_every{k}th_atom", p.mol, p.basis,
                        synth.Grid(xyz=p.grid.xyz[mask], w=p.grid.w[mask], atom=p.grid.atom[mask]), p.P, p.meta)
    run = Runner(snk, [sub], dict(PLAIN), False, dev, stream)
    ms, acc = timed(run, 1, warmup, stream, barrier)
    ss = run.stats()[0]
    K = run.Ks()[0]
    run.close()
    r_int = sf["integral_flops"] / max(ss["integral_flops"], 1.0)
    r_gemm = sf["gemm_flops"] / max(ss["gemm_flops"], 1.0)
    r_pts = sf["n_points"] / max(ss["n_points"], 1)
    est = (sf["ms_screen"] + acc["ms_integrals"] * r_int + (acc["ms_fgemm"] + acc["ms_kgemm"]) * r_gemm +
           acc["ms_collocation"] * r_pts + acc["ms_finish"] + max(ms - acc["ms_screen"] - acc["ms_integrals"] -
                                                                  acc["ms_fgemm"] - acc["ms_kgemm"] -
                                                                  acc["ms_collocation"] - acc["ms_finish"], 0.0))
    info = {"method": (f"plain FP64 build timed on the grid points of every {k}th atom ({len(atoms)} of "
                       f"{p.mol.Z.shape[0]} atoms, heavy then light, each by distance from the centre, from "
                       f"offset {k // 2}); per-atom batching makes its batches, basis screen and pair lists those of "
                       "the full build; scaled phase by phase with the full build's own screened work "
                       "(integrals x FP64 integral flops, products x their flops, collocation x points; the "
                       "screen timed on the full grid)"),
            "subset_points": int(ss["n_points"]), "full_points": int(sf["n_points"]),
            "subset_ms": ms, "ratio_integral_flops": r_int, "ratio_gemm_flops": r_gemm,
            "integral_flops_full": sf["integral_flops"], "pairs_kept_full": int(sf["pairs_kept"]),
            "ms_integrals_subset": acc["ms_integrals"], "integral_flops_subset": ss["integral_flops"]}
    return est, info, K, sub


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="host-API steps of the e2e measurement (default: min(steps, 3))")
    ap.add_argument("--plain-steps", type=int, default=None)
    ap.add_argument("--plain-warmup", type=int, default=None)
    ap.add_argument("--plain-subset", type=int, default=None,
                    help="run the plain FP64 arm on every k-th atom (default: 16 for cluster512, else off)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--gemm", default=None, choices=["split", "df32"],
                    help="products of the chosen form (default: its own)")
    ap.add_argument("--slices", default=None, help="split: slices of the high and low tier, e.g. 5,4")
    ap.add_argument("--eps-tile", type=float, default=None, help="tile screen of the FP32 lists (0 = off)")
    ap.add_argument("--workload", default=WORKLOAD,  # cluster24: a small case of cluster96's shape for profiles
                    choices=["cluster24", "cluster96", "cluster256", "cluster512", "batch64", "batch64_small"])
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
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
    stream = torch.cuda.current_stream()
    batch = args.workload.startswith("batch64")
    probs = make_problems(args.workload, device=dev)
    n_mol = len(probs)
    subset_k = args.plain_subset if args.plain_subset is not None else PLAIN_SUBSET.get(args.workload)
    if batch:
        subset_k = None

    # ---- chosen form
    learned = None
    if batch:
        # FP64-grade for the 1e-10 per-molecule target: every pair in double-FP32, double-FP32 GEMMs
        chosen_opts = dict(graph=1, precision="mixed", fp32_bound=0.0, ds_integrals=1, gemm="df32")
        form = ("batched: 64 molecules in one handle, one launch per phase, CUDA graph replay, autotuned tiles; "
                "every pair's integrals and both GEMMs in double-FP32 (FP64-grade, ~1e-14 relative)")
    else:
        chosen_opts = dict(CHOSEN)
        if args.gemm:
            chosen_opts["gemm"] = args.gemm
        if args.slices:
            hi, lo = (int(x) for x in args.slices.split(","))
            chosen_opts.update(tc_slices_hi=hi, tc_slices_lo=lo)
        if args.eps_tile is not None:
            chosen_opts["eps_tile"] = args.eps_tile
        form = ("mixed: rigorous sn-LinK at 1e-10, FP32 integrals for pairs with estimate < 3e-4, double-FP32 "
                "integrals otherwise; F = X P and Kt = G^T X on the tcgen05 tensor cores as sums of bf16 "
                "fixed-point slice products (5 slices for the columns / rows of shells in double-FP32 pairs, 4 "
                "for the rest, exact FP32 accumulation per 256-term run, double-FP32 run sums); FP32 blocks "
                "screened again per 128-point tile at 1e-11 (tile skipped, or its primitive-pair tail trimmed); "
                "FP64 G and K accumulation")
        if chosen_opts["gemm"] != "split":
            form = form.replace("on the tcgen05 tensor cores", f"with gemm={chosen_opts['gemm']} instead of")
        if not args.no_learned and os.path.exists(snk.SCREEN_WEIGHTS):
            learned, thr, meta = snk.trained_screen()
            thr32 = float(meta.get("fp32_threshold", -99.0))
            chosen_opts.update(screen="learned", learned_skip=thr, learned_fp32=thr32)
            form += (f", learned block screen (skip below 10^{thr:g}, double-FP32 blocks predicted below "
                     f"10^{thr32:g} moved to the FP32 tier)")
    ch = Runner(snk, probs, chosen_opts, batch, dev, stream, learned)
    with ClockSampler(local) as clk:
        ms, acc = timed(ch, args.steps, args.warmup, stream, barrier)
    clocks = clk.summary()
    ms = max_over_ranks(ms, dist, dev)
    value = job_throughput(ms, args.steps, world, n_mol if batch else 1)
    unit = "molecule K-builds/s" if batch else "K-builds/s"
    st_ch = ch.stats()
    K_ch = ch.Ks()

    # e2e through the C ABI with host buffers (P upload and K download inside)
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else min(args.steps, 3)
    Ph, Kh = ch.host_buffers()
    barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        if batch:
            ch.engs[0].set_density(Ph[0])
            Kh = [ch.engs[0].build_K()]
        else:
            ch.host_step(Ph, Kh)
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t, dist, dev)
    e2e_value = job_throughput(e2e_s * 1e3, e2e_steps, world, n_mol if batch else 1)
    nbytes = sum(p.P.nbytes for p in probs)
    ch_create = ch.create_s
    vxc = None
    if not batch:
        try:
            vxc = measure_vxc(ch.engs[0], ch.P[0], stream)
        except Exception as e:        # reported, not fatal: the K-build line above stands
            vxc = {"error": str(e)}
    ch.close()

    # ---- plain FP64 beside it: the full build, or its stated subset scaled to the full build
    pw = args.plain_warmup if args.plain_warmup is not None else (1 if subset_k else args.warmup)
    err_ch_pl_sub = None
    acc_pl = None
    if subset_k:
        est_ms, plain_info, K_sub, subp = plain_subset(snk, probs[0], subset_k, stream, barrier, pw, dev)
        ms_pl = max_over_ranks(est_ms, dist, dev)
        ps = 1
        value_pl = job_throughput(ms_pl, 1, world, 1)
        # the chosen form on the same subset grid, against the plain K there (every entry)
        sub_ch = Runner(snk, [subp], chosen_opts, False, dev, stream, learned)
        sub_ch.step()
        torch.cuda.synchronize()
        err_ch_pl_sub = float(np.max(np.abs(sub_ch.Ks()[0] - K_sub)))
        sub_ch.close()
        K_pl = None
        pairs_pl = plain_info["pairs_kept_full"]
    else:
        pl = Runner(snk, probs, dict(PLAIN), False, dev, stream)
        ps = args.plain_steps if args.plain_steps is not None else args.steps
        ms_pl, acc_pl = timed(pl, ps, pw, stream, barrier)
        ms_pl = max_over_ranks(ms_pl, dist, dev) / ps
        value_pl = job_throughput(ms_pl * ps, ps, world, n_mol)
        K_pl = pl.Ks()
        pairs_pl = sum(s["pairs_kept"] for s in pl.stats())
        pl.close()
        plain_info = {"method": f"full plain FP64 builds, {ps} timed after {pw} warm-up"}

    dK_ch_pl = max(float(np.max(np.abs(a - b))) for a, b in zip(K_ch, K_pl)) if K_pl is not None else None
    err_ch = golden_err(args.workload, K_ch[0]) if not batch else None
    err_pl = golden_err(args.workload, K_pl[0]) if (not batch and K_pl is not None) else None

    # ---- rooflines of the chosen step's kernels (library events, same stream)
    n = args.steps
    kern = {}
    if acc.get("ms_integrals_fp32", 0) > 0:
        a = acc["flops_fp32"] / (acc["ms_integrals_fp32"] * 1e-3) / 1e12
        kern["integral_kernel_f32"] = {"ms_per_step": acc["ms_integrals_fp32"] / n, "bound": "alu", "achieved": a,
                                       "peak": FP32_PEAK, "unit": "TFLOP/s", "frac": a / FP32_PEAK}
    ms64 = acc["ms_integrals"]          # the FP64 (or ds) lists; the FP32 lists are counted apart
    if ms64 > 0:
        a = acc["integral_flops"] / (ms64 * 1e-3) / 1e12
        if chosen_opts.get("ds_integrals"):
            # ds arithmetic on the FP32 pipe: ceiling = FP32 instruction rate / instructions per flop
            peak = FP32_INSTR_RATE / DS_OPS_PER_FLOP
            kern["integral_kernel_ds"] = {"ms_per_step": ms64 / n, "bound": "alu", "achieved": a, "peak": peak,
                                          "unit": "TFLOP/s (FP64-equivalent flops)", "frac": a / peak,
                                          "vs_fp64_pipe_peak": a / FP64_PEAK}
        else:
            kern["integral_kernel"] = {"ms_per_step": ms64 / n, "bound": "alu", "achieved": a, "peak": FP64_PEAK,
                                       "unit": "TFLOP/s", "frac": a / FP64_PEAK}
    gms = acc["ms_fgemm"] + acc["ms_kgemm"]
    if chosen_opts.get("gemm") == "split" and gms > 0:
        # tensor-core products against the measured bf16 peak: flops of the slice
        # products issued (padded tiles), and the algorithmic FP64-equivalent rate
        sh = chosen_opts.get("tc_slices_hi", 5)
        sl = chosen_opts.get("tc_slices_lo", 4)
        fh = acc["gemm_flops_hi"]
        fl = acc["gemm_flops"] - fh
        for name, ms_k, f64, prods in (("tc_gemm_hi", acc["ms_gemm_hi"], fh, sh * (sh + 1) // 2),
                                       ("tc_gemm_lo", acc["ms_gemm_lo"], fl, sl * (sl + 1) // 2)):
            if ms_k > 0:
                a = f64 * prods / (ms_k * 1e-3) / 1e12
                kern[name] = {"ms_per_step": ms_k / n, "bound": "tensor", "achieved": a, "peak": BF16_PEAK,
                              "unit": "TFLOP/s (bf16 slice products, algorithmic sizes)", "frac": a / BF16_PEAK,
                              "fp64_equivalent_tflops": f64 / (ms_k * 1e-3) / 1e12, "slice_products": prods,
                              "peak_source": "MEASURED_PEAKS.json bf16_tflops" if BF16_MEASURED else
                              "fallback 1900 TFLOP/s"}
        if acc["ms_gemm_hi"] + acc["ms_gemm_lo"] > 0:
            kern["tc_gemm_issued"] = {"tflops": acc["gemm_tc_flops"] / ((acc["ms_gemm_hi"] + acc["ms_gemm_lo"]) * 1e-3)
                                      / 1e12, "note": "bf16 flops issued incl. tile padding, both tiers"}
        kern["gemm_operand_split"] = {"ms_per_step": acc["ms_gemm_split"] / n, "bound": "hbm",
                                      "note": "slicing X, P[S_j,B_j], G into bf16 blocks and the FP32-tier G merge"}
    elif gms > 0:
        a = acc["gemm_flops"] / (gms * 1e-3) / 1e12
        if not batch:     # double-FP32 (12 FP32 instructions per multiply-add) and split-TF32 columns
            peak = FP32_PEAK / DF32_OPS_PER_MAC
            kern["fgemm_kgemm_split"] = {"ms_per_step": gms / n, "bound": "alu", "achieved": a, "peak": peak,
                                        "unit": "TFLOP/s (FP64-equivalent 2 flop per multiply-add)",
                                        "frac": a / peak}
        else:
            kern["fgemm_kgemm_fp64"] = {"ms_per_step": gms / n, "bound": "alu", "achieved": a, "peak": FP64_PEAK,
                                        "unit": "TFLOP/s", "frac": a / FP64_PEAK}
    if acc.get("ms_collocation", 0) > 0 and acc.get("colloc_bytes", 0) > 0:
        a = acc["colloc_bytes"] / (acc["ms_collocation"] * 1e-3) / 1e9
        kern["collocation_kernel"] = {"ms_per_step": acc["ms_collocation"] / n, "bound": "hbm", "achieved": a,
                                      "peak": HBM_PEAK, "unit": "GB/s", "frac": a / HBM_PEAK,
                                      "peak_source": "MEASURED_PEAKS.json hbm_gbs" if HBM_MEASURED else
                                      "fallback 6800 GB/s"}
    # the plain arm's FP64 integral kernel against the FP64 pipe
    plain_kernel = None
    if subset_k:
        if plain_info["ms_integrals_subset"] > 0:
            a = plain_info["integral_flops_subset"] / (plain_info["ms_integrals_subset"] * 1e-3) / 1e12
            plain_kernel = {"ms": plain_info["ms_integrals_subset"], "achieved": a, "unit": "TFLOP/s",
                            "peak": FP64_PEAK, "frac": a / FP64_PEAK, "frac_of_measured_dfma": a / FP64_DFMA_MEASURED,
                            "on": "the plain subset build"}
    elif acc_pl and acc_pl["ms_integrals"] > 0:
        a = acc_pl["integral_flops"] / (acc_pl["ms_integrals"] * 1e-3) / 1e12
        plain_kernel = {"ms_per_step": acc_pl["ms_integrals"] / ps, "achieved": a, "unit": "TFLOP/s",
                        "peak": FP64_PEAK, "frac": a / FP64_PEAK, "frac_of_measured_dfma": a / FP64_DFMA_MEASURED}
    if plain_kernel:
        kern["plain_integral_kernel_fp64"] = dict(plain_kernel, bound="alu")
    dom = max((k for k in kern if k != "plain_integral_kernel_fp64" and "achieved" in kern[k]),
              key=lambda k: kern[k]["ms_per_step"], default=None)
    roof = None
    if dom:
        d = kern[dom]
        roof = {"bound": d["bound"], "kernel": dom, "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
                "frac": d["frac"], "traffic": None,
                "peak_source": "derived ALU ceiling at 2070 MHz, not in MEASURED_PEAKS.json: FP64 = the recipe's "
                               "nominal 1.25 TFLOP/s; FP32 = 152 SMs x 128 lanes x 2 flop = 80.5 TFLOP/s; "
                               "double-FP32 = 40.3 T FP32 instructions/s / 7.5 per flop (integrals) or / 6 per "
                               "flop (GEMM tiles)"}

    line = {
        "metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": workload_config(args.workload, probs),
        "form": form,
        "max_abs_dK": {"chosen_vs_oracle_entries": err_ch, "plain_vs_oracle_entries": err_pl,
                       "chosen_vs_plain_full": dK_ch_pl, "chosen_vs_plain_on_plain_subset_grid": err_ch_pl_sub,
                       "stated_tolerance": 1e-10 if batch else 1e-8},
        "plain_fp64": dict({"value": value_pl, "unit": unit, "ms_per_step": ms_pl, "steps": ps, "warmup": pw,
                            "pairs_kept": pairs_pl}, **plain_info),
        "speedup_vs_plain_fp64": value / value_pl,
        "integrals_per_s": acc["integrals"] / (ms * 1e-3),
        "phases_ms_per_step": {k: acc[k] / n for k in ("ms_screen", "ms_collocation", "ms_fgemm", "ms_integrals",
                                                         "ms_integrals_fp32", "ms_kgemm", "ms_finish")},
        "kernels": kern,
        "integral_ms_by_class": {tier: dict(zip(["ss", "ps", "pp", "ds", "dp", "dd"],
                                                [round(x, 2) for x in st_ch[0][key]]))
                                 for tier, key in (("high", "ms_integrals_class"),
                                                   ("fp32", "ms_integrals_class_fp32"))},
        "pairs_kept": sum(s["pairs_kept"] for s in st_ch),
        "pairs_kept_fp32": sum(s["pairs_kept_fp32"] for s in st_ch),
        "pairs_learned_skipped": sum(s["pairs_learned_skipped"] for s in st_ch),
        "fp32_pair_points_computed_fraction": (acc["pair_points_fp32"] / acc["pair_points_fp32_listed"]
                                               if acc.get("pair_points_fp32_listed") else None),
        "create_s": ch_create,
        "vxc": vxc,
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": int(acc["kernel_launches"]),
        "e2e": {"value": e2e_value, "unit": unit, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "steps": e2e_steps},
    }
    if vxc and "products" in vxc:
        mixed = chosen_opts.get("precision") == "mixed"
        pr = vxc["products"]
        if mixed and chosen_opts.get("gemm") == "split":
            # tcgen05 split products: S(S+1)/2 bf16 slice products per FP64-equivalent product
            sl = chosen_opts.get("tc_slices_hi", 5)
            f64 = pr["achieved"]
            a = f64 * sl * (sl + 1) // 2
            pr.update(achieved=a, unit="TFLOP/s (bf16 slice products, algorithmic sizes)", bound="tensor",
                      peak=BF16_PEAK, frac=a / BF16_PEAK, fp64_equivalent_tflops=f64,
                      tiles=f"tcgen05 split products, {sl} slices")
        else:                          # double-FP32 tiles in the mixed form, FP64 tiles otherwise
            peak = FP32_PEAK / DF32_OPS_PER_MAC if mixed else FP64_PEAK
            pr.update(peak=peak, frac=pr["achieved"] / peak, tiles="double-FP32" if mixed else "FP64")
    if batch:
        line["autotuned_pairs_per_tile"] = ch.runs
        line["phases_ms_per_step"] = None   # graph replay: no per-phase events
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate(probs[0] if not batch else probs[int(np.argmax(
            [p.grid.n_points for p in probs]))])
        if batch:
            sample += " (largest molecule of the batch; molecule builds/s)"
        line["cpu_baseline"] = {"value": rate, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample,
                                "cpu_model": cpu_model()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

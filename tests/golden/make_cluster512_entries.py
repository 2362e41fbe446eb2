#!/usr/bin/env python3
"""Write cluster512_K_entries.txt: sampled entries of the unscreened FP64 sn-K
exchange matrix of the 512-atom workload (5,280 functions, 4,096,000 grid
points), computed by the CPU oracle alone (blocked entries mode: per block of
points Phi, F = Phi P as a library matrix product, and only the G rows of the
chosen shells).

The entries are every (mu, nu), mu <= nu, with mu and nu among the functions
of three shells chosen by a fixed rule: the first d shell of the heavy atom
nearest the centre, and the s and p shells of the light (H-like, 2s1p) atom
nearest to that heavy atom (10 functions, 55 entries: diagonal, intra-atom
and inter-atom blocks, heavy and light rows).

Run from the repository root:  python tests/golden/make_cluster512_entries.py
(about 2-3 hours on 8 cores).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cluster512_K_entries.txt")


def chosen_shells(p):
    b = p.basis
    Z, xyz = p.mol.Z, p.mol.xyz
    heavy = [a for a in range(Z.shape[0]) if Z[a] == 8]
    light = [a for a in range(Z.shape[0]) if Z[a] == 1]
    centre = xyz.mean(axis=0)
    h = heavy[int(np.argmin([np.linalg.norm(xyz[a] - centre) for a in heavy]))]
    li = light[int(np.argmin([np.linalg.norm(xyz[a] - xyz[h]) for a in light]))]
    shells = []
    for a, l in ((h, 2), (li, 0), (li, 1)):
        shells.append([s for s in range(b.n_shells) if b.atom[s] == a and b.l[s] == l][0])
    return shells


def entries(p):
    b = p.basis
    foff = np.concatenate([[0], np.cumsum([(int(l) + 1) * (int(l) + 2) // 2 for l in b.l])])
    funcs = np.concatenate([np.arange(foff[s], foff[s + 1]) for s in chosen_shells(p)])
    mu, nu = np.meshgrid(funcs, funcs, indexing="ij")
    keep = mu <= nu
    return mu[keep].astype(np.int32), nu[keep].astype(np.int32)


def main():
    t0 = time.time()
    p = synth.cluster512()
    print(f"inputs in {time.time() - t0:.0f} s", flush=True)
    mu, nu = entries(p)
    t = time.time()

    def progress(done, n):
        print(f"{done}/{n} points, {time.time() - t:.0f} s", flush=True)

    vals = oracle.snk_K_entries_blocked(p.basis, p.grid, p.P, mu, nu, progress=progress)
    dt = time.time() - t
    with open(OUT, "w") as f:
        f.write("# unscreened FP64 sn-K of synth.cluster512() by the CPU oracle (oracle.snk_K_entries_blocked)\n")
        f.write(f"# n_functions {p.basis.n_functions} n_points {p.grid.n_points} oracle seconds {dt:.1f}\n")
        f.write("# mu nu K_mu_nu\n")
        for a, b_, v in zip(mu, nu, vals):
            f.write(f"{a} {b_} {v:.17e}\n")
    print(f"wrote {len(mu)} entries in {dt:.1f} s")


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Write cluster96_light_K_entries.txt: sampled entries of the unscreened FP64
sn-K exchange matrix of the 96-atom workload (992 functions, 768,000 grid
points) on the light (H-like, 2s1p) atoms, computed by the CPU oracle alone
(blocked entries mode: per block of points Phi, F = Phi P as a library matrix
product, and only the G rows of the chosen shells).

The entries are every (mu, nu), mu <= nu, among the functions of four shells
chosen by a fixed rule: the s and p shells of the light atom nearest the
centre and of the light atom farthest from it (8 functions, 36 entries:
diagonal, intra-atom, and a far-apart inter-atom block).

Run from the repository root:  python tests/golden/make_cluster96_light_entries.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cluster96_light_K_entries.txt")


def chosen_shells(p):
    b = p.basis
    Z, xyz = p.mol.Z, p.mol.xyz
    light = [a for a in range(Z.shape[0]) if Z[a] == 1]
    d = [np.linalg.norm(xyz[a] - xyz.mean(axis=0)) for a in light]
    shells = []
    for a in (light[int(np.argmin(d))], light[int(np.argmax(d))]):
        for l in (0, 1):
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
    p = synth.cluster96()
    mu, nu = entries(p)
    t = time.time()
    vals = oracle.snk_K_entries_blocked(p.basis, p.grid, p.P, mu, nu)
    dt = time.time() - t
    with open(OUT, "w") as f:
        f.write("# unscreened FP64 sn-K of synth.cluster96() by the CPU oracle (oracle.snk_K_entries_blocked)\n")
        f.write(f"# n_functions {p.basis.n_functions} n_points {p.grid.n_points} oracle seconds {dt:.1f}\n")
        f.write("# mu nu K_mu_nu\n")
        for a, b_, v in zip(mu, nu, vals):
            f.write(f"{a} {b_} {v:.17e}\n")
    print(f"wrote {len(mu)} entries in {dt:.1f} s")


if __name__ == "__main__":
    main()

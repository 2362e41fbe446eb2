#!/usr/bin/env python3
"""Write cluster96_vxc_entries.txt: sampled entries of the FP64 PBE
exchange-correlation matrix V^xc (Sec. II.C) and E_xc of the 96-atom workload
(992 functions, 768,000 grid points), computed by the CPU oracle alone
(oracle.vxc_entries: every function on every point, no screening).

The entries are every (mu, nu), mu <= nu, among the functions of eight shells
chosen by a fixed rule: the s, p and d shells of the heavy atoms nearest to and
farthest from the centre, and the s and p shells of the light atom nearest to
the centre.

Run from the repository root:  python tests/golden/make_cluster96_vxc_entries.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cluster96_vxc_entries.txt")
FUNCTIONAL = oracle.XC_PBE


def chosen_shells(p):
    b = p.basis
    centre = p.mol.xyz.mean(axis=0)
    d = np.linalg.norm(p.mol.xyz - centre, axis=1)
    heavy = [a for a in range(p.mol.Z.shape[0]) if p.mol.Z[a] == 8]
    light = [a for a in range(p.mol.Z.shape[0]) if p.mol.Z[a] == 1]
    picks = [(heavy[int(np.argmin(d[heavy]))], (0, 1, 2)), (heavy[int(np.argmax(d[heavy]))], (0, 1, 2)),
             (light[int(np.argmin(d[light]))], (0, 1))]
    shells = []
    for a, ls in picks:
        for l in ls:
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
    vals, exc = oracle.vxc_entries(p.basis, p.grid, p.P, FUNCTIONAL, mu, nu)
    dt = time.time() - t
    with open(OUT, "w") as f:
        f.write("# FP64 PBE V^xc of synth.cluster96() by the CPU oracle (oracle.vxc_entries), no screening\n")
        f.write(f"# n_functions {p.basis.n_functions} n_points {p.grid.n_points} oracle seconds {dt:.1f}\n")
        f.write(f"# E_xc {exc:.17e}\n")
        f.write("# mu nu V_mu_nu\n")
        for a, b_, v in zip(mu, nu, vals):
            f.write(f"{a} {b_} {v:.17e}\n")
    print(f"{len(mu)} entries, E_xc {exc:.12f}, {dt:.1f} s -> {OUT}")


if __name__ == "__main__":
    main()

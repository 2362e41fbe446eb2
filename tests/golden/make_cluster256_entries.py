#!/usr/bin/env python3
"""Write cluster256_K_entries.txt: sampled entries of the unscreened FP64 sn-K
exchange matrix of the 256-atom workload (mixed-precision form's test case,
about 2,700 functions and 2,048,000 grid points), computed by the CPU oracle
alone (entries mode: only the G rows of the chosen shells are formed).

The entries are every (mu, nu), mu <= nu, with mu and nu among the functions
of five shells chosen by a fixed rule: the s, p and d shells of the heavy atom
nearest the centre and the s and p shells of the heavy atom farthest from it
(14 functions, 105 entries: diagonal, intra-atom and inter-atom blocks).

Run from the repository root:  python tests/golden/make_cluster256_entries.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cluster256_K_entries.txt")


def chosen_shells(p):
    b = p.basis
    heavy = [a for a in range(p.mol.Z.shape[0]) if p.mol.Z[a] == 8]
    centre = p.mol.xyz.mean(axis=0)
    d = [np.linalg.norm(p.mol.xyz[a] - centre) for a in heavy]
    near, far = heavy[int(np.argmin(d))], heavy[int(np.argmax(d))]
    shells = []
    for a, ls in ((near, (0, 1, 2)), (far, (0, 1))):
        for l in ls:
            cand = [s for s in range(b.n_shells) if b.atom[s] == a and b.l[s] == l]
            shells.append(cand[0])
    return shells


def entries(p):
    b = p.basis
    foff = np.concatenate([[0], np.cumsum([(int(l) + 1) * (int(l) + 2) // 2 for l in b.l])])
    funcs = np.concatenate([np.arange(foff[s], foff[s + 1]) for s in chosen_shells(p)])
    mu, nu = np.meshgrid(funcs, funcs, indexing="ij")
    keep = mu <= nu
    return mu[keep].astype(np.int32), nu[keep].astype(np.int32)


def main():
    p = synth.cluster256()
    mu, nu = entries(p)
    t = time.time()
    vals = oracle.snk_K_entries(p.basis, p.grid, p.P, mu, nu)
    dt = time.time() - t
    with open(OUT, "w") as f:
        f.write("# unscreened FP64 sn-K of synth.cluster256() by the CPU oracle (oracle.snk_K_entries)\n")
        f.write(f"# n_functions {p.basis.n_functions} n_points {p.grid.n_points} oracle seconds {dt:.1f}\n")
        f.write("# mu nu K_mu_nu\n")
        for a, b_, v in zip(mu, nu, vals):
            f.write(f"{a} {b_} {v:.17e}\n")
    print(f"wrote {len(mu)} entries in {dt:.1f} s")


if __name__ == "__main__":
    main()

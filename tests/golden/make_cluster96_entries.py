#!/usr/bin/env python3
"""Write cluster96_K_entries.txt: sampled entries of the unscreened FP64 sn-K
exchange matrix of the 96-atom workload (992 functions, 768,000 grid points),
computed by the CPU oracle alone (entries mode: only the G rows of the chosen
shells are formed).

The entries are every (mu, nu) with mu and nu among the functions of six
shells chosen by a fixed rule (an s, a p and a d shell of two different
heavy atoms), i.e. diagonal blocks, intra-atom and inter-atom blocks.

Run from the repository root:  python tests/golden/make_cluster96_entries.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cluster96_K_entries.txt")


def chosen_shells(p):
    b = p.basis
    heavy = [a for a in range(p.mol.Z.shape[0]) if p.mol.Z[a] == 8]
    centre = p.mol.xyz.mean(axis=0)
    # the heavy atom nearest the centre and the one farthest from it
    d = [np.linalg.norm(p.mol.xyz[a] - centre) for a in heavy]
    atoms = [heavy[int(np.argmin(d))], heavy[int(np.argmax(d))]]
    shells = []
    for a in atoms:
        for l in (0, 1, 2):
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
    p = synth.cluster96()
    mu, nu = entries(p)
    t = time.time()
    vals = oracle.snk_K_entries(p.basis, p.grid, p.P, mu, nu)
    dt = time.time() - t
    with open(OUT, "w") as f:
        f.write("# unscreened FP64 sn-K of synth.cluster96() by the CPU oracle (oracle.snk_K_entries)\n")
        f.write(f"# n_functions {p.basis.n_functions} n_points {p.grid.n_points} oracle seconds {dt:.1f}\n")
        f.write("# mu nu K_mu_nu\n")
        for a, b_, v in zip(mu, nu, vals):
            f.write(f"{a} {b_} {v:.17e}\n")
    print(f"wrote {len(mu)} entries in {dt:.1f} s")


if __name__ == "__main__":
    main()

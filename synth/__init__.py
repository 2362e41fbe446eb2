"""Seeded synthetic inputs for the sn-K build: molecule, basis, grid, density.

This module is shared by the oracle-side tests and the CUDA path. It holds no
arithmetic of the sn-K method itself (no normalisation, no integrals, no
collocation): it only draws geometries, raw basis data, quadrature grids and
density matrices, each from a seeded NumPy generator.

The workloads stand in for the molecules of the paper's results section
(Taxol ... Ubiquitin, 6-31G(d) Cartesian, Table "mol"), whose geometries and
basis data are not available.  They keep the shapes: roughly 10 Cartesian
functions per atom with d shells, a few thousand grid points per atom, grid
batches of at most 4096 points.

Units: coordinates are drawn in Angstrom and returned in bohr.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903

# Shell recipes per element: list of (l, j) where shell j of angular momentum l
# uses the even-tempered exponents alpha_{3j}, alpha_{3j+1}, alpha_{3j+2},
# alpha_k = 0.1 * 3**k.
RECIPES = {
    # 3s2p1d heavy (15 Cartesian functions), 2s light (2)
    "small": {8: [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (2, 0)],
              1: [(0, 0), (0, 1)]},
    # 3s2p2d heavy (21), 2s1p light (5)
    "scale": {8: [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (2, 0), (2, 1)],
              1: [(0, 0), (0, 1), (1, 0)]},
}
NPRIM = 3


def even_tempered(k: int) -> float:
    return 0.1 * 3.0 ** k


@dataclass
class Molecule:
    Z: np.ndarray          # (n_atoms,) int32
    xyz: np.ndarray        # (n_atoms, 3) bohr


@dataclass
class Basis:
    l: np.ndarray          # (n_shells,) int32
    nprim: np.ndarray      # (n_shells,) int32
    atom: np.ndarray       # (n_shells,) int32
    center: np.ndarray     # (n_shells, 3) float64, bohr
    exps: np.ndarray       # (sum nprim,) float64
    coefs: np.ndarray      # (sum nprim,) float64, w.r.t. x^l-normalised primitives

    @property
    def n_shells(self) -> int:
        return int(self.l.shape[0])

    @property
    def n_functions(self) -> int:
        return int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in self.l))


@dataclass
class Grid:
    xyz: np.ndarray        # (n_points, 3) float64, bohr
    w: np.ndarray          # (n_points,) float64
    atom: np.ndarray       # (n_points,) int32

    @property
    def n_points(self) -> int:
        return int(self.w.shape[0])


@dataclass
class Problem:
    name: str
    mol: Molecule
    basis: Basis
    grid: Grid
    P: np.ndarray          # (n_b, n_b) float64, symmetric
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# molecules
# --------------------------------------------------------------------------

def make_chain_molecule(seed: int) -> Molecule:
    """H-O-O-H chain: bonds ~ U(0.9, 1.5) A along random directions, every
    non-bonded pair at least 0.9 A apart."""
    rng = np.random.default_rng(seed)
    Z = np.array([1, 8, 8, 1], dtype=np.int32)
    while True:
        pos = [np.zeros(3)]
        for _ in range(3):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            pos.append(pos[-1] + rng.uniform(0.9, 1.5) * d)
        pos = np.array(pos)
        ok = all(np.linalg.norm(pos[i] - pos[j]) >= 0.9
                 for i in range(4) for j in range(i + 2, 4))
        if ok:
            break
    return Molecule(Z=Z, xyz=pos * ANGSTROM_TO_BOHR)


def make_cluster_molecule(n_atoms: int, seed: int, density: float = 0.08,
                          min_sep: float = 1.0) -> Molecule:
    """Random sequential placement of n_atoms in a sphere holding `density`
    atoms per cubic Angstrom; pairs closer than `min_sep` A are rejected.
    One atom in three is heavy (Z=8), the rest light (Z=1)."""
    rng = np.random.default_rng(seed)
    n_heavy = n_atoms // 3
    radius = (3.0 * n_atoms / density / (4.0 * math.pi)) ** (1.0 / 3.0)
    pos = np.zeros((n_atoms, 3))
    n = 0
    tries = 0
    while n < n_atoms:
        tries += 1
        if tries > 10_000_000:
            raise RuntimeError("placement failed")
        p = rng.uniform(-radius, radius, size=3)
        if p @ p > radius * radius:
            continue
        if n and np.min(np.sum((pos[:n] - p) ** 2, axis=1)) < min_sep * min_sep:
            continue
        pos[n] = p
        n += 1
    Z = np.ones(n_atoms, dtype=np.int32)
    Z[rng.permutation(n_atoms)[:n_heavy]] = 8
    return Molecule(Z=Z, xyz=pos * ANGSTROM_TO_BOHR)


# --------------------------------------------------------------------------
# basis
# --------------------------------------------------------------------------

def make_basis(mol: Molecule, recipe: str, seed: int) -> Basis:
    """Raw contracted Cartesian shells: three even-tempered primitives per
    shell, coefficients ~ U(0.2, 1] with respect to the x^l-normalised
    primitive.  Normalisation of the contraction is left to the consumer."""
    rng = np.random.default_rng(seed + 7919)
    rec = RECIPES[recipe]
    ls, nps, atoms, centers, exps, coefs = [], [], [], [], [], []
    for a, z in enumerate(mol.Z):
        for (l, j) in rec[int(z)]:
            ls.append(l)
            nps.append(NPRIM)
            atoms.append(a)
            centers.append(mol.xyz[a])
            for k in range(NPRIM):
                exps.append(even_tempered(3 * j + k))
                coefs.append(1.0 - 0.8 * rng.random())   # in (0.2, 1]
    return Basis(l=np.array(ls, dtype=np.int32), nprim=np.array(nps, dtype=np.int32),
                 atom=np.array(atoms, dtype=np.int32),
                 center=np.array(centers, dtype=np.float64).reshape(-1, 3),
                 exps=np.array(exps, dtype=np.float64), coefs=np.array(coefs, dtype=np.float64))


# --------------------------------------------------------------------------
# grid: Mura-Knowles radial x (Gauss-Legendre theta x trapezoid phi), Becke
# --------------------------------------------------------------------------

MK_ALPHA = 5.0


def mk_radial(n_r: int, alpha: float = MK_ALPHA):
    """Mura-Knowles radial nodes r_k and weights r_k^2 dr_k (bohr)."""
    k = np.arange(1, n_r + 1, dtype=np.float64)
    x = (k - 0.5) / n_r
    r = -alpha * np.log1p(-x ** 3)
    dr = 3.0 * alpha * x ** 2 / ((1.0 - x ** 3) * n_r)
    return r, r * r * dr


def angular_product(n_theta: int, n_phi: int):
    """Unit vectors and weights (summing to 4 pi) of a Gauss-Legendre in
    cos(theta) x equispaced phi product rule."""
    ct, wt = np.polynomial.legendre.leggauss(n_theta)
    phi = 2.0 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    st = np.sqrt(1.0 - ct ** 2)
    dirs = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)),
                     np.outer(ct, np.ones(n_phi))], axis=-1).reshape(-1, 3)
    w = np.outer(wt, np.full(n_phi, 2.0 * math.pi / n_phi)).reshape(-1)
    return dirs, w


def _becke_s(mu):
    f = mu
    for _ in range(3):
        f = 1.5 * f - 0.5 * f ** 3
    return 0.5 * (1.0 - f)


_HERE = os.path.dirname(os.path.abspath(__file__))
_BECKE_SRC = os.path.join(_HERE, "becke.c")
_BECKE_LIB = os.path.join(_HERE, "_build", "libsynth_becke.so")
_becke_lib = None
_becke_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile becke.c (the fused CPU Becke partition) with gcc."""
    os.makedirs(os.path.dirname(_BECKE_LIB), exist_ok=True)
    if (not force and os.path.exists(_BECKE_LIB)
            and os.path.getmtime(_BECKE_LIB) >= os.path.getmtime(_BECKE_SRC)):
        return _BECKE_LIB
    tmp = _BECKE_LIB + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, _BECKE_SRC, "-lm"],
                   check=True)
    os.replace(tmp, _BECKE_LIB)
    return _BECKE_LIB


def _becke_cpu(points, owner, atoms_xyz):
    global _becke_lib
    with _becke_lock:
        if _becke_lib is None:
            L = ctypes.CDLL(build())
            D, I = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
            L.synth_becke.argtypes = [ctypes.c_long, D, I, ctypes.c_int, D, D, ctypes.c_int]
            L.synth_becke.restype = ctypes.c_int
            _becke_lib = L
    pts = np.ascontiguousarray(points, dtype=np.float64)
    own = np.ascontiguousarray(owner, dtype=np.int32)
    A = np.ascontiguousarray(atoms_xyz, dtype=np.float64)
    out = np.empty(pts.shape[0])
    D = ctypes.POINTER(ctypes.c_double)
    rc = _becke_lib.synth_becke(pts.shape[0], pts.ctypes.data_as(D), own.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                A.shape[0], A.ctypes.data_as(D), out.ctypes.data_as(D), 0)
    if rc != 0:
        raise RuntimeError(f"synth_becke failed (rc={rc})")
    return out


def becke_weights(points, owner, atoms_xyz, chunk: int = 4096, device=None):
    """Becke fuzzy-cell partition weight of each point for its own atom
    (three-fold iterated polynomial, no atomic-size adjustment).  On the CPU
    (device None) the fused C routine of becke.c computes it; on a GPU the
    same formula runs as torch tensor operations."""
    if device is None:
        return _becke_cpu(points, owner, atoms_xyz)
    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    A = torch.as_tensor(atoms_xyz, dtype=torch.float64, device=dev)
    nat = A.shape[0]
    if nat == 1:
        return np.ones(points.shape[0])
    Rab = torch.cdist(A, A)
    inv = torch.where(Rab > 0, 1.0 / torch.where(Rab > 0, Rab, torch.ones_like(Rab)),
                      torch.zeros_like(Rab))
    out = np.empty(points.shape[0])
    own = torch.as_tensor(owner, dtype=torch.int64, device=dev)
    eye = torch.eye(nat, dtype=torch.bool, device=dev)
    for s in range(0, points.shape[0], chunk):
        r = torch.as_tensor(points[s:s + chunk], dtype=torch.float64, device=dev)
        d = torch.cdist(r, A)                                   # (c, nat)
        mu = (d[:, :, None] - d[:, None, :]) * inv[None]        # (c, nat, nat)
        sv = _becke_s(mu)
        sv = torch.where(eye[None], torch.ones_like(sv), sv)
        Pc = torch.prod(sv, dim=2)                              # (c, nat)
        tot = Pc.sum(dim=1)
        mine = Pc.gather(1, own[s:s + chunk, None])[:, 0]
        out[s:s + chunk] = (mine / tot).cpu().numpy()
    return out


def make_grid(mol: Molecule, n_r: int, n_theta: int, n_phi: int,
              per_atom=None, device=None) -> Grid:
    """Atom-centred product grid with Becke partition weights.  `per_atom`
    optionally gives (n_r, n_theta, n_phi) for each atom."""
    xyzs, ws, owners = [], [], []
    for a in range(mol.xyz.shape[0]):
        nr, nt, npf = per_atom[a] if per_atom is not None else (n_r, n_theta, n_phi)
        r, wr = mk_radial(nr)
        dirs, wa = angular_product(nt, npf)
        pts = (r[:, None, None] * dirs[None, :, :]).reshape(-1, 3) + mol.xyz[a]
        w = (wr[:, None] * wa[None, :]).reshape(-1)
        xyzs.append(pts)
        ws.append(w)
        owners.append(np.full(w.shape[0], a, dtype=np.int32))
    xyz = np.concatenate(xyzs)
    w = np.concatenate(ws)
    owner = np.concatenate(owners)
    w = w * becke_weights(xyz, owner, mol.xyz, device=device)
    return Grid(xyz=np.ascontiguousarray(xyz), w=w, atom=owner)


# --------------------------------------------------------------------------
# density
# --------------------------------------------------------------------------

def function_centers(basis: Basis) -> np.ndarray:
    out = []
    for s in range(basis.n_shells):
        n = (int(basis.l[s]) + 1) * (int(basis.l[s]) + 2) // 2
        out.extend([basis.center[s]] * n)
    return np.array(out).reshape(-1, 3)


def make_density(mol: Molecule, basis: Basis, n_occ: int, seed: int,
                 sigma: float | None = 3.0) -> np.ndarray:
    """P = C C^T, C = Loewdin-orthonormalised (Euclidean metric) N(0,1)
    columns, each optionally multiplied by a Gaussian envelope of width sigma
    (bohr) around a seeded centre atom."""
    rng = np.random.default_rng(seed + 104729)
    nb = basis.n_functions
    C = rng.normal(size=(nb, n_occ))
    if sigma is not None:
        fc = function_centers(basis)
        centres = rng.integers(0, mol.xyz.shape[0], size=n_occ)
        d2 = np.sum((fc[:, None, :] - mol.xyz[centres][None, :, :]) ** 2, axis=-1)
        C *= np.exp(-d2 / (2.0 * sigma * sigma))
    S = C.T @ C
    ev, U = np.linalg.eigh(S)
    C = C @ (U * (1.0 / np.sqrt(ev))) @ U.T
    P = C @ C.T
    return 0.5 * (P + P.T)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def chain4(seed: int = 101, n_r: int = 40, n_theta: int = 5, n_phi: int = 15) -> Problem:
    """4-atom H-O-O-H, 34 functions, 40 x (5 x 15) points per atom."""
    mol = make_chain_molecule(seed)
    basis = make_basis(mol, "small", seed)
    grid = make_grid(mol, n_r, n_theta, n_phi)
    P = make_density(mol, basis, 5, seed, sigma=None)
    return Problem("chain4", mol, basis, grid, P, dict(seed=seed))


def cluster(n_atoms: int, seed: int, n_r: int = 50, n_theta: int = 8, n_phi: int = 20,
            occ_frac: float = 0.2, n_occ: int | None = None, device=None,
            recipe: str = "scale", per_atom=None) -> Problem:
    """Globular cluster of n_atoms (1:2 heavy:light), scale basis, product grid,
    localised density with n_occ = ceil(occ_frac * N_b) unless given."""
    mol = make_cluster_molecule(n_atoms, seed)
    basis = make_basis(mol, recipe, seed)
    grid = make_grid(mol, n_r, n_theta, n_phi, per_atom=per_atom, device=device)
    nb = basis.n_functions
    if n_occ is None:
        n_occ = int(math.ceil(occ_frac * nb))
    P = make_density(mol, basis, n_occ, seed)
    return Problem(f"cluster{n_atoms}", mol, basis, grid, P,
                   dict(seed=seed, n_occ=n_occ, n_r=n_r, n_theta=n_theta, n_phi=n_phi))


def cluster96(device=None) -> Problem:
    """96 atoms (32 O-like, 64 H-like), 992 functions, 50 x (8 x 20) = 8,000
    points per atom (768,000 total), 200 occupied columns."""
    return cluster(96, 102, n_occ=200, device=device)


def cluster24(device=None) -> Problem:
    """24 atoms (8 O-like, 16 H-like), 248 functions, 192,000 points: a small
    case of the 96-atom workload's shape for kernel profiles."""
    return cluster(24, 124, device=device)


def cluster256(device=None) -> Problem:
    return cluster(256, 103, device=device)


def cluster512(device=None) -> Problem:
    return cluster(512, 105, device=device)


def small_molecule(m: int, device=None) -> Problem:
    """Molecule m of a batch of small molecules: 4..12 atoms, 40 radial x
    (5 x 15) angular points per atom, drawn from seed 5000 + m."""
    seed = 5000 + m
    rng = np.random.default_rng(seed)
    n_atoms = int(rng.integers(4, 13))
    return cluster(n_atoms, seed, n_r=40, n_theta=5, n_phi=15, device=device)


def multi_molecule(m: int, device=None) -> Problem:
    """Molecule m of the 64-molecule batch: 6..60 atoms, N_r in {40, 50},
    angular rule in {5x15, 8x15, 8x20}, all drawn from seed 2000 + m."""
    seed = 2000 + m
    rng = np.random.default_rng(seed)
    n_atoms = int(rng.integers(6, 61))
    n_r = int(rng.choice([40, 50]))
    nt, npf = [(5, 15), (8, 15), (8, 20)][int(rng.integers(0, 3))]
    return cluster(n_atoms, seed, n_r=n_r, n_theta=nt, n_phi=npf, device=device)

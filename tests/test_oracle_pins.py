"""Pins of the FP64 CPU oracle against closed forms, independent routes,
invariants and brute force (no GPU).

Each test fixes the oracle to something other than itself, chosen so that a
plausible mistake (a dropped term, a wrong sign or index, a transposed
operand, a lost weight or normalisation) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


# ---------------------------------------------------------------- Boys, Eq. (boys)

def test_boys_at_zero():
    """F_n(0) = 1/(2n+1)."""
    F = oracle.boys(12, 0.0)
    np.testing.assert_allclose(F, [1.0 / (2 * n + 1) for n in range(13)], rtol=1e-15)


@pytest.mark.parametrize("T", [1e-8, 0.3, 1.7, 6.0, 14.5, 29.9, 30.0, 45.0, 120.0])
def test_boys_F0_erf(T):
    """F_0(T) = sqrt(pi/T) erf(sqrt(T)) / 2, on both branches of the oracle."""
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(oracle.boys(0, T)[0] - ref) <= 1e-14 * ref


@pytest.mark.parametrize("T", [60.0, 200.0, 1000.0])
def test_boys_large_T_asymptote(T):
    """F_n(T) -> (2n-1)!! / 2^{n+1} sqrt(pi / T^{2n+1}) for large T."""
    F = oracle.boys(8, T)
    for n in range(9):
        ref = _dfact(2 * n - 1) / 2 ** (n + 1) * math.sqrt(math.pi / T ** (2 * n + 1))
        assert abs(F[n] - ref) <= 1e-12 * ref


def test_boys_gauss_legendre_of_definition():
    """Eq. (boys) integrated by 400-node Gauss-Legendre quadrature."""
    x, wx = np.polynomial.legendre.leggauss(400)
    y = 0.5 * (x + 1.0)
    wy = 0.5 * wx
    rng = np.random.default_rng(1)
    for T in np.concatenate([rng.uniform(0, 35, 40), [0.05, 29.99, 30.01]]):
        F = oracle.boys(10, T)
        for n in range(11):
            ref = np.sum(wy * y ** (2 * n) * np.exp(-T * y * y))
            assert abs(F[n] - ref) <= 5e-13 * ref   # numpy quadrature sums to ~2e-13


def test_boys_downward_recursion():
    """F_n = (2T F_{n+1} + e^{-T}) / (2n+1) holds for every n and both branches."""
    for T in [0.01, 2.0, 11.0, 29.5, 30.5, 50.0]:
        F = oracle.boys(9, T)
        for n in range(9):
            rhs = (2 * T * F[n + 1] + math.exp(-T)) / (2 * n + 1)
            assert abs(F[n] - rhs) <= 1e-13 * F[n]


def test_boys_incomplete_gamma_mpmath():
    """F_n(T) = gamma(n + 1/2, T) / (2 T^{n+1/2}) at 30 digits."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for T in [0.2, 3.0, 17.0, 29.0, 33.0, 80.0]:
        F = oracle.boys(8, T)
        for n in range(9):
            ref = float(mpmath.gammainc(n + 0.5, 0, T) / (2 * mpmath.mpf(T) ** (n + 0.5)))
            assert abs(F[n] - ref) <= 5e-15 * ref


# ---------------------------------------------------------------- 3c-CP, Eq. (3c_grid)

def test_ss_potential_closed_form():
    """Raw s-s primitive: A = (pi/z)^{3/2} K_ab erf(sqrt(z) R)/R, 2 pi K_ab / z at R = 0."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        A, B = rng.normal(size=3), rng.normal(size=3)
        a, b = rng.uniform(0.05, 20), rng.uniform(0.05, 20)
        z = a + b
        P = (a * A + b * B) / z
        K = math.exp(-a * b / z * np.sum((A - B) ** 2))
        C = P + rng.normal(size=3) * rng.choice([1e-3, 0.3, 3.0, 30.0])
        R = np.linalg.norm(P - C)
        ref = (math.pi / z) ** 1.5 * K * math.erf(math.sqrt(z) * R) / R
        got = oracle.prim_A(0, 0, A, a, B, b, C)[0, 0]
        assert abs(got - ref) <= 1e-13 * ref
    got = oracle.prim_A(0, 0, A, a, B, b, P)[0, 0]
    assert abs(got - 2 * math.pi * K / z) <= 1e-14 * got


@pytest.mark.parametrize("la", [0, 1, 2])
@pytest.mark.parametrize("lb", [0, 1, 2])
def test_obara_saika_equals_mcmurchie_davidson(la, lb):
    """App. A (VRR + HRR) and Sec. II.B (Hermite E and R) give the same A."""
    rng = np.random.default_rng(10 * la + lb)
    for _ in range(30):
        A, B = rng.normal(size=3), rng.normal(size=3) * 1.5
        C = rng.normal(size=3) * rng.choice([0.1, 1.0, 4.0])
        a, b = rng.uniform(0.1, 30), rng.uniform(0.1, 30)
        x = oracle.prim_A(la, lb, A, a, B, b, C, "os")
        y = oracle.prim_A(la, lb, A, a, B, b, C, "md")
        assert np.max(np.abs(x - y)) <= 1e-13 * np.max(np.abs(y))


def test_contracted_os_md_and_symmetry(chain4):
    """Contracted, normalised shell pairs: OS == MD, and A_{mu lambda} = A_{lambda mu}."""
    basis = chain4.basis
    rng = np.random.default_rng(3)
    for sa in range(basis.n_shells):
        for sb in range(basis.n_shells):
            C = chain4.mol.xyz[rng.integers(0, 4)] + rng.normal(size=3)
            x = oracle.shell_A(basis, sa, sb, C, "os")
            y = oracle.shell_A(basis, sa, sb, C, "md")
            z = oracle.shell_A(basis, sb, sa, C, "os")
            s = np.max(np.abs(y))
            assert np.max(np.abs(x - y)) <= 1e-13 * s
            assert np.max(np.abs(x - z.T)) <= 1e-13 * s


# ---------------------------------------------------------------- normalisation, collocation

def _overlap_gh(basis, d, f):
    """Analytic overlap matrix of the normalised contracted Cartesian functions,
    each 1D factor by Gauss-Hermite quadrature (exact for these polynomials)."""
    t, wt = np.polynomial.hermite.hermgauss(12)
    comps = {l: [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]
             for l in range(3)}
    poff = np.concatenate([[0], np.cumsum(basis.nprim)])
    funcs = []
    for s in range(basis.n_shells):
        for c in comps[int(basis.l[s])]:
            funcs.append((s, c))
    nf = len(funcs)
    S = np.zeros((nf, nf))
    for i, (sa, ca) in enumerate(funcs):
        for j, (sb, cb) in enumerate(funcs):
            A, B = basis.center[sa], basis.center[sb]
            tot = 0.0
            for k in range(poff[sa], poff[sa + 1]):
                for m in range(poff[sb], poff[sb + 1]):
                    a, b = basis.exps[k], basis.exps[m]
                    p = a + b
                    P = (a * A + b * B) / p
                    val = d[k] * d[m]
                    for q in range(3):
                        x = P[q] + t / math.sqrt(p)
                        Kq = math.exp(-a * b / p * (A[q] - B[q]) ** 2)
                        val *= Kq * np.sum(wt * (x - A[q]) ** ca[q] * (x - B[q]) ** cb[q]) / math.sqrt(p)
                    tot += val
            S[i, j] = tot * f[i] * f[j]
    return S


def test_normalised_functions_have_unit_norm(chain4):
    d, f = oracle.normalise(chain4.basis)
    S = _overlap_gh(chain4.basis, d, f)
    np.testing.assert_allclose(np.diag(S), 1.0, rtol=1e-13)


def test_collocation_overlap_on_fine_grid():
    """sum_i w_i Phi_mu Phi_nu -> S_mu nu on a fine grid (grid and normalisation sanity)."""
    mol = synth.Molecule(Z=np.array([8, 1], dtype=np.int32), xyz=np.array([[0, 0, 0], [0, 0.9, 1.1]]))
    basis = synth.make_basis(mol, "small", 5)
    keep = [0, 1, 3, 5, 6, 7]                     # drop the tightest s and p shells
    basis = _subset_shells(basis, keep)
    grid = synth.make_grid(mol, 80, 16, 32)
    d, f = oracle.normalise(basis)
    S = _overlap_gh(basis, d, f)
    Phi = oracle.collocation(basis, grid.xyz)
    Sg = (Phi * grid.w[:, None]).T @ Phi
    assert np.max(np.abs(Sg - S)) <= 1e-6


def _subset_shells(basis, keep):
    poff = np.concatenate([[0], np.cumsum(basis.nprim)])
    pidx = np.concatenate([np.arange(poff[s], poff[s + 1]) for s in keep])
    return synth.Basis(l=basis.l[keep], nprim=basis.nprim[keep], atom=basis.atom[keep],
                       center=basis.center[keep], exps=basis.exps[pidx], coefs=basis.coefs[pidx])


# ---------------------------------------------------------------- ERIs, Eq. (full_k)

def test_eri_ssss_closed_form():
    rng = np.random.default_rng(4)
    for _ in range(20):
        cs = [rng.normal(size=3) for _ in range(4)]
        es = rng.uniform(0.1, 10, 4)
        p, q = es[0] + es[1], es[2] + es[3]
        P = (es[0] * cs[0] + es[1] * cs[1]) / p
        Q = (es[2] * cs[2] + es[3] * cs[3]) / q
        Kab = math.exp(-es[0] * es[1] / p * np.sum((cs[0] - cs[1]) ** 2))
        Kcd = math.exp(-es[2] * es[3] / q * np.sum((cs[2] - cs[3]) ** 2))
        rho = p * q / (p + q)
        T = rho * np.sum((P - Q) ** 2)
        ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * oracle.boys(0, T)[0]
        got = oracle.prim_eri([0, 0, 0, 0], cs, es)[0, 0, 0, 0]
        assert abs(got - ref) <= 1e-13 * ref


def test_eri_eightfold_symmetry():
    rng = np.random.default_rng(5)
    ls = [2, 1, 2, 0]
    cs = [rng.normal(size=3) for _ in range(4)]
    es = rng.uniform(0.2, 5, 4)
    x = oracle.prim_eri(ls, cs, es)
    y = oracle.prim_eri([ls[1], ls[0], ls[2], ls[3]], [cs[1], cs[0], cs[2], cs[3]], [es[1], es[0], es[2], es[3]])
    z = oracle.prim_eri([ls[2], ls[3], ls[0], ls[1]], [cs[2], cs[3], cs[0], cs[1]], [es[2], es[3], es[0], es[1]])
    s = np.max(np.abs(x))
    assert np.max(np.abs(x - y.transpose(1, 0, 2, 3))) <= 1e-13 * s
    assert np.max(np.abs(x - z.transpose(2, 3, 0, 1))) <= 1e-13 * s


def test_eri_limit_is_potential_of_point_charge():
    """(ab|cc) with a very tight normalised s charge at C equals A_ab(C)."""
    rng = np.random.default_rng(6)
    A, B, C = rng.normal(size=3), rng.normal(size=3), rng.normal(size=3)
    g = 1e9
    norm = (g / math.pi) ** 1.5          # int exp(-g r^2) = (pi/g)^{3/2}
    for la in range(3):
        for lb in range(3):
            e = oracle.prim_eri([la, lb, 0, 0], [A, B, C, C], [0.8, 1.1, g / 2, g / 2])[:, :, 0, 0] * norm
            a = oracle.prim_A(la, lb, A, 0.8, B, 1.1, C)
            assert np.max(np.abs(e - a)) <= 1e-7 * np.max(np.abs(a))


# ---------------------------------------------------------------- sn-K, Eqs. (gmat)-(sn_k)

def _single_s_basis(alpha):
    return synth.Basis(l=np.array([0], dtype=np.int32), nprim=np.array([1], dtype=np.int32),
                       atom=np.array([0], dtype=np.int32), center=np.zeros((1, 3)),
                       exps=np.array([alpha]), coefs=np.array([1.0]))


def test_self_exchange_single_gaussian():
    """One normalised s Gaussian, P = [[1]]: exact K = (phi phi|phi phi) = 2 sqrt(alpha/pi).
    The sn-K quadrature equals sum_i w_i erf(sqrt(2 alpha) r_i)/r_i phi(r_i)^2 at any
    grid and converges to the exact value as the grid is refined."""
    from scipy.special import erf
    alpha = 0.7
    basis = _single_s_basis(alpha)
    mol = synth.Molecule(Z=np.array([8], dtype=np.int32), xyz=np.zeros((1, 3)))
    exact = 2 * math.sqrt(alpha / math.pi)
    assert abs(oracle.eri_K(basis, np.ones((1, 1)))[0, 0] - exact) <= 1e-14
    errs = []
    for nr in (10, 20, 40, 80):
        grid = synth.make_grid(mol, nr, 4, 8)
        K = oracle.snk_K(basis, grid, np.ones((1, 1)))[0, 0]
        r = np.linalg.norm(grid.xyz, axis=1)
        phi2 = (2 * alpha / math.pi) ** 1.5 * np.exp(-2 * alpha * r * r)
        quad = np.sum(grid.w * erf(math.sqrt(2 * alpha) * r) / r * phi2)
        assert abs(K - quad) <= 1e-13 * quad
        errs.append(abs(K - exact))
    assert errs[-1] < 1e-9 and errs[-1] < errs[0]


def test_snk_symmetric_linear_positive(chain4):
    b, g = chain4.basis, chain4.grid
    rng = np.random.default_rng(7)
    nb = b.n_functions
    X = rng.normal(size=(nb, nb))
    P2 = 0.5 * (X + X.T) * 0.1
    K1 = oracle.snk_K(b, g, chain4.P)
    K2 = oracle.snk_K(b, g, P2)
    K12 = oracle.snk_K(b, g, chain4.P + P2)
    assert np.max(np.abs(K1 - K1.T)) == 0.0
    s = np.max(np.abs(K12))
    assert np.max(np.abs(K12 - K1 - K2)) <= 1e-13 * s
    assert np.trace(K1 @ chain4.P) > 0


def _permute_problem(p, perm_atoms):
    b = p.basis
    shells = np.concatenate([np.nonzero(b.atom == a)[0] for a in perm_atoms])
    poff = np.concatenate([[0], np.cumsum(b.nprim)])
    foff = np.concatenate([[0], np.cumsum([(l + 1) * (l + 2) // 2 for l in b.l])])
    pidx = np.concatenate([np.arange(poff[s], poff[s + 1]) for s in shells])
    fidx = np.concatenate([np.arange(foff[s], foff[s + 1]) for s in shells])
    inv = np.argsort(perm_atoms)
    nb = synth.Basis(l=b.l[shells], nprim=b.nprim[shells], atom=inv[b.atom[shells]].astype(np.int32),
                     center=b.center[shells], exps=b.exps[pidx], coefs=b.coefs[pidx])
    pts = np.concatenate([np.nonzero(p.grid.atom == a)[0] for a in perm_atoms])
    ng = synth.Grid(xyz=p.grid.xyz[pts], w=p.grid.w[pts], atom=inv[p.grid.atom[pts]].astype(np.int32))
    return nb, ng, p.P[np.ix_(fidx, fidx)], fidx


def test_atom_relabelling_permutes_K(chain4):
    K = oracle.snk_K(chain4.basis, chain4.grid, chain4.P)
    b, g, P, fidx = _permute_problem(chain4, np.array([2, 0, 3, 1]))
    Kp = oracle.snk_K(b, g, P)
    assert np.max(np.abs(Kp - K[np.ix_(fidx, fidx)])) <= 1e-12


def test_rigid_translation_leaves_K(chain4):
    K = oracle.snk_K(chain4.basis, chain4.grid, chain4.P)
    t = np.array([3.1, -1.7, 0.4])
    b = chain4.basis
    bt = synth.Basis(l=b.l, nprim=b.nprim, atom=b.atom, center=b.center + t, exps=b.exps, coefs=b.coefs)
    gt = synth.Grid(xyz=chain4.grid.xyz + t, w=chain4.grid.w, atom=chain4.grid.atom)
    Kt = oracle.snk_K(bt, gt, chain4.P)
    assert np.max(np.abs(Kt - K)) <= 1e-12


def test_entries_mode_matches_full_build(chain4):
    K = oracle.snk_K(chain4.basis, chain4.grid, chain4.P)
    rng = np.random.default_rng(8)
    mu = rng.integers(0, 34, 20)
    nu = rng.integers(0, 34, 20)
    e = oracle.snk_K_entries(chain4.basis, chain4.grid, chain4.P, mu, nu)
    assert np.max(np.abs(e - K[mu, nu])) <= 1e-14 * np.max(np.abs(K))


@pytest.mark.slow
def test_blocked_entries_mode_matches_full_build(chain4):
    """The blocked entries mode (F = Phi P as a library matrix product per
    block of points, the wanted G rows by the oracle) reproduces the full
    build's entries, across blocks of ragged size."""
    p = chain4
    K = oracle.snk_K(p.basis, p.grid, p.P)
    mu = np.array([0, 3, 10, 33, 17, 5, 20])
    nu = np.array([0, 7, 2, 33, 30, 5, 11])
    vals = oracle.snk_K_entries_blocked(p.basis, p.grid, p.P, mu, nu, block=997)
    assert np.max(np.abs(vals - K[mu, nu])) <= 1e-15 * max(1.0, np.max(np.abs(K)))


def test_becke_partition_c_matches_tensor_form():
    """The fused C Becke partition of synth (CPU grids) agrees with the tensor
    form of the same definition, and the cell weights of each point sum to 1."""
    import torch  # noqa: F401  (the tensor form runs as torch operations)
    mol = synth.make_cluster_molecule(24, 124)
    r, _ = synth.mk_radial(20)
    dirs, _ = synth.angular_product(4, 9)
    xyz = np.concatenate([(r[:, None, None] * dirs[None]).reshape(-1, 3) + mol.xyz[a] for a in range(24)])
    own = np.repeat(np.arange(24, dtype=np.int32), r.shape[0] * dirs.shape[0])
    sel = np.random.default_rng(0).choice(xyz.shape[0], 3000, replace=False)
    wc = synth.becke_weights(xyz[sel], own[sel], mol.xyz)
    wt = synth.becke_weights(xyz[sel], own[sel], mol.xyz, device="cpu")
    assert np.max(np.abs(wc - wt)) <= 1e-13
    # partition of unity: the weights of one point for every atom add to 1
    pts = xyz[sel[:50]]
    tot = sum(synth.becke_weights(pts, np.full(50, a, dtype=np.int32), mol.xyz) for a in range(24))
    assert np.max(np.abs(tot - 1.0)) <= 1e-12


def test_grid_refinement_converges_to_eri_K():
    """Brute force: sn-K approaches the four-centre-ERI exchange as the grid is refined
    (two atoms, s/p/d shells, two occupied orbitals)."""
    mol = synth.Molecule(Z=np.array([8, 1], dtype=np.int32), xyz=np.array([[0, 0, 0], [0.3, 0.8, 1.2]]))
    basis = synth.make_basis(mol, "scale", 9)
    basis = _subset_shells(basis, [0, 1, 3, 5, 7, 9])     # O: s s p d ; H: s p
    P = synth.make_density(mol, basis, 2, 9, sigma=None)
    Kx = oracle.eri_K(basis, P)
    errs = []
    for (nr, nt, npf) in [(20, 6, 12), (40, 12, 24), (80, 20, 40)]:
        grid = synth.make_grid(mol, nr, nt, npf)
        errs.append(np.max(np.abs(oracle.snk_K(basis, grid, P) - Kx)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 1e-6, errs

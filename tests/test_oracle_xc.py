"""Pins of the oracle's exchange-correlation potential (Sec. II.C: Eqs.
collocation, fmat, den_grid, exc_grid, zmat, vxc_num) against published
values, closed forms, limits and finite differences (no GPU).

A plausible mistake fails at least one of them: a wrong constant or power in
a functional (published H-atom exchange energies, the PW92 limits, the PBE
gradient coefficients), a wrong derivative (finite differences of eps), a
wrong factor in Z or in grad rho (finite differences of E_xc in P, the
homogeneity identity of Slater exchange), a wrong gradient of Phi (finite
differences of the collocation).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
import synth

LDA_X, PBE_X, PBE = oracle.XC_LDA_X, oracle.XC_PBE_X, oracle.XC_PBE
CX = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0)      # Slater's exchange constant
BETA = 0.06672455060314922                       # PBE's gradient coefficient of correlation
MU = BETA * math.pi ** 2 / 3.0                   # PBE's gradient coefficient of exchange


def _sigma(rho, s):
    """sigma = |grad rho|^2 at reduced gradient s = |grad rho| / (2 (3 pi^2)^{1/3} rho^{4/3})."""
    return (2.0 * (3.0 * math.pi ** 2) ** (1.0 / 3.0) * rho ** (4.0 / 3.0) * s) ** 2


@pytest.mark.parametrize("fun", [LDA_X, PBE_X, PBE])
def test_derivatives_match_finite_differences(fun):
    """d eps / d rho and d eps / d sigma against central differences of eps."""
    for rho in (1e-5, 1e-3, 0.05, 0.7, 8.0, 150.0):
        for s in (0.0, 0.2, 0.9, 2.5, 6.0):
            sig = _sigma(rho, s)
            e, er, es = oracle.xc_point(fun, rho, sig)
            h = 1e-5 * rho
            fd_r = (oracle.xc_point(fun, rho + h, sig)[0] - oracle.xc_point(fun, rho - h, sig)[0]) / (2 * h)
            assert abs(er - fd_r) <= 2e-8 * max(abs(er), abs(e) / rho), (rho, s)
            if fun != LDA_X and sig > 0:
                hs = 1e-5 * sig
                fd_s = (oracle.xc_point(fun, rho, sig + hs)[0] - oracle.xc_point(fun, rho, sig - hs)[0]) / (2 * hs)
                assert abs(es - fd_s) <= 2e-8 * max(abs(es), abs(e) / sig), (rho, s)
            if fun == LDA_X:
                assert es == 0.0


def test_slater_exchange_closed_form():
    """Slater: eps = C_x rho^{4/3}; PBE exchange reduces to it at zero gradient (F_x(0) = 1)."""
    for rho in (1e-6, 0.01, 1.0, 42.0):
        e = oracle.xc_point(LDA_X, rho, 0.0)
        assert abs(e[0] - CX * rho ** (4 / 3)) <= 4e-15 * abs(e[0])
        assert abs(e[1] - 4 / 3 * CX * rho ** (1 / 3)) <= 4e-15 * abs(e[1])
        assert oracle.xc_point(PBE_X, rho, 0.0)[0] == e[0]


def _h_atom_exchange(fun):
    """Exchange energy of the hydrogen atom's exact density e^{-2r}/pi, fully
    spin-polarised, from the spin-restricted functional by spin scaling:
    E_x[rho_up, 0] = E_x[2 rho_up] / 2."""
    def f(r):
        rho = math.exp(-2 * r) / math.pi
        e = oracle.xc_point(fun, 2 * rho, (2 * 2 * rho) ** 2)[0]   # |grad 2 rho| = 4 rho
        return 4 * math.pi * r * r * 0.5 * e
    return quad(f, 0, 60, limit=400, epsabs=1e-13)[0]


def test_hydrogen_atom_exchange_energies():
    """Published exchange energies of the H atom (exact density): LSD -0.268
    (here in closed form: -(81/128) (3/4)^{1/3} pi^{-2/3}) and PBE -0.306."""
    lsd = -(81.0 / 128.0) * 0.75 ** (1 / 3) * math.pi ** (-2 / 3)
    assert abs(lsd + 0.268) < 5e-4
    assert abs(_h_atom_exchange(LDA_X) - lsd) < 1e-10
    assert abs(_h_atom_exchange(PBE_X) + 0.306) < 5e-4


def _ec(rho, sigma=0.0):
    """correlation energy per electron of functional 3 (exchange taken off)"""
    return (oracle.xc_point(PBE, rho, sigma)[0] - oracle.xc_point(PBE_X, rho, sigma)[0]) / rho


def test_pw92_limits():
    """PW92's high-density limit e_c -> a ln r_s - c_1 with c_1 = 0.046644 and
    low-density limit r_s e_c -> -d_0 with d_0 = 0.4335 (the constants of the
    PW92 fit), taken at zero gradient where PBE's H vanishes."""
    a = 0.031091
    for rs in (1e-8, 1e-7):
        rho = 3.0 / (4.0 * math.pi * rs ** 3)
        assert abs(_ec(rho) - (a * math.log(rs) - 0.046644)) < 5e-6
    # r_s e_c = -d_0 + c / sqrt(r_s) + ...: Richardson on r_s = 2500, 10^4
    f = [rs * _ec(3.0 / (4.0 * math.pi * rs ** 3)) for rs in (1e4, 2500.0)]
    assert abs((2 * f[0] - f[1]) + 0.4335) < 2e-3


def test_pbe_gradient_limits():
    """PBE: exchange enhancement F_x -> 1 + mu s^2 at small s (mu = beta pi^2/3
    = 0.21951) and -> 1 + kappa = 1.804 at large s; correlation H -> beta t^2
    at small t (beta = 0.066725) and e_c + H -> 0 at large t."""
    rho = 0.3
    lda = oracle.xc_point(LDA_X, rho, 0.0)[0]
    for s in (1e-3, 3e-3):
        Fx = oracle.xc_point(PBE_X, rho, _sigma(rho, s))[0] / lda
        assert abs((Fx - 1) / s ** 2 - 0.21951) < 1e-4
    assert abs(oracle.xc_point(PBE_X, rho, _sigma(rho, 1e5))[0] / lda - 1.804) < 1e-6
    kF = (3 * math.pi ** 2 * rho) ** (1 / 3)
    ks = math.sqrt(4 * kF / math.pi)
    ec0 = _ec(rho)
    for t in (1e-3, 2e-3):
        sig = (2 * ks * rho * t) ** 2
        assert abs((_ec(rho, sig) - ec0) / t ** 2 - 0.066725) < 1e-4
    sig = (2 * ks * rho * 1e4) ** 2
    assert abs(_ec(rho, sig)) < 1e-9 * abs(ec0)


def test_collocation_gradient_matches_finite_differences(chain4):
    b = chain4.basis
    rng = np.random.default_rng(3)
    pts = chain4.mol.xyz[rng.integers(0, 4, 20)] + rng.normal(scale=0.8, size=(20, 3))
    phi, g = oracle.collocation_grad(b, pts)
    np.testing.assert_allclose(phi, oracle.collocation(b, pts), rtol=1e-14, atol=1e-300)
    h = 1e-4
    for q in range(3):
        e = np.zeros(3)
        e[q] = h
        fd = (-oracle.collocation(b, pts + 2 * e) + 8 * oracle.collocation(b, pts + e)
              - 8 * oracle.collocation(b, pts - e) + oracle.collocation(b, pts - 2 * e)) / (12 * h)
        assert np.max(np.abs(g[:, q, :] - fd)) <= 1e-9 * max(1.0, np.max(np.abs(fd)))


def _subgrid(grid, k):
    return synth.Grid(xyz=np.ascontiguousarray(grid.xyz[::k]), w=np.ascontiguousarray(grid.w[::k]),
                      atom=np.ascontiguousarray(grid.atom[::k]))


@pytest.mark.parametrize("fun", [LDA_X, PBE_X, PBE])
def test_vxc_is_the_derivative_of_exc(chain4, fun):
    """V^xc = dE_xc/dP (Eqs. zmat, vxc_num): for a symmetric perturbation S,
    (E(P + hS) - E(P - hS)) / 2h = sum V_{mu nu} S_{mu nu}; V symmetric."""
    b, g = chain4.basis, _subgrid(chain4.grid, 7)
    P = chain4.P
    V, E = oracle.vxc(b, g, P, fun)
    assert np.array_equal(V, V.T)
    rng = np.random.default_rng(11)
    for _ in range(3):
        X = rng.normal(size=P.shape)
        S = 0.5 * (X + X.T)
        h = 1e-5
        fd = (oracle.vxc(b, g, P + h * S, fun)[1] - oracle.vxc(b, g, P - h * S, fun)[1]) / (2 * h)
        an = float(np.sum(V * S))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3)


def test_slater_homogeneity(chain4):
    """Slater exchange is homogeneous of degree 4/3 in rho, so on any grid
    E_x[lambda P] = lambda^{4/3} E_x[P] and tr(V P) = 4/3 E_x."""
    b, g = chain4.basis, _subgrid(chain4.grid, 5)
    V, E = oracle.vxc(b, g, chain4.P, LDA_X)
    assert abs(np.sum(V * chain4.P) - 4 / 3 * E) <= 1e-12 * abs(E)
    E2 = oracle.vxc(b, g, 2.0 * chain4.P, LDA_X)[1]
    assert abs(E2 - 2 ** (4 / 3) * E) <= 1e-12 * abs(E)


def test_single_gaussian_slater_energy():
    """One normalised s Gaussian (exponent alpha), P = [[1]]: rho = (2 alpha/pi)^{3/2}
    e^{-2 alpha r^2}, so E_x = C_x (2 alpha/pi)^2 (3 pi / (8 alpha))^{3/2}; the
    quadrature converges to it."""
    alpha = 0.9
    basis = synth.Basis(l=np.array([0], dtype=np.int32), nprim=np.array([1], dtype=np.int32),
                        atom=np.array([0], dtype=np.int32), center=np.zeros((1, 3)),
                        exps=np.array([alpha]), coefs=np.array([1.0]))
    mol = synth.Molecule(Z=np.array([8], dtype=np.int32), xyz=np.zeros((1, 3)))
    exact = CX * (2 * alpha / math.pi) ** 2 * (3 * math.pi / (8 * alpha)) ** 1.5
    errs = []
    for nr in (10, 40, 120):
        grid = synth.make_grid(mol, nr, 4, 8)
        V, E = oracle.vxc(basis, grid, np.ones((1, 1)), LDA_X)
        errs.append(abs(E - exact))
        assert abs(V[0, 0] - 4 / 3 * E) <= 1e-13 * abs(E)     # tr(V P) = 4/3 E with P = [[1]]
    assert errs[-1] < 1e-9 * abs(exact) and errs[-1] < errs[0]


def test_vxc_entries_mode_matches_full(chain4):
    """The entries mode accumulates the same sums as the full V."""
    b, g = chain4.basis, _subgrid(chain4.grid, 3)
    V, E = oracle.vxc(b, g, chain4.P, PBE)
    rng = np.random.default_rng(2)
    mu = rng.integers(0, V.shape[0], 40)
    nu = rng.integers(0, V.shape[0], 40)
    Ve, Ee = oracle.vxc_entries(b, g, chain4.P, PBE, mu, nu)
    np.testing.assert_allclose(Ve, V[mu, nu], rtol=1e-13, atol=1e-15)
    assert abs(Ee - E) <= 1e-13 * abs(E)


def test_vxc_rejects_bad_arguments(chain4):
    """An unknown functional or an entry outside the basis is refused, not read out of bounds."""
    b, g = chain4.basis, _subgrid(chain4.grid, 50)
    with pytest.raises(ValueError):
        oracle.vxc(b, g, chain4.P, 7)
    with pytest.raises(ValueError):
        oracle.vxc_entries(b, g, chain4.P, PBE, [0, 34], [0, 0])
    with pytest.raises(ValueError):
        oracle.xc_point(0, 1.0, 0.0)
    assert np.all(oracle.xc_point(PBE, 1e-15, 1.0) == 0.0)    # below the density cut-off

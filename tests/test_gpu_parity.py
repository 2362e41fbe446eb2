"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerance: max|dK| <= 1e-10 Eh (the accuracy target of the plain FP64 build);
unit checks of the Boys function and of the 3c-CP blocks use relative bounds
derived from the device Boys interpolation (8-term Taylor, |dT| <= 0.05:
truncation ~1e-15 relative) and FP64 rounding of the recursions.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_K = 1e-10


@pytest.fixture(scope="module")
def snk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_14280_gb300 as m
    m.lib()
    return m


def test_boys_device_matches_oracle(snk):
    T = np.concatenate([np.linspace(0, 60, 6001), [1e-12, 0.05, 0.0499999, 49.95, 49.9999999, 50.0, 50.0000001,
                                                   75.0, 300.0, 1e4]])
    for nmax in range(5):
        d = snk.debug_boys(T, nmax)
        ref = np.array([oracle.boys(nmax, t) for t in T])
        rel = np.max(np.abs(d - ref) / ref)
        assert rel <= 2e-14, (nmax, rel)


@pytest.mark.parametrize("recipe", ["small", "scale"])
def test_shell_blocks_match_oracle(snk, recipe):
    """Every class (ss ... dd), points at the pair centre (T = 0), near and far."""
    mol = synth.make_cluster_molecule(6, 31)
    basis = synth.make_basis(mol, recipe, 31)
    grid = synth.make_grid(mol, 6, 2, 4)
    eng = snk.Engine(basis, grid)
    rng = np.random.default_rng(5)
    seen = set()
    for sa in range(basis.n_shells):
        for sb in range(basis.n_shells):
            cls = (max(basis.l[sa], basis.l[sb]), min(basis.l[sa], basis.l[sb]))
            if (cls, sa == sb) in seen and rng.random() > 0.15:
                continue
            seen.add((cls, sa == sb))
            mid = 0.5 * (basis.center[sa] + basis.center[sb])
            pts = np.concatenate([mid[None], basis.center[[sa]], mid + rng.normal(size=(6, 3)) * 0.7,
                                  mid + rng.normal(size=(4, 3)) * 6.0, mid + np.array([[40.0, 3.0, -2.0]])])
            dev = eng.debug_shell_A(sa, sb, pts)
            ref = np.stack([oracle.shell_A(basis, sa, sb, r) for r in pts])
            # relative 1e-12 per point plus an absolute 1e-14 of the pair's largest
            # value: blocks that vanish by symmetry (an s-p pair at its own centre)
            # are FP64 rounding of cancelling O(max) terms, ~1e-16 max on both sides
            # (primitive pairs whose rigorous bound is below 1e-20 are left out at
            # setup: at most 9 of them per pair here, so an absolute 1e-18 floor)
            tol = 1e-12 * np.max(np.abs(ref), axis=(1, 2), keepdims=True) + 1e-14 * np.max(np.abs(ref)) + 1e-18
            bad = np.abs(dev - ref) > tol
            if bad.any():
                i, u, v = np.argwhere(bad)[0]
                raise AssertionError(f"pair ({sa},{sb}) l=({basis.l[sa]},{basis.l[sb]}) point {i} {pts[i]} "
                                     f"comp ({u},{v}): dev {dev[i, u, v]!r} ref {ref[i, u, v]!r} tol {tol[i, 0, 0]:.3e} "
                                     f"pair max {np.max(np.abs(ref)):.3e} worst ratio {np.max(np.abs(dev - ref) / tol):.3e}")
    eng.close()


def _gpu_K(snk, p, P=None, **opts):
    eng = snk.Engine(p.basis, p.grid, **opts)
    eng.set_density(p.P if P is None else P)
    K = eng.build_K()
    st = eng.stats()
    eng.close()
    return K, st


def test_chain4_unscreened_matches_oracle(snk, chain4):
    Kref = oracle.snk_K(chain4.basis, chain4.grid, chain4.P)
    K, st = _gpu_K(snk, chain4, screen="none", eps_basis=0.0)
    assert st["pairs_kept"] == st["n_batches"] * st["n_pairs"]
    assert np.max(np.abs(K - Kref)) <= TOL_K
    assert np.max(np.abs(K - K.T)) == 0.0


def test_chain4_screened_matches_oracle(snk, chain4):
    Kref = oracle.snk_K(chain4.basis, chain4.grid, chain4.P)
    K, st = _gpu_K(snk, chain4)
    assert np.max(np.abs(K - Kref)) <= TOL_K


def test_many_ragged_batches_and_chunks(snk):
    """12-atom cluster, scale basis: small batches (ragged 128-point tails), several
    workspace chunks (Alg. 1 loop), screened and unscreened, against the full oracle."""
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    for opts in (dict(batch_max=300, workspace_bytes=6 << 20), dict(batch_max=4096, screen="none", eps_basis=0.0),
                 dict(batch_max=97, workspace_bytes=1 << 20)):
        K, st = _gpu_K(snk, p, **opts)
        assert st["n_batches"] >= 12
        assert np.max(np.abs(K - Kref)) <= TOL_K, opts
    assert st["n_chunks"] > 1


def test_linearity_in_the_density(snk, chain4):
    rng = np.random.default_rng(3)
    X = rng.normal(size=chain4.P.shape)
    P2 = 0.05 * (X + X.T)
    K1, _ = _gpu_K(snk, chain4, screen="none")
    K2, _ = _gpu_K(snk, chain4, P=P2, screen="none")
    K12, _ = _gpu_K(snk, chain4, P=chain4.P + P2, screen="none")
    assert np.max(np.abs(K12 - K1 - K2)) <= 1e-12


def test_device_resident_path_matches_host_path(snk, chain4):
    import torch
    eng = snk.Engine(chain4.basis, chain4.grid)
    eng.set_stream(torch.cuda.current_stream())
    eng.set_density(chain4.P)
    Kh = eng.build_K()
    Pd = torch.from_numpy(chain4.P).cuda()
    eng.set_density(Pd)
    Kd = torch.zeros_like(Pd)
    eng.build_K(out=Kd)
    torch.cuda.synchronize()
    assert np.max(np.abs(Kd.cpu().numpy() - Kh)) <= 1e-14
    eng.close()


def test_edge_cases(snk):
    # one atom, one s shell; batch_max = 1 makes every point its own batch
    basis = synth.Basis(l=np.array([0], dtype=np.int32), nprim=np.array([1], dtype=np.int32),
                        atom=np.array([0], dtype=np.int32), center=np.zeros((1, 3)),
                        exps=np.array([0.7]), coefs=np.array([1.0]))
    mol = synth.Molecule(Z=np.array([8], dtype=np.int32), xyz=np.zeros((1, 3)))
    grid = synth.make_grid(mol, 5, 2, 3)
    P = np.ones((1, 1))
    p = synth.Problem("one", mol, basis, grid, P)
    K, st = _gpu_K(snk, p, batch_max=1)
    assert st["n_batches"] == grid.n_points
    assert abs(K[0, 0] - oracle.snk_K(basis, grid, P)[0, 0]) <= 1e-13
    # empty grid: K = 0
    empty = synth.Grid(xyz=np.zeros((0, 3)), w=np.zeros(0), atom=np.zeros(0, dtype=np.int32))
    K, st = _gpu_K(snk, synth.Problem("e", mol, basis, empty, P))
    assert st["n_batches"] == 0 and K[0, 0] == 0.0


def test_errors_leave_the_handle_usable(snk, chain4):
    eng = snk.Engine(chain4.basis, chain4.grid)
    with pytest.raises(snk.SnkError) as e:
        eng.build_K()
    assert e.value.status == -4                      # build before set_density
    Pbad = chain4.P.copy()
    Pbad[0, 1] += 1e-6
    with pytest.raises(snk.SnkError) as e:
        eng.set_density(Pbad)
    assert e.value.status == -3
    Pnan = chain4.P.copy()
    Pnan[2, 2] = np.nan
    with pytest.raises(snk.SnkError):
        eng.set_density(Pnan)
    eng.set_density(chain4.P)                        # recovers
    K = eng.build_K()
    assert np.max(np.abs(K - oracle.snk_K(chain4.basis, chain4.grid, chain4.P))) <= TOL_K
    eng.close()


def test_distance_bound_and_global_bound_agree(snk):
    """The per-batch charge/distance refinement of A-tilde keeps parity and keeps
    no more pairs than the global bound of the paper."""
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    K0, s0 = _gpu_K(snk, p, batch_max=300, distance_bound=0)
    K1, s1 = _gpu_K(snk, p, batch_max=300, distance_bound=1)
    assert np.max(np.abs(K0 - Kref)) <= TOL_K
    assert np.max(np.abs(K1 - Kref)) <= TOL_K
    assert s1["pairs_kept"] <= s0["pairs_kept"]


def test_mixed_precision_form(snk):
    """Form 1: kept pairs whose sn-LinK estimate is below fp32_bound run their
    integrals in FP32 (FP32 Boys table, recursions and contraction); the result
    stays within 1e-7 of the FP64 build and of the oracle."""
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    K64, s64 = _gpu_K(snk, p, batch_max=300)
    Km, sm = _gpu_K(snk, p, batch_max=300, precision="mixed")
    assert sm["pairs_kept_fp32"] > 0
    assert sm["pairs_kept"] == s64["pairs_kept"]
    assert np.max(np.abs(Km - K64)) <= 1e-7
    assert np.max(np.abs(Km - Kref)) <= 1e-7
    assert np.max(np.abs(Km - Km.T)) == 0.0
    # a looser split (1e-3) stays within the 1e-8 target of the mixed form
    Kl, sl = _gpu_K(snk, p, batch_max=300, precision="mixed", fp32_bound=1e-3)
    assert sl["pairs_kept_fp32"] > sm["pairs_kept_fp32"]
    assert np.max(np.abs(Kl - Kref)) <= 1e-8
    # everything in FP32: still a sane exchange matrix, error well above FP64's
    Kf, sf = _gpu_K(snk, p, batch_max=300, precision="mixed", fp32_bound=1e300)
    assert sf["pairs_kept_fp32"] == sf["pairs_kept"]
    assert 1e-12 < np.max(np.abs(Kf - Kref)) <= 1e-5
    # tensor-core split products at their fewest slices (3 per operand, ~2^-22 of the run maxima)
    Kt, st = _gpu_K(snk, p, batch_max=300, precision="mixed", gemm="split", tc_slices_hi=3, tc_slices_lo=3)
    assert np.max(np.abs(Kt - Kref)) <= 1e-6
    assert np.max(np.abs(Kt - Kt.T)) == 0.0


def test_double_fp32_gemms(snk):
    """The double-FP32 GEMMs (hi + lo float pairs, TwoSum accumulation) keep
    the FP64 build's parity: with every pair in FP64 the only change from the
    plain build is the arithmetic of F = X P and Kt = G^T X (~2^-46 relative)."""
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    K64, _ = _gpu_K(snk, p, batch_max=300)
    Kd, sd = _gpu_K(snk, p, batch_max=300, precision="mixed", fp32_bound=0.0, gemm="df32")
    assert sd["pairs_kept_fp32"] == 0
    assert np.max(np.abs(Kd - Kref)) <= TOL_K
    assert np.max(np.abs(Kd - K64)) <= 1e-12
    assert np.max(np.abs(Kd - Kd.T)) == 0.0
    # ragged chunks: the in-place split covers each chunk's X and G exactly
    Kc, sc = _gpu_K(snk, p, batch_max=97, precision="mixed", fp32_bound=0.0, gemm="df32", workspace_bytes=1 << 20)
    assert sc["n_chunks"] > 1
    assert np.max(np.abs(Kc - Kref)) <= TOL_K
    # with the FP32 pairs of the mixed form
    Km, sm = _gpu_K(snk, p, batch_max=300, precision="mixed", fp32_bound=1e-3, gemm="df32")
    assert sm["pairs_kept_fp32"] > 0
    assert np.max(np.abs(Km - Kref)) <= 1e-8
    # plain precision ignores the GEMM mode; out-of-range GEMM options are rejected
    Kp, _ = _gpu_K(snk, p, batch_max=300, gemm="df32")
    assert np.max(np.abs(Kp - K64)) <= 1e-15       # FP64 atomics: summation order only
    for bad in (dict(gemm=3), dict(gemm="split", tc_slices_hi=7), dict(gemm="split", tc_slices_lo=2)):
        with pytest.raises(snk.SnkError) as e:
            snk.Engine(p.basis, p.grid, precision="mixed", **bad)
        assert e.value.status == -1
    # captured in a CUDA graph and replayed
    eng = snk.Engine(p.basis, p.grid, batch_max=300, precision="mixed", fp32_bound=1e-3, gemm="df32", graph=1)
    eng.set_density(p.P)
    Kg1 = eng.build_K()
    Kg2 = eng.build_K()
    eng.close()
    # the FP32 pairs' G goes through FP64 atomics: summation order only, ~1e-14 run to run
    assert np.max(np.abs(Kg1 - Km)) <= 1e-12 and np.max(np.abs(Kg2 - Km)) <= 1e-12


def test_double_fp32_integrals(snk, chain4):
    """The high lists of the mixed form in double-FP32 arithmetic (Boys seeds,
    VRR, HRR and contraction on hi + lo float pairs): with every pair in that
    tier K keeps the FP64 build's parity with the oracle."""
    Kref = oracle.snk_K(chain4.basis, chain4.grid, chain4.P)
    K, st = _gpu_K(snk, chain4, screen="none", precision="mixed", fp32_bound=0.0, ds_integrals=1)
    assert st["pairs_kept_fp32"] == 0
    assert np.max(np.abs(K - Kref)) <= TOL_K
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    K64, _ = _gpu_K(snk, p, batch_max=300)
    Kd, _ = _gpu_K(snk, p, batch_max=300, precision="mixed", fp32_bound=0.0, ds_integrals=1)
    assert np.max(np.abs(Kd - Kref)) <= TOL_K
    assert np.max(np.abs(Kd - K64)) <= 1e-11
    # the mixed form's three tiers: FP32 below 1e-3, ds above, ds GEMMs; graph replay
    Km, sm = _gpu_K(snk, p, batch_max=300, precision="mixed", fp32_bound=1e-3, ds_integrals=1, gemm="df32")
    assert sm["pairs_kept_fp32"] > 0
    assert np.max(np.abs(Km - Kref)) <= 1e-8
    eng = snk.Engine(p.basis, p.grid, batch_max=300, precision="mixed", fp32_bound=1e-3, ds_integrals=1,
                     gemm="df32", graph=1)
    eng.set_density(p.P)
    eng.build_K()
    Kg = eng.build_K()
    eng.close()
    assert np.max(np.abs(Kg - Km)) <= 1e-10         # FP32 atomics: order-dependent at ~1e-11
    with pytest.raises(snk.SnkError):
        snk.Engine(p.basis, p.grid, precision="mixed", ds_integrals=2)


def test_split_gemms(snk):
    """SNK_GEMM_SPLIT: the tcgen05 split products, 5 slices for the F columns
    / G rows of shells in FP64-tier pairs and 4 for the shells only FP32-tier
    pairs touch; the FP32 tier's own accuracy bounds the result."""
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    form = dict(batch_max=300, precision="mixed", fp32_bound=1e-3, ds_integrals=1)
    Kd, sd = _gpu_K(snk, p, gemm="df32", **form)
    Ks, ss = _gpu_K(snk, p, gemm="split", **form)
    assert 0 < ss["gemm_flops_hi"] < ss["gemm_flops"]
    assert sd["gemm_flops_hi"] == sd["gemm_flops"]
    assert np.max(np.abs(Ks - Kref)) <= 1e-8
    assert np.max(np.abs(Ks - Kd)) <= 1e-8
    assert np.max(np.abs(Ks - Ks.T)) == 0.0
    # several chunks; and with no FP32 pairs every column is high-tier
    Kc, sc = _gpu_K(snk, p, gemm="split", workspace_bytes=1 << 20, **form)
    assert sc["n_chunks"] > 1 and np.max(np.abs(Kc - Kref)) <= 1e-8
    K0, s0 = _gpu_K(snk, p, batch_max=300, precision="mixed", fp32_bound=0.0, ds_integrals=1, gemm="split")
    assert s0["gemm_flops_hi"] == s0["gemm_flops"]
    assert np.max(np.abs(K0 - Kref)) <= TOL_K


def test_tile_screen(snk):
    """The per-tile screen of the FP32 lists skips (tile, pair) blocks whose
    bound on the tile's points is below eps_tile and trims the primitive
    pairs whose bounds add up to less; at 1e-11 (the chosen form's value)
    the mixed form stays within its 1e-8 target with less work."""
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    form = dict(batch_max=300, precision="mixed", fp32_bound=1e-3, ds_integrals=1, gemm="split")
    K0, s0 = _gpu_K(snk, p, **form)
    K1, s1 = _gpu_K(snk, p, eps_tile=1e-11, **form)
    assert s0["pair_points_fp32"] == s0["pair_points_fp32_listed"] > 0
    assert 0 < s1["pair_points_fp32"] < s1["pair_points_fp32_listed"] == s0["pair_points_fp32_listed"]
    assert s1["flops_fp32"] < s0["flops_fp32"]
    assert np.max(np.abs(K1 - Kref)) <= 1e-8 and np.max(np.abs(K1 - K0)) <= 1e-9
    assert np.max(np.abs(K1 - K1.T)) == 0.0
    # an enormous threshold skips every FP32 block: only the high tier remains
    K2, s2 = _gpu_K(snk, p, eps_tile=1e300, **form)
    assert s2["pair_points_fp32"] == 0 and np.all(np.isfinite(K2))
    with pytest.raises(snk.SnkError):
        snk.Engine(p.basis, p.grid, eps_tile=-1.0, **form)


@pytest.mark.parametrize("form", [
    dict(),                                                            # plain FP64
    dict(precision="mixed", fp32_bound=1e-3, ds_integrals=1, gemm="df32"),
    dict(precision="mixed", fp32_bound=1e-3, ds_integrals=1, gemm="split", eps_tile=1e-11),
    dict(precision="mixed", fp32_bound=1e-3, ds_integrals=1, gemm="split", workspace_bytes=1 << 20),
])
def test_builds_are_bitwise_reproducible(snk, form):
    """Every G entry of an integral launch has one writer whose additions come
    in list order, and K-hat sums the batches' contributions as exact 64-bit
    integers: repeated builds, and builds on a fresh handle (another ticket
    order of the persistent CTAs), give the same K bit for bit."""
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Ks = []
    for _ in range(2):
        eng = snk.Engine(p.basis, p.grid, batch_max=300, **form)
        eng.set_density(p.P)
        Ks += [eng.build_K() for _ in range(2)]
        st = eng.stats()
        eng.close()
    for K in Ks[1:]:
        assert np.array_equal(K, Ks[0])
    assert np.max(np.abs(Ks[0] - Ks[0].T)) == 0.0
    if "workspace_bytes" in form:
        assert st["n_chunks"] > 1


def test_two_densities_in_one_build(snk, chain4):
    """Several densities share every 3c-CP block (one screen on sum_d |P_d|):
    each K_d matches the oracle's K of P_d and the single-density build, in the
    plain and the mixed form; wrong counts and single-output builds are refused."""
    P2 = synth.make_density(chain4.mol, chain4.basis, 3, 4242, sigma=None)
    Ks = snk.Engine(chain4.basis, chain4.grid, screen="none")
    Ks.set_density([chain4.P, P2])
    K1, K2 = Ks.build_K()
    for K, P in ((K1, chain4.P), (K2, P2)):
        assert np.max(np.abs(K - oracle.snk_K(chain4.basis, chain4.grid, P))) <= TOL_K
    Ks.close()

    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Pb = synth.make_density(p.mol, p.basis, 14, 78)
    refs = [oracle.snk_K(p.basis, p.grid, P) for P in (p.P, Pb)]
    for form, tol in ((dict(), TOL_K),
                      (dict(eps=1e-10, precision="mixed", fp32_bound=3e-4, ds_integrals=1, gemm="split"), 1e-8)):
        eng = snk.Engine(p.basis, p.grid, batch_max=300, **form)
        eng.set_density([p.P, Pb])
        Kd = eng.build_K()
        st = eng.stats()
        assert len(Kd) == 2 and st["gemm_flops"] > 0
        for K, Kr in zip(Kd, refs):
            assert np.max(np.abs(K - Kr)) <= tol
            assert np.max(np.abs(K - K.T)) == 0.0
        Kone = np.empty((p.basis.n_functions,) * 2)
        rc = snk.lib().snk_build_K(eng._h, snk._P(Kone.ctypes.data))
        assert rc == -4                             # one output for two loaded densities
        eng.set_density(p.P)                        # back to one density
        assert np.max(np.abs(eng.build_K() - refs[0])) <= tol
        with pytest.raises(snk.SnkError) as e:
            eng.set_density([p.P, Pb, p.P])
        assert e.value.status == -1
        eng.close()


@pytest.mark.parametrize("recipe", ["small", "scale"])
def test_rigorous_pair_bound_holds(snk, recipe):
    """The screen's bound of max_r |A_ab(r)| (C9: product-centre expansion and
    the potential of a positive charge peaking at its centre) is never below
    the oracle's integrals: every shell pair of a six-atom molecule, at the
    atoms, the pair centre and random points near and far."""
    mol = synth.make_cluster_molecule(6, 31)
    basis = synth.make_basis(mol, recipe, 31)
    grid = synth.make_grid(mol, 6, 2, 4)
    eng = snk.Engine(basis, grid)
    rng = np.random.default_rng(9)
    worst = 0.0
    for sa in range(basis.n_shells):
        for sb in range(sa + 1):
            bound = eng.debug_pair_bound(sa, sb)
            mid = 0.5 * (basis.center[sa] + basis.center[sb])
            pts = np.concatenate([mid[None], basis.center[[sa, sb]], mid + rng.normal(size=(8, 3)) * 0.3,
                                  mid + rng.normal(size=(8, 3)) * 2.0, mid + rng.normal(size=(4, 3)) * 8.0])
            amax = max(float(np.max(np.abs(oracle.shell_A(basis, sa, sb, r)))) for r in pts)
            assert amax <= bound * (1.0 + 1e-12), (sa, sb, amax, bound)
            if bound > 0.0:   # a zero bound (product factor below the double range) has zero integrals
                worst = max(worst, amax / bound)
    eng.close()
    assert 0.0 < worst <= 1.0 + 1e-12   # the bound is attained (s-s pairs at their product centre)

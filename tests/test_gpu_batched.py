"""Batched form: several molecules of different sizes in one handle, all
batches in the same launches (persistent integral kernels over one device
work queue), optionally replayed from a CUDA graph, with autotuned tiles.
Every molecule's K must match its own oracle build to 1e-10."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_14280_gb300 as m
    return m


@pytest.fixture(scope="module")
def molecules():
    """Five molecules of 3..14 atoms with uneven grids (coarse enough for the
    oracle), a small batch_max so that batches are uneven too."""
    out = []
    for k, (n, nr, nt, npf) in enumerate([(3, 12, 3, 6), (14, 10, 3, 7), (6, 14, 4, 8), (9, 10, 3, 5), (4, 16, 4, 9)]):
        out.append(synth.cluster(n, 500 + k, n_r=nr, n_theta=nt, n_phi=npf, n_occ=max(2, n)))
    refs = [oracle.snk_K(p.basis, p.grid, p.P) for p in out]
    return out, refs


def test_batch_matches_oracle_per_molecule(snk, molecules):
    probs, refs = molecules
    eng = snk.Engine([p.basis for p in probs], [p.grid for p in probs], batch_max=200)
    assert eng.n_mol == len(probs)
    eng.set_density([p.P for p in probs])
    Ks = eng.build_K()
    for K, Kref in zip(Ks, refs):
        assert np.max(np.abs(K - Kref)) <= 1e-10
    st = eng.stats()
    assert st["n_batches"] > len(probs)
    eng.close()


def test_batch_equals_single_molecule_builds(snk, molecules):
    probs, _ = molecules
    eng = snk.Engine([p.basis for p in probs], [p.grid for p in probs])
    eng.set_density([p.P for p in probs])
    Ks = eng.build_K()
    for p, K in zip(probs, Ks):
        one = snk.Engine(p.basis, p.grid)
        one.set_density(p.P)
        K1 = one.build_K()
        one.close()
        assert np.max(np.abs(K - K1)) <= 1e-14
    eng.close()


def test_graph_replay_and_autotune(snk, molecules):
    import torch
    probs, refs = molecules
    eng = snk.Engine([p.basis for p in probs], [p.grid for p in probs], graph=1, batch_max=300)
    eng.set_stream(torch.cuda.current_stream())
    eng.set_density([p.P for p in probs])
    runs = eng.autotune()
    assert set(runs.values()) <= {2, 4, 8, 16, 32, 64, 128}
    out = torch.zeros(eng.packed, dtype=torch.float64, device="cuda")
    for rep in range(3):                       # capture, then two replays
        out.zero_()
        eng.build_K(out=out)
        torch.cuda.synchronize()
        flat = out.cpu().numpy()
        off = 0
        for n, Kref in zip(eng.nfs, refs):
            assert np.max(np.abs(flat[off:off + n * n].reshape(n, n) - Kref)) <= 1e-10
            off += n * n
    assert eng.stats()["ms_build"] > 0.0
    # a new density invalidates the captured plan
    P2 = [0.5 * p.P for p in probs]
    eng.set_density(P2)
    eng.build_K(out=out)
    torch.cuda.synchronize()
    flat = out.cpu().numpy()
    n0 = eng.nfs[0]
    assert np.max(np.abs(flat[:n0 * n0].reshape(n0, n0) - 0.5 * refs[0])) <= 1e-10
    eng.close()


def test_batch_mixed_precision(snk, molecules):
    probs, refs = molecules
    eng = snk.Engine([p.basis for p in probs], [p.grid for p in probs], precision="mixed", fp32_bound=1e-4)
    eng.set_density([p.P for p in probs])
    Ks = eng.build_K()
    assert eng.stats()["pairs_kept_fp32"] > 0
    for K, Kref in zip(Ks, refs):
        assert np.max(np.abs(K - Kref)) <= 1e-8
    eng.close()

"""Learned block screen: the GPU training kernels against the FP64 oracle MLP,
the FP16 tensor-core inference against FP32, and an end-to-end A/B of the
trained screen against the rigorous sn-LinK screen alone."""
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


def _random_mlp(seed, n):
    rng = np.random.default_rng(seed)
    w = (rng.normal(size=oracle.MLP_WEIGHTS) * 0.25).astype(np.float32)
    X = rng.normal(size=(n, 16)).astype(np.float32)
    Y = rng.normal(size=n).astype(np.float32)
    return w, X, Y


def test_gradients_match_oracle(snk):
    """GPU backward (FP32) vs FP64 backpropagation of the oracle, per layer
    relative to the layer's largest gradient."""
    w, X, Y = _random_mlp(11, 300)
    loss, g = snk.mlp_grad(w, X, Y, 4.0)
    lref, gref = oracle.mlp_loss_grad(w.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), 4.0)
    assert abs(loss - lref) <= 1e-5 * lref
    bounds = [0, 1024, 1088, 5184, 5248, 9344, 9408, 9472, 9473]
    for a, b in zip(bounds[:-1], bounds[1:]):
        scale = max(np.max(np.abs(gref[a:b])), 1e-12)
        assert np.max(np.abs(g[a:b] - gref[a:b])) <= 1e-5 * scale, (a, b)


def test_forward_fp32_and_fp16_inference(snk):
    w, X, _ = _random_mlp(12, 1000)
    y32 = snk.mlp_eval(w, X)
    yref = oracle.mlp_forward(w.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y32 - yref)) <= 1e-5 * max(1.0, np.max(np.abs(yref)))
    y16 = snk.mlp_eval(w, X, f16=True)          # FP16 operands, FP32 accumulation
    assert np.max(np.abs(y16 - yref)) <= 2e-2 * max(1.0, np.max(np.abs(yref)))


def test_training_reduces_the_loss(snk):
    rng = np.random.default_rng(13)
    X = rng.normal(size=(20000, 16)).astype(np.float32)
    Y = (0.3 * X[:, 0] - 0.2 * X[:, 1] * X[:, 2] + 0.1 * np.abs(X[:, 3])).astype(np.float32)
    w, hist = snk.mlp_train(X, Y, epochs=8, batch=1024, lr=2e-3, seed=1)
    assert hist[-1] < 0.2 * hist[0]
    pred = snk.mlp_eval(w, X[:2000])
    assert np.mean((pred - Y[:2000]) ** 2) < 0.05


def _cluster(seed):
    return synth.cluster(10, seed, n_r=20, n_theta=5, n_phi=10, n_occ=8)


def test_learned_screen_beats_rigorous_screen_within_tolerance(snk):
    """Trained on blocks the plain FP64 method computes for three instances,
    applied to a fourth: fewer blocks than the rigorous screen alone, K within
    1e-8 of the oracle; without weights the learned mode is the rigorous screen."""
    feats, labs = [], []
    for s in range(3):
        p = _cluster(3100 + s)
        eng = snk.Engine(p.basis, p.grid, eps=1e-10, batch_max=400)
        eng.set_density(p.P)
        f, l = eng.learn_collect(stride=1)
        eng.close()
        assert f.shape[0] == l.shape[0] > 1000 and np.all(np.isfinite(l))
        feats.append(f)
        labs.append(l)
    w, hist = snk.mlp_train(np.concatenate(feats), np.concatenate(labs), epochs=40, batch=2048, lr=2e-3,
                            under_weight=8.0, seed=3)
    assert hist[-1] < hist[0]
    p = _cluster(3200)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    rig = snk.Engine(p.basis, p.grid, eps=1e-10, batch_max=400)
    rig.set_density(p.P)
    K0 = rig.build_K()
    s0 = rig.stats()
    fb = snk.Engine(p.basis, p.grid, eps=1e-10, batch_max=400, screen="learned")   # no weights: fallback
    fb.set_density(p.P)
    assert np.max(np.abs(fb.build_K() - K0)) <= 1e-14
    lrn = snk.Engine(p.basis, p.grid, eps=1e-10, batch_max=400, screen="learned", learned_skip=-9.5)
    lrn.screen_load(w)
    lrn.set_density(p.P)
    K1 = lrn.build_K()
    s1 = lrn.stats()
    assert s1["pairs_learned_skipped"] > 0
    assert s1["pairs_kept"] == s0["pairs_kept"] - s1["pairs_learned_skipped"]
    assert np.max(np.abs(K0 - Kref)) <= 1e-8
    assert np.max(np.abs(K1 - Kref)) <= 1e-8


def test_learned_tier_routing(snk):
    """With learned_fp32 the trained screen also moves high-tier blocks whose
    predicted contribution is small to the FP32 tier: fewer double-FP32
    blocks, the same kept blocks, K within 1e-8 of the oracle.  The molecule is
    smaller and its grid coarser than the training clusters, so the threshold
    is a decade below the calibrated one."""
    w, thr, _ = snk.trained_screen()
    p = _cluster(3200)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    form = dict(eps=1e-10, batch_max=400, precision="mixed", fp32_bound=3e-4, ds_integrals=1, gemm="split",
                screen="learned", learned_skip=thr)
    out = {}
    for lf in (-99.0, -5.0):
        e = snk.Engine(p.basis, p.grid, learned_fp32=lf, **form)
        e.screen_load(w)
        e.set_density(p.P)
        out[lf] = (e.build_K(), e.stats())
        e.close()
    (K0, s0), (K1, s1) = out[-99.0], out[-5.0]
    assert s1["pairs_kept"] == s0["pairs_kept"]
    assert s1["pairs_kept_fp32"] > s0["pairs_kept_fp32"]
    assert s1["gemm_flops_hi"] <= s0["gemm_flops_hi"]
    assert np.max(np.abs(K0 - Kref)) <= 1e-8
    assert np.max(np.abs(K1 - Kref)) <= 1e-8
    assert np.max(np.abs(K1 - K1.T)) == 0.0

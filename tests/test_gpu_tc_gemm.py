"""The split-product tensor-core GEMM (gemm = SNK_GEMM_SPLIT) through the C ABI.

Unit level (snk_debug_tc_gemm, C = A B^T): integer matrices whose slices are
exact must come out exact, which pins the shared-memory layout, the tcgen05
descriptors and the exact FP32 accumulation of each 256-term run; random and
badly scaled matrices must stay within the truncation bound of the slices.
Build level: the mixed form with the tensor-core products against the CPU
oracle and against the double-FP32 products, with ragged batches and
several chunks.
"""
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
    m.lib()
    return m


def _bound(A, B, slices, chunk=256):
    """Error bound of the split products, per run of `chunk` columns and
    summed over runs: the truncation of the fixed-point slices, (2 slices + 4)
    2^(-8 slices) 4 max_run|A_m| max_run|B_n| per term, plus the FP32
    rounding of the accumulator that sums the products of level >= 2 (about
    2^-16 of the run's scale, rounded at 2^-24 relative once per 16 terms and
    product), bounded by 2^-36 4 max max per term."""
    M, K = A.shape
    N = B.shape[0]
    out = np.zeros((M, N))
    for c0 in range(0, K, chunk):
        am = np.abs(A[:, c0:c0 + chunk]).max(axis=1)
        bm = np.abs(B[:, c0:c0 + chunk]).max(axis=1)
        n = min(chunk, K - c0)
        out += n * np.outer(am, bm)
    return ((2 * slices + 4) * 2.0 ** (-8 * slices) + 2.0 ** -36) * 4 * out


@pytest.mark.parametrize("slices", [3, 4, 5, 6])
def test_integer_products_are_exact(snk, slices):
    """Entries -30..30: the first slice holds each exactly, every run sum is
    an integer below 2^24 units, so C must equal A B^T exactly.  A layout,
    descriptor or accumulation error shows up as a wrong integer."""
    rng = np.random.default_rng(slices)
    for M, N, K in ((128, 128, 32), (200, 300, 700), (37, 5, 1000), (1, 129, 257)):
        A = rng.integers(-30, 31, size=(M, K)).astype(np.float64)
        B = rng.integers(-30, 31, size=(N, K)).astype(np.float64)
        C = snk.debug_tc_gemm(A, B, slices)
        assert np.array_equal(C, A @ B.T), (M, N, K, np.max(np.abs(C - A @ B.T)))


@pytest.mark.parametrize("slices", [3, 5, 6])
def test_random_products_within_the_slice_bound(snk, slices):
    rng = np.random.default_rng(10 + slices)
    M, N, K = 257, 190, 1100
    A = rng.normal(size=(M, K))
    B = rng.normal(size=(N, K))
    # rows spanning many orders of magnitude, and a few all-zero rows
    A *= 10.0 ** rng.uniform(-12, 3, size=(M, 1))
    B *= 10.0 ** rng.uniform(-6, 2, size=(N, 1))
    A[5] = 0.0
    B[7] = 0.0
    C = snk.debug_tc_gemm(A, B, slices)
    ref = A @ B.T
    err = np.abs(C - ref)
    bound = _bound(A, B, slices)
    assert np.all(err <= bound + 1e-300), np.max(err / (bound + 1e-300))
    assert np.all(C[5] == 0.0) and np.all(C[:, 7] == 0.0)
    if slices >= 5:   # far below FP32 relative to the operand scales
        rel = err / (np.abs(A) @ np.abs(B).T + 1e-300)
        assert np.median(rel) < 1e-11


def test_tiny_and_subnormal_runs(snk):
    """Runs whose largest value is subnormal, or far below every other run,
    give finite results: their slices are zero."""
    rng = np.random.default_rng(3)
    A = rng.normal(size=(130, 600))
    B = rng.normal(size=(70, 600))
    A[:, :256] *= 1e-310
    A[3] *= 1e-200
    B[:, 300:] *= 1e-305
    C = snk.debug_tc_gemm(A, B, 5)
    assert np.all(np.isfinite(C))
    assert np.max(np.abs(C - A @ B.T)) <= 1e-8 * np.max(np.abs(A @ B.T))


def test_degenerate_shapes(snk):
    A = np.ones((3, 0))
    assert np.array_equal(snk.debug_tc_gemm(A, np.ones((4, 0))), np.zeros((3, 4)))
    with pytest.raises(snk.SnkError):
        snk.debug_tc_gemm(np.ones((2, 2)), np.ones((2, 2)), slices=7)


def _gpu_K(snk, p, **opt):
    eng = snk.Engine(p.basis, p.grid, **opt)
    eng.set_density(p.P)
    K = eng.build_K()
    st = eng.stats()
    eng.close()
    return K, st


def test_tensor_core_products_in_the_mixed_form(snk):
    """F = X P and Kt = G^T X on the tensor cores (5 slices on the high-tier
    columns and rows, 4 on the rest) against the oracle and the double-FP32
    products, on ragged batches, one chunk and several."""
    p = synth.cluster(12, 77, n_r=16, n_theta=4, n_phi=9, n_occ=10)
    Kref = oracle.snk_K(p.basis, p.grid, p.P)
    form = dict(batch_max=300, precision="mixed", fp32_bound=1e-3, ds_integrals=1)
    Kd, sd = _gpu_K(snk, p, gemm="df32", **form)
    Kt, st = _gpu_K(snk, p, gemm="split", **form)
    assert 0 < st["gemm_flops_hi"] < st["gemm_flops"] and st["gemm_tc_flops"] > 0
    assert np.max(np.abs(Kt - Kref)) <= 1e-8
    assert np.max(np.abs(Kt - Kd)) <= 1e-8
    assert np.max(np.abs(Kt - Kt.T)) == 0.0 and np.all(np.isfinite(Kt))
    Kc, sc = _gpu_K(snk, p, gemm="split", workspace_bytes=1 << 20, **form)
    assert sc["n_chunks"] > 1 and np.max(np.abs(Kc - Kref)) <= 1e-8
    # every pair in the high tier: FP64-grade products (6 slices) keep the plain form's 1e-10
    K0, s0 = _gpu_K(snk, p, batch_max=300, precision="mixed", fp32_bound=0.0, ds_integrals=1, gemm="split",
                    tc_slices_hi=6)
    assert s0["gemm_flops_hi"] == s0["gemm_flops"]
    assert np.max(np.abs(K0 - Kref)) <= 1e-10

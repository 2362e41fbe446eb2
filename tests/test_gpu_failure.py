"""Failure detection on the GPU without a fault: a bounded wait that nothing
completes gives up after its limit, the kernel sets the handle's device flag
and returns, and the host reports SNK_ERR_TIMEOUT; the context and the handle
stay usable (the next build is correct)."""
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


def test_wait_that_runs_out_reports_timeout(snk):
    p = synth.cluster(4, 5, n_r=12, n_theta=4, n_phi=8, n_occ=4)
    eng = snk.Engine(p.basis, p.grid, precision="mixed", fp32_bound=1e-3, ds_integrals=1, gemm="split")
    eng.set_density(p.P)
    assert eng.debug_wait_timeout(10_000_000) == -7          # SNK_ERR_TIMEOUT after 10 ms
    assert "waiting" in snk.lib().snk_last_error(eng._h).decode()
    assert eng.debug_wait_timeout(0) == -1                   # limit out of range
    K = eng.build_K()                                        # the flag was cleared: the handle works
    assert np.max(np.abs(K - oracle.snk_K(p.basis, p.grid, p.P))) <= 1e-8
    eng.close()

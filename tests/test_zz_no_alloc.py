"""The allocation-free entry point snk_shell_A_noalloc, through the C ABI.

Some callers cannot call cudaMalloc (for example while a CUDA graph is being
captured, or when a host owns all device memory through its own pool).  For
them the library evaluates the 3c-CP block of a shell pair into a fixed
scratch array instead of a per-call allocation.  This test checks that entry
point against the allocating snk_debug_shell_A on two calls in a row (the
scratch keeps the previous call's contents, so the second call must not see
stale data), and that sizes beyond the scratch are rejected.  It lives in a
file of its own that pytest collects last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_14280_gb300 as snk
    mol = synth.make_cluster_molecule(6, 31)
    basis = synth.make_basis(mol, "scale", 31)
    grid = synth.make_grid(mol, 6, 2, 4)
    eng = snk.Engine(basis, grid)
    eng.set_stream(torch.cuda.current_stream())
    yield snk, eng, basis
    eng.close()


def _pairs(basis):
    """One shell pair of every class in both orders, plus a diagonal pair."""
    out, seen = [], set()
    for sa in range(basis.n_shells):
        for sb in range(basis.n_shells):
            key = (int(basis.l[sa]), int(basis.l[sb]), sa == sb)
            if key not in seen:
                seen.add(key)
                out.append((sa, sb))
    return out


def test_no_alloc_matches_allocating_entry_point_on_two_calls(engine):
    import torch
    snk, eng, basis = engine
    rng = np.random.default_rng(11)
    for sa, sb in _pairs(basis):
        na = (int(basis.l[sa]) + 1) * (int(basis.l[sa]) + 2) // 2
        nb = (int(basis.l[sb]) + 1) * (int(basis.l[sb]) + 2) // 2
        # two consecutive calls with different point sets and sizes
        for n in (4096, 777):
            mid = 0.5 * (basis.center[sa] + basis.center[sb])
            pts = mid + rng.normal(size=(n, 3)) * rng.choice([0.5, 3.0, 12.0], size=(n, 1))
            ref = eng.debug_shell_A(sa, sb, pts)
            xyz = torch.from_numpy(pts).cuda()
            out = torch.full((n, na, nb), float("nan"), dtype=torch.float64, device="cuda")
            eng.shell_A_noalloc(sa, sb, xyz, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            # the tolerance of the shell-block parity test
            tol = 1e-12 * np.max(np.abs(ref), axis=(1, 2), keepdims=True) + 1e-14 * np.max(np.abs(ref)) + 1e-18
            assert np.all(np.abs(got - ref) <= tol), (sa, sb, n)


def test_no_alloc_rejects_sizes_beyond_its_scratch(engine):
    import torch
    snk, eng, basis = engine
    xyz = torch.zeros((4097, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros((4097, 1, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(snk.SnkError) as e:
        eng.shell_A_noalloc(0, 0, xyz, out)
    assert e.value.status == -1 and "4096" in str(e.value)

"""The device-memory hook snk_set_allocator (include/snk.h), through the C ABI.

Failures are injected on the host: the caller's allocator returns NULL (here:
a Python callback that refuses after a chosen number of blocks), never a GPU
fault.  The call that needed the memory must return SNK_ERR_OOM, the handle
must stay usable for snk_last_error, another allocator and a later build, and
that build must equal the one made with cudaMalloc."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_14280_gb300 as snk
    p = synth.chain4()
    eng = snk.Engine(p.basis, p.grid)
    eng.set_density(p.P)
    K0 = eng.build_K()
    eng.close()
    return torch, snk, p, K0


class TorchPool:
    """Blocks from PyTorch's caching allocator; refuses after `limit` blocks."""

    def __init__(self, torch, limit=None):
        self.torch, self.limit, self.blocks, self.calls, self.frees = torch, limit, {}, 0, 0

    def alloc(self, nbytes):
        self.calls += 1
        if self.limit is not None and self.calls > self.limit:
            return 0
        t = self.torch.empty(nbytes, dtype=self.torch.uint8, device="cuda")
        self.blocks[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr):
        self.frees += 1
        assert ptr in self.blocks, "free of a block the allocator never gave out"
        del self.blocks[ptr]


def test_every_buffer_moves_to_the_callers_allocator(setup):
    torch, snk, p, K0 = setup
    eng = snk.Engine(p.basis, p.grid)
    pool = TorchPool(torch)
    eng.set_allocator(pool.alloc, pool.free)
    n_geometry = len(pool.blocks)
    assert n_geometry > 10                       # the geometry tables moved out of cudaMalloc
    eng.set_density(p.P)
    K = eng.build_K()
    assert np.max(np.abs(K - K0)) <= 1e-13
    assert len(pool.blocks) > n_geometry        # density, lists and workspaces from the hook too
    eng.close()
    assert not pool.blocks and pool.frees == pool.calls   # every block handed back at destroy


def test_moving_into_a_refusing_allocator_keeps_the_old_buffers(setup):
    torch, snk, p, K0 = setup
    eng = snk.Engine(p.basis, p.grid)
    eng.set_density(p.P)
    pool = TorchPool(torch, limit=3)
    with pytest.raises(snk.SnkError) as e:
        eng.set_allocator(pool.alloc, pool.free)
    assert e.value.status == -5 and "memory" in str(e.value).lower()
    assert not pool.blocks                      # the blocks it did get went back
    eng.set_density(p.P)                        # the handle kept its cudaMalloc buffers
    assert np.max(np.abs(eng.build_K() - K0)) <= 1e-13
    eng.close()


@pytest.mark.parametrize("where", [0.0, 0.34, 0.67, 1.0])
def test_allocation_failure_returns_oom_and_the_handle_stays_usable(setup, where):
    """The allocator refuses the k-th block that set_density + build_K ask
    for, k spread over all of them: that call returns SNK_ERR_OOM, and the
    same handle then builds the right K with a working allocator."""
    torch, snk, p, K0 = setup
    # how many blocks does a density + build need after the geometry moved?
    probe = snk.Engine(p.basis, p.grid)
    counting = TorchPool(torch)
    probe.set_allocator(counting.alloc, counting.free)
    n_geom = counting.calls
    probe.set_density(p.P)
    probe.build_K()
    n_need = counting.calls - n_geom
    probe.close()
    assert n_need >= 4
    k = min(n_need - 1, int(where * (n_need - 1)))
    eng = snk.Engine(p.basis, p.grid)
    pool = TorchPool(torch)
    eng.set_allocator(pool.alloc, pool.free)
    pool.limit = pool.calls + k                 # refuse the (k+1)-th new block
    with pytest.raises(snk.SnkError) as e:
        eng.set_density(p.P)
        eng.build_K()
    assert e.value.status == -5, e.value
    assert lib_error(snk, eng)                  # snk_last_error says what failed
    pool.limit = None                           # the same allocator works again
    eng.set_density(p.P)
    K = eng.build_K()
    assert np.max(np.abs(K - K0)) <= 1e-13
    eng.set_allocator(None, None)               # and back to cudaMalloc
    assert not pool.blocks
    eng.set_density(p.P)
    assert np.max(np.abs(eng.build_K() - K0)) <= 1e-13
    eng.close()


def lib_error(snk, eng):
    return snk.lib().snk_last_error(eng._h).decode()


def test_torch_caching_allocator_owns_the_workspace(setup):
    torch, snk, p, K0 = setup
    eng = snk.Engine(p.basis, p.grid)
    before = torch.cuda.memory_allocated()
    blocks = eng.use_torch_allocator()
    eng.set_density(p.P)
    K = eng.build_K()
    held = torch.cuda.memory_allocated() - before
    assert held >= sum(t.numel() for t in blocks.values()) > 0
    assert np.max(np.abs(K - K0)) <= 1e-13
    eng.close()
    assert not blocks
    assert torch.cuda.memory_allocated() <= before


def test_bad_allocator_arguments(setup):
    torch, snk, p, K0 = setup
    eng = snk.Engine(p.basis, p.grid)
    with pytest.raises(ValueError):
        eng.set_allocator(lambda n: 0, None)
    L = snk.lib()
    assert L.snk_set_allocator(eng._h, snk.ALLOC_FN(lambda n, u: None), snk.FREE_FN(), None) == -1
    assert L.snk_set_allocator(None, snk.ALLOC_FN(), snk.FREE_FN(), None) == -1
    eng.close()

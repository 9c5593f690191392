"""Failure paths of the C ABI on the GPU, made without faulting it: an allocator that fails
on its k-th call (CFR_ENOMEM; nothing leaked; the next create succeeds) and a bounded
device-side wait that gives up (CFR_ETIMEOUT; the context stays usable).  The paper has no
fault handling: these are the library's own error contracts (include/pcfr.h)."""
import numpy as np
import pytest

from paper_2605_19928_gb300 import capi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_19928_gb300 import build as pbuild
    pbuild.build()
    capi.load()
    import torch
    assert torch.cuda.is_available()
    capi.use_torch_allocator()
    yield
    capi.use_torch_allocator()


class CountingAllocator:
    """PyTorch's caching allocator behind a counter that fails the fail_at-th call."""

    def __init__(self, fail_at=None):
        self.calls, self.fail_at, self.live = 0, fail_at, {}

    def alloc(self, nbytes, stream):
        import torch
        self.calls += 1
        if self.calls == self.fail_at:
            raise MemoryError("planted allocation failure")  # the binding returns NULL
        p = torch.cuda.caching_allocator_alloc(nbytes, stream=stream or 0)
        self.live[p] = nbytes
        return p

    def free(self, p):
        import torch
        del self.live[p]
        torch.cuda.caching_allocator_delete(p)


def _specs():
    return [synth.river_subgame(n_hands=64, seed=3, range_seed=4),
            synth.river_subgame(n_hands=203, seed=5, range_seed=6)]


def test_allocation_failure_reports_enomem_and_leaks_nothing():
    opts = capi.make_opts("dcfr")
    probe = CountingAllocator()
    capi.cfr_set_allocator(probe.alloc, probe.free)
    try:
        t = capi.cfr_batch_create(_specs(), opts)
        n = probe.calls
        capi.cfr_tree_destroy(t)
        assert n >= 3 and not probe.live
        for k in sorted({1, 2, n // 2, n - 1, n}):
            a = CountingAllocator(fail_at=k)
            capi.cfr_set_allocator(a.alloc, a.free)
            with pytest.raises(capi.CfrError) as e:
                capi.cfr_batch_create(_specs(), opts)
            assert e.value.code == capi.CFR_ENOMEM, (k, e.value)
            assert a.calls == k, "create went on allocating after a failure"
            assert not a.live, f"allocation {k} failed and {len(a.live)} blocks were not released"
        ok = CountingAllocator()
        capi.cfr_set_allocator(ok.alloc, ok.free)
        t = capi.cfr_batch_create(_specs(), opts)
        try:
            capi.cfr_iterate(t, 3)
            expl, _ = capi.cfr_exploitability(t, 2)
            assert np.all(np.isfinite(expl)) and np.all(expl > 0)
        finally:
            capi.cfr_tree_destroy(t)
        assert not ok.live
    finally:
        capi.use_torch_allocator()


def _solve(spec, iters):
    t = capi.cfr_tree_create(spec, capi.make_opts("dcfr"))
    try:
        capi.cfr_iterate(t, iters)
        return capi.cfr_exploitability(t)[0][0]
    finally:
        capi.cfr_tree_destroy(t)


@pytest.mark.parametrize("schedule", ["level", "stream"])
def test_a_wait_that_gives_up_is_reported_as_timeout(schedule):
    """The terminal kernel's first bulk-copy wait is told to give up at once: every block
    drains its copies, sets the device flag and returns; the next synchronising call
    reports CFR_ETIMEOUT, and afterwards a fresh handle solves exactly as before."""
    spec = synth.river_subgame(n_hands=203, seed=3, range_seed=4)
    want = _solve(spec, 4)
    t = capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule=schedule))
    try:
        capi.cfr_iterate(t, 2)
        capi.cfr_sync(t)
        capi.cfr_debug_first_wait_polls(0)
        try:
            capi.cfr_iterate(t, 1)
            with pytest.raises(capi.CfrError) as e:
                capi.cfr_sync(t)
            assert e.value.code == capi.CFR_ETIMEOUT
            with pytest.raises(capi.CfrError) as e:  # the flag stays set on this handle
                capi.cfr_exploitability(t)
            assert e.value.code == capi.CFR_ETIMEOUT
        finally:
            import torch
            torch.cuda.synchronize()
            capi.cfr_debug_first_wait_polls(-1)
    finally:
        capi.cfr_tree_destroy(t)
    assert _solve(spec, 4) == want

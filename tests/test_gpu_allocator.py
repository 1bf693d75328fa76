"""Device memory through the caller's allocator (fsi_exec_desc.dev_alloc): contexts whose every buffer, offline
temporaries included, comes from PyTorch's caching allocator run bit-identically to contexts on cudaMalloc and
hand every buffer back (needs a GB300 and the library)."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


class TorchAllocator:
    """alloc/free on torch's caching allocator, with a record of what is live."""

    def __init__(self):
        self.live, self.calls, self.peak = {}, 0, 0

    def alloc(self, n):
        import torch
        p = torch.cuda.caching_allocator_alloc(n)
        self.live[p] = n
        self.calls += 1
        self.peak = max(self.peak, sum(self.live.values()))
        return p

    def free(self, p):
        import torch
        assert p in self.live, "a pointer the allocator did not hand out"
        self.live.pop(p)
        torch.cuda.caching_allocator_delete(p)


@pytest.mark.parametrize("workload,drop_tol", [("small_flag", 0.0), ("tandem_small", 0.007)])
def test_context_on_a_caller_allocator_matches_cudamalloc(workload, drop_tol):
    w = getattr(wl, workload)()
    ref = gpu_context(w, drop_tol=drop_tol)
    ref.advance(8)
    want = [ref.history(b) for b in range(len(w["bodies"]))]
    ref.close()
    a = TorchAllocator()
    c = gpu_context(w, drop_tol=drop_tol, allocator=(a.alloc, a.free))
    held = sum(a.live.values())
    assert held > 0 and a.calls > len(a.live)         # lifetime buffers plus freed offline temporaries
    assert held >= c.stats()["device_bytes"] > 0
    c.advance(8)
    for b, h in enumerate(want):
        assert np.array_equal(c.history(b), h), b
    c.close()
    assert not a.live


def test_allocator_without_memory_fails_cleanly():
    """An allocator that gives nothing: fsi_create fails with FSI_ERR_OOM and nothing stays allocated."""
    import paper_2103_06415_gb300 as lib
    given = []

    def alloc(n):
        given.append(n)
        return 0

    with pytest.raises(lib.FsiError) as e:
        gpu_context(wl.small_plate(), allocator=(alloc, lambda p: None))
    assert "OOM" in str(e.value) and given

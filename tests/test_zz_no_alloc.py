"""scd_propagate_noalloc: the propagation entry point for callers that cannot
allocate device memory when they call (software with no allocation after
start-up, hosts whose allocator the library cannot reach, loops that cannot
pay for cudaMalloc's device-wide synchronisation).  Its scratch is a fixed
device array inside the library instead of an allocation.

Checked through the C ABI against scd_propagate, the allocating entry point,
on two calls in a row with different inputs (the shared array keeps the
previous call's contents, which must not leak into the next result): both
run the same kernels on the same inputs, so the results must be equal bit
for bit.  A counting allocator installed through scd_set_allocator checks
the promise itself: the variant makes no allocation or free at all, where
scd_propagate makes at least one of each.  This file is collected last so
that a stop at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import population as P

pytestmark = pytest.mark.gpu


def _call(fn, d_el, n, d_obj, d_t, m, d_out):
    return fn(ctypes.c_void_p(d_el.data_ptr()), n, ctypes.c_void_p(d_obj.data_ptr()),
              ctypes.c_void_p(d_t.data_ptr()), m, ctypes.c_void_p(d_out.data_ptr()),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


class _CountingAllocator:
    """Device allocation hooks that count their calls (and hand the work to
    torch's caching allocator); the previous hooks come back on exit."""

    def __init__(self, B):
        self.B = B
        self.allocs = self.frees = 0

        def _alloc(nbytes, stream, ctx):
            self.allocs += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))

        def _free(ptr, stream, ctx):
            self.frees += 1
            torch.cuda.caching_allocator_delete(int(ptr))

        self.hooks = (B.ALLOC_FN(_alloc), B.FREE_FN(_free))

    def __enter__(self):
        assert self.B.lib().scd_set_allocator(self.hooks[0], self.hooks[1], None) == 0
        return self

    def __exit__(self, *exc):
        prev = self.B._torch_hooks
        if prev is not None:
            self.B.lib().scd_set_allocator(prev[0], prev[1], None)
        else:
            self.B.lib().scd_set_allocator(ctypes.cast(None, self.B.ALLOC_FN),
                                           ctypes.cast(None, self.B.FREE_FN), None)


def test_noalloc_propagate_matches_allocating_entry_point_twice():
    from paper_1901_10475_gb300 import _binding as B
    lib = B.lib()
    torch.cuda.set_device(0)
    # two different populations and time sets: call two's elements differ
    # from call one's at every index below its n, so an entry of the shared
    # array that call two's set-up kernel failed to rewrite would show
    for call, (n, m, seed) in enumerate([(5000, 40000, 1), (1200, 30000, 2)]):
        els = P.catalog_mixture(n=n, seed=900 + seed)
        g = np.random.default_rng(seed)
        d_el = torch.as_tensor(np.ascontiguousarray(els), device="cuda")
        d_obj = torch.as_tensor(g.integers(0, n, m).astype(np.int32), device="cuda")
        d_t = torch.as_tensor(g.uniform(0, 2 * 86400.0, m), device="cuda")
        ref = torch.zeros((m, 3), dtype=torch.float64, device="cuda")
        got = torch.full((m, 3), float("nan"), dtype=torch.float64, device="cuda")
        with _CountingAllocator(B) as ca:
            assert _call(lib.scd_propagate, d_el, n, d_obj, d_t, m, ref) == B.SCD_OK
            torch.cuda.synchronize()
            assert ca.allocs >= 1 and ca.frees >= 1, (ca.allocs, ca.frees)
            ca.allocs = ca.frees = 0
            assert _call(lib.scd_propagate_noalloc, d_el, n, d_obj, d_t, m, got) == B.SCD_OK
            torch.cuda.synchronize()
            assert ca.allocs == 0 and ca.frees == 0, (ca.allocs, ca.frees)
        # the same kernels on the same inputs: equal bit for bit
        assert torch.equal(got, ref), (call, (got - ref).abs().max().item())


def test_noalloc_rejects_sizes_beyond_its_capacity():
    from paper_1901_10475_gb300 import _binding as B
    lib = B.lib()
    n = B.SCD_NOALLOC_MAX_OBJECTS + 1
    d_el = torch.zeros((n, 7), dtype=torch.float64, device="cuda")
    d_obj = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    rc = _call(lib.scd_propagate_noalloc, d_el, n, d_obj, d_t, 1, out)
    assert rc == B.SCD_ERR_CAPACITY
    assert "capacity" in B.status_string(rc)

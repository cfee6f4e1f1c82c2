"""Allocation failure through the allocator hook (hmat_set_allocator): a build or a product whose
n-th device allocation fails returns HMAT_ENOMEM with a NULL output handle, and releases every
buffer it had taken (the hook sees as many frees as allocations). The failure is made on the
host, in the hook; no kernel is made to fail."""
import ctypes

import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


class CountingAllocator:
    """Device buffers from torch's caching allocator, counted; the fail_at-th allocation since the
    last reset() returns NULL."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.unknown_frees = 0
        self.reset()

    def reset(self, fail_at=-1):
        self.calls = 0
        self.fail_at = fail_at
        self.failed = False

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.calls == self.fail_at:
            self.failed = True
            return 0
        t = self.torch.empty(max(int(nbytes), 1), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr):
        if self.live.pop(ptr, None) is None:
            self.unknown_frees += 1


def _raw_multiply(H, A, B, eps):
    out = ctypes.c_void_p(12345)  # must come back NULL on failure
    opts = H.MultOpts(eps=eps, mode=H.MODE_F64, seed=3, power_iters=-1, compressor=H.COMP_RANDOMIZED)
    st = H.lib().hmat_multiply(A.handle, B.handle, ctypes.byref(opts), None, ctypes.byref(out))
    return st, out.value


def _raw_build(H, P):
    out = ctypes.c_void_p(12345)
    n, dim = P.shape
    opts = H.BuildOpts(32, 1.0, 1e-10, 64, 0)
    st = H.lib().hmat_build(P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, dim, 0, ctypes.byref(opts),
                            None, None, ctypes.byref(out))
    return st, out.value


def test_nth_allocation_failure_is_clean(H):
    import torch
    P = np.ascontiguousarray(inputs.points(0, 2, 1500, 9))
    ca = CountingAllocator()
    H.hmat_set_allocator(ca.alloc, ca.free)
    try:
        # a build and a product that succeed, to count their allocations
        ca.reset()
        A = H.hmat_build(P, 0, leaf_size=32, aca_eps=1e-10)
        n_build = ca.calls
        live_a = len(ca.live)
        assert n_build > 0 and live_a > 0
        ca.reset()
        C = H.hmat_multiply(A, A, 1e-6, mode=H.MODE_F64, seed=3)
        n_mult = ca.calls
        C_ref = C.to_dense()
        C.close()
        torch.cuda.synchronize()
        assert len(ca.live) == live_a and n_mult > 3
        for k in sorted({1, 2, n_mult // 3, (2 * n_mult) // 3, n_mult}):
            ca.reset(fail_at=k)
            st, h = _raw_multiply(H, A, A, 1e-6)
            torch.cuda.synchronize()
            assert ca.failed, k
            assert st == H.HMAT_ENOMEM, (k, st, H.lib().hmat_last_error())
            assert h is None, k
            assert b"custom allocator" in H.lib().hmat_last_error()
            assert len(ca.live) == live_a, (k, len(ca.live), live_a)
        for k in sorted({1, n_build // 2, n_build}):
            ca.reset(fail_at=k)
            st, h = _raw_build(H, P)
            torch.cuda.synchronize()
            assert ca.failed and st == H.HMAT_ENOMEM and h is None, (k, st)
            assert len(ca.live) == live_a, (k, len(ca.live), live_a)
        # the library is usable after the failures: the same product, the same result
        ca.reset()
        C2 = H.hmat_multiply(A, A, 1e-6, mode=H.MODE_F64, seed=3)
        assert np.linalg.norm(C2.to_dense() - C_ref) <= 3e-6 * np.linalg.norm(C_ref)
        C2.close()
        A.close()
        torch.cuda.synchronize()
        assert len(ca.live) == 0 and ca.unknown_frees == 0
    finally:
        H.hmat_set_allocator(None, None)
    # and with the default pool again
    A = H.hmat_build(P, 0, leaf_size=32, aca_eps=1e-10)
    assert H.hmat_multiply(A, A, 1e-6).leaf_count() > 0

"""The allocation-free gradient entry point against the allocating one, through the C-ABI.

This file is collected last so that the fixed-scratch call also runs after every other GPU test
of the session has used the device (and passes when run alone as well)."""
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


def test_grad_noalloc_matches_grad(H):
    F, NP = H.RANK_FEATURES, H.RANK_PARAMS
    w = ((inputs.uniform01(71, NP) * 2.0 - 1.0) * 0.3).astype(np.float16).astype(np.float32)
    mean = (inputs.uniform01(72, F) - 0.5).astype(np.float32)
    dev = (inputs.uniform01(73, F) + 0.5).astype(np.float32)
    M = H.hmat_rankmodel_create(w, mean, dev)
    for count in (777, 1):
        X = (inputs.uniform01(74 + count, count * F).reshape(count, F) * 4.0 - 2.0).astype(np.float32)
        r = np.floor(inputs.uniform01(75 + count, count) * 30.0).astype(np.float32)
        g_ref, l_ref = M.grad(X, r)
        for _ in range(2):  # two calls in a row: the accumulators start at zero each time
            g, l = H.hmat_rankmodel_grad_noalloc(M, X, r)
            assert np.abs(g - g_ref).max() <= 1e-5 * np.abs(g_ref).max()
            assert abs(l - l_ref) <= 1e-5 * l_ref


def test_grad_noalloc_rejects_oversize(H):
    F = H.RANK_FEATURES
    M = H.hmat_rankmodel_create(np.zeros(H.RANK_PARAMS, np.float32), np.zeros(F), np.ones(F))
    n = H.RANKGRAD_NOALLOC_MAX + 1
    with pytest.raises(H.HmatError) as e:
        H.hmat_rankmodel_grad_noalloc(M, np.zeros((n, F), np.float32), np.zeros(n, np.float32))
    assert e.value.status == H.HMAT_EINVAL and "HMAT_RANKGRAD_NOALLOC_MAX" in str(e.value)

"""The allocation-free gradient entry point, through the C-ABI: against the allocating call and
against the FP64 network of the oracle.

Some callers cannot allocate device memory while they fine-tune the rank model: code that runs
under a device-memory budget fixed up front, or code called from inside a custom allocator
hook, which must not re-enter the allocator. hmat_rankmodel_grad_noalloc serves them from one
fixed array compiled into the library.

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


def _model_and_samples(H, count):
    F, NP = H.RANK_FEATURES, H.RANK_PARAMS
    w = ((inputs.uniform01(71, NP) * 2.0 - 1.0) * 0.3).astype(np.float16).astype(np.float32)
    mean = (inputs.uniform01(72, F) - 0.5).astype(np.float32)
    dev = (inputs.uniform01(73, F) + 0.5).astype(np.float32)
    M = H.hmat_rankmodel_create(w, mean, dev)
    X = (inputs.uniform01(74 + count, count * F).reshape(count, F) * 4.0 - 2.0).astype(np.float32)
    r = np.floor(inputs.uniform01(75 + count, count) * 30.0).astype(np.float32)
    return M, w, mean, dev, X, r


@pytest.mark.parametrize("count", [777, 1])
def test_grad_noalloc_matches_grad(H, count):
    M, _, _, _, X, r = _model_and_samples(H, count)
    g_ref, l_ref = M.grad(X, r)
    for _ in range(2):  # two calls in a row: the accumulators start at zero each time
        g, l = H.hmat_rankmodel_grad_noalloc(M, X, r)
        assert np.abs(g - g_ref).max() <= 1e-5 * np.abs(g_ref).max()
        assert abs(l - l_ref) <= 1e-5 * l_ref


def test_grad_noalloc_matches_oracle_network(H):
    """The same call against the FP64 network of the oracle, on the standardised features (FP32,
    as the library computes them) and the FP64 targets: the bars of the network kernels' own
    parity test."""
    from oracle import rank_mlp as R
    M, w, mean, dev, X, r = _model_and_samples(H, 1003)
    Xs = ((X - mean) / dev).astype(np.float32).astype(np.float64)
    Lo, go = R.loss_grad(w.astype(np.float64), Xs, R.target(r))
    for _ in range(2):
        g, l = H.hmat_rankmodel_grad_noalloc(M, X, r)
        assert abs(l - Lo) <= 2e-5 * Lo
        assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()


def test_grad_noalloc_on_a_user_stream(H):
    """On a caller's non-blocking stream: the copies and kernels are ordered on that stream and
    the call has synchronised it when it returns. A NULL loss pointer is accepted."""
    import torch
    M, _, _, _, X, r = _model_and_samples(H, 500)
    g_ref, l_ref = M.grad(X, r)
    s = torch.cuda.Stream()
    for _ in range(2):
        g, l = H.hmat_rankmodel_grad_noalloc(M, X, r, stream=s)
        assert s.query()
        assert np.abs(g - g_ref).max() <= 1e-5 * np.abs(g_ref).max()
        assert abs(l - l_ref) <= 1e-5 * l_ref
    g, l = H.hmat_rankmodel_grad_noalloc(M, X, r, stream=s, want_loss=False)
    assert l is None and np.abs(g - g_ref).max() <= 1e-5 * np.abs(g_ref).max()


def test_grad_noalloc_rejects_oversize(H):
    F = H.RANK_FEATURES
    M = H.hmat_rankmodel_create(np.zeros(H.RANK_PARAMS, np.float32), np.zeros(F), np.ones(F))
    n = H.RANKGRAD_NOALLOC_MAX + 1
    with pytest.raises(H.HmatError) as e:
        H.hmat_rankmodel_grad_noalloc(M, np.zeros((n, F), np.float32), np.zeros(n, np.float32))
    assert e.value.status == H.HMAT_EINVAL and "HMAT_RANKGRAD_NOALLOC_MAX" in str(e.value)

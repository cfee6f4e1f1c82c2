"""The learned rank proposal: its network kernels against the FP64 oracle of the network, its
features against the tree and the restriction plan, training, and what the proposal buys in
the product (fewer sampling passes, the same accuracy bar)."""
import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs
from parity_util import _check_product, _oracle_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


@pytest.mark.parametrize("count", [1, 33, 1003])
def test_mlp_kernels_match_oracle(H, count):
    """Forward, loss and gradient of the FP16-weight / FP32-accumulation kernels against the FP64
    network on the same (FP16-representable) weights."""
    from oracle import rank_mlp as R
    w = ((inputs.uniform01(41, R.N_PARAMS) * 2.0 - 1.0) * 0.3).astype(np.float16).astype(np.float64)
    X = ((inputs.uniform01(42 + count, count * R.F).reshape(count, R.F) * 2.0 - 1.0) * 2.0).astype(np.float32)
    ranks = np.floor(inputs.uniform01(43 + count, count) * 40.0).astype(np.float32)
    M = H.hmat_rankmodel_create(w, np.zeros(R.F), np.ones(R.F))
    wg, mu, dv, _ = M.get()
    assert np.array_equal(wg.astype(np.float64), w)
    g, L = M.grad(X, ranks)
    Lo, go = R.loss_grad(w, X.astype(np.float64), R.target(ranks))
    assert abs(L - Lo) <= 2e-5 * Lo
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()
    np.testing.assert_allclose(M.predict(X), R.predicted_rank(R.forward(w, X.astype(np.float64))),
                               rtol=1e-4, atol=1e-3)


def test_rank_features_match_tree(H, oracle):
    P = inputs.points(0, 2, 2048, 0)
    A = H.hmat_build(P, 0, leaf_size=32, aca_eps=1e-10)
    B = H.hmat_build(P, 1, leaf_size=32, aca_eps=1e-10, tree_from=A)
    C = H.hmat_multiply(A, B, 1e-6)
    F, r = H.hmat_rank_features(A, B, 1e-6, C)
    T = oracle.Tree(P, 32, 1.0)
    la, lb, lc = H.leaf_arrays(A), H.leaf_arrays(B), H.leaf_arrays(C)
    far = np.nonzero(la.far)[0]
    assert F.shape == (len(far), H.RANK_FEATURES)
    lr, hp, _ = T.sumexpr_counts()
    rg = np.array([T.leaf_ranges(l) for l in far])
    np.testing.assert_allclose(F[:, 0], np.log2(rg[:, 1]), rtol=1e-6)
    np.testing.assert_allclose(F[:, 1], np.log2(rg[:, 3]), rtol=1e-6)
    assert np.array_equal(F[:, 2], T.leaf_blocks[far, 3])
    np.testing.assert_allclose(F[:, 5], np.log2(1.0 + lr[far]), rtol=1e-6)
    np.testing.assert_allclose(F[:, 6], np.log2(1.0 + hp[far]), rtol=1e-6)
    assert np.array_equal(F[:, 9], la.rank[far]) and np.array_equal(F[:, 10], lb.rank[far])
    assert np.all(F[:, 11] == np.float32(6.0))
    assert np.array_equal(r, lc.rank[far])
    # the largest term rank is at most the largest factor rank, and the sum is zero iff no terms
    assert F[:, 7].max() <= max(la.rank.max(), lb.rank.max())
    assert np.array_equal(F[:, 8] == 0, F[:, 5] == 0) and np.all(2.0 ** F[:, 8] - 1 >= F[:, 7] - 1e-3)
    # geometry: diameters of the two clusters' bounding boxes over their distance
    Pp = P[T.perm]
    for i in range(0, len(far), 11):
        r0, m, c0, n = rg[i]
        X, Y = Pp[r0:r0 + m], Pp[c0:c0 + n]
        gap = np.maximum(0.0, np.maximum(Y.min(0) - X.max(0), X.min(0) - Y.max(0)))
        dist = np.linalg.norm(gap)
        assert F[i, 3] == pytest.approx(np.linalg.norm(X.max(0) - X.min(0)) / dist, rel=1e-5)
        assert F[i, 4] == pytest.approx(np.linalg.norm(Y.max(0) - Y.min(0)) / dist, rel=1e-5)


@pytest.fixture(scope="module")
def trained(H):
    """A model trained on the products of two point sets at three tolerances."""
    feats, ranks = [], []
    for seed in (0, 1):
        P = inputs.points(0, 3, 3000, seed)
        A = H.hmat_build(P, 1, leaf_size=32, aca_eps=1e-10)
        for eps in (1e-4, 1e-6, 1e-8):
            C = H.hmat_multiply(A, A, eps, seed=seed)
            F, r = H.hmat_rank_features(A, A, eps, C)
            feats.append(F)
            ranks.append(r)
    X, y = np.concatenate(feats), np.concatenate(ranks)
    return H.hmat_rankmodel_train(X, y, epochs=1500, lr=3e-3, seed=7), X, y


def test_training_fits(H, trained):
    """Training lowers the loss well below the variance of the target, and the loss it reports
    is the FP64 network's loss at the weights it returns."""
    from oracle import rank_mlp as R
    M, X, y = trained
    w, mu, dv, loss = M.get()
    t = R.target(y)
    Xn = (X.astype(np.float64) - mu) / dv
    assert loss == pytest.approx(R.loss(w.astype(np.float64), Xn, t), rel=2e-3)
    assert loss <= 0.2 * np.var(t), (loss, np.var(t))
    pred = M.predict(X)
    assert np.median(np.abs(pred - y)) <= 2.0


def test_learned_proposal_parity_and_gain(H, oracle, trained):
    """On unseen points: with the learned proposal every far block still meets the bar (error
    <= 1.5 eps, rank <= eps-rank + 2) and the far blocks take fewer sampling passes than with
    the fixed first round."""
    M = trained[0]
    P = inputs.points(0, 3, 3000, 5)
    eps = 1e-6
    T, Ao, _ = _oracle_pair(oracle, P, 32, 1.0, 1, 1, 1e-10)
    A = H.hmat_build(P, 1, leaf_size=32, aca_eps=1e-10)
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    st = {}
    for prop in (H.PROP_NONE, H.PROP_LEARNED, H.PROP_HEURISTIC):
        C = H.hmat_multiply(A, A, eps, seed=9, rank_proposal=prop, rank_model=M if prop == H.PROP_LEARNED else None)
        assert C.last_status == H.HMAT_OK
        _check_product(oracle, T, C, DC, eps, near_rtol=1e-11)
        st[prop] = C.stats()
    s0, s1 = st[H.PROP_NONE], st[H.PROP_LEARNED]
    print({k: {f: v[f] for f in ("rounds", "sample_passes", "first_round_cols", "done_in_first_round", "ms_sample")}
           for k, v in st.items()})
    assert s1["done_in_first_round"] > s0["done_in_first_round"]
    # most blocks here have eps-ranks above what a 16-column first round can verify; the wider
    # first round still saves the third round of those
    assert s1["sample_passes"] <= 0.9 * s0["sample_passes"]
    assert s1["rounds"] <= s0["rounds"]


def test_proposal_invalid(H):
    P = inputs.points(0, 2, 500, 0)
    A = H.hmat_build(P, 0, leaf_size=16)
    with pytest.raises(H.HmatError) as e:
        H.hmat_multiply(A, A, 1e-6, rank_proposal=H.PROP_LEARNED)
    assert e.value.status == H.HMAT_EINVAL
    with pytest.raises(H.HmatError) as e:
        H.hmat_multiply(A, A, 1e-6, rank_proposal=5)
    assert e.value.status == H.HMAT_EINVAL
    with pytest.raises(H.HmatError) as e:
        H.hmat_rankmodel_create(np.zeros(H.RANK_PARAMS), np.zeros(H.RANK_FEATURES), np.zeros(H.RANK_FEATURES))
    assert e.value.status == H.HMAT_EINVAL

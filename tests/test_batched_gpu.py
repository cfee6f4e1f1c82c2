"""Batched products: 48 independent products of uneven size in one call (points uniform in
[0,1]^3, N_i = floor(4096 * 16^u_i) with u_i the splitmix64 uniforms of seed 1000, point seed
i, exp(-r), leaf 64, eta 1, FP32 factors by ACA to 1e-7, eps = 1e-5, MODE_MIXED). The larger
products run in subtree groups (their stored low-rank products alone take tens of GB). The eight
smallest must match the same products computed alone, and every product of the batch is checked
on sampled blocks (far blocks stratified by level, near blocks) against the oracle."""
import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs
from parity_util import check_sampled, sampled_far_near

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

EPS, ACA, LEAF = 1e-5, 1e-7, 64


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


@pytest.fixture(scope="module")
def batch(H):
    u = inputs.uniform01(1000, 48)
    sizes = np.floor(4096.0 * 16.0 ** u).astype(np.int64)
    pts = [inputs.points(inputs.PTS_CUBE, 3, int(n), i) for i, n in enumerate(sizes)]
    As = [H.hmat_build(P, H.K_EXP, leaf_size=LEAF, eta=1.0, aca_eps=ACA, factor_prec=32) for P in pts]
    Cs = H.hmat_multiply_batched(As, As, EPS, mode=H.MODE_MIXED, seed=3)
    return sizes, pts, As, Cs


def test_batched_matches_single(H, batch):
    sizes, pts, As, Cs = batch
    assert len(Cs) == 48 and all(C.last_status == H.HMAT_OK for C in Cs)
    assert sizes.min() >= 4096 and sizes.max() < 65536
    assert max(C.stats()["groups"] for C in Cs) > 1
    for i in np.argsort(sizes)[:8]:
        C1 = H.hmat_multiply(As[i], As[i], EPS, mode=H.MODE_MIXED, seed=3)
        la, lb = H.leaf_arrays(Cs[i]), H.leaf_arrays(C1)
        assert np.array_equal(la.far, lb.far)
        far = np.nonzero(la.far)[0]
        assert np.mean(la.rank[far] == lb.rank[far]) >= 0.95
        for l in far[:: max(1, len(far) // 16)]:
            (U, V), (U1, V1) = Cs[i].leaf_get(l), C1.leaf_get(l)
            M, M1 = U @ V.T, U1 @ V1.T
            assert np.linalg.norm(M - M1) <= 2 * EPS * np.linalg.norm(M1)


def test_batched_all_against_oracle(H, oracle, batch):
    sizes, pts, As, Cs = batch
    for i in np.argsort(sizes):
        T = oracle.Tree(pts[i], LEAF, 1.0)
        Ao = oracle.HMatrix(T, oracle.KERNEL_EXP, ACA, prec32=True)
        far, near = sampled_far_near(T, 8, 4, seed=int(i))
        check_sampled(oracle, T, Ao, Ao, Cs[i], EPS, 1.5 * EPS, far, near)


def test_batched_edge_cases(H):
    assert H.hmat_multiply_batched([], [], 1e-6) == []
    P = inputs.points(0, 2, 300, 0)
    A = H.hmat_build(P, 0, leaf_size=16)
    with pytest.raises(H.HmatError) as e:
        H.hmat_multiply_batched([A, A], [A, A], -1.0)
    assert e.value.status == H.HMAT_EINVAL

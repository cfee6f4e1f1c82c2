"""The learned rank proposal at scale: a network trained on ranks logged from smaller products
(the N = 2048 plane case, 3-D point sets of 4096-8192 points with exp(-r) and 1/(1+r^2)) sets
the first round of the product of N = 131072 points uniform in [0,1]^3 (seed 0), 1/(1+r^2),
leaf 64, eta 1, FP32 factors by ACA to 1e-8, eps = 1e-6, with the adaptive rounds as fallback.
Checked on sampled blocks against the oracle; the proposal must save sampling passes."""
import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs
from parity_util import check_sampled, sampled_far_near

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

EPS = 1e-6


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


@pytest.fixture(scope="module")
def model(H):
    feats, ranks = [], []
    cases = [(0, 2, 2048, 0, 32, H.K_EXP, (1e-6,)),
             (0, 3, 4096, 1, 64, H.K_EXP, (1e-5, 1e-6)),
             (0, 3, 8192, 2, 64, H.K_INVQ, (1e-5, 1e-6, 1e-7)),
             (0, 3, 6000, 3, 64, H.K_INVQ, (1e-6,))]
    for kind, dim, n, seed, leaf, kern, epss in cases:
        P = inputs.points(kind, dim, n, seed)
        A = H.hmat_build(P, kern, leaf_size=leaf, aca_eps=1e-8, factor_prec=32)
        for eps in epss:
            C = H.hmat_multiply(A, A, eps, mode=H.MODE_MIXED, seed=seed)
            F, r = H.hmat_rank_features(A, A, eps, C)
            feats.append(F)
            ranks.append(r)
    return H.hmat_rankmodel_train(np.concatenate(feats), np.concatenate(ranks), epochs=1500, lr=3e-3, seed=4)


def test_learned_proposal_n131072(H, oracle, model):
    P = inputs.points(inputs.PTS_CUBE, 3, 131072, 0)
    A = H.hmat_build(P, H.K_INVQ, leaf_size=64, eta=1.0, aca_eps=1e-8, factor_prec=32)
    C1 = H.hmat_multiply(A, A, EPS, mode=H.MODE_MIXED, seed=0, rank_proposal=H.PROP_LEARNED, rank_model=model)
    assert C1.last_status == H.HMAT_OK
    s1 = C1.stats()
    T = oracle.Tree(P, 64, 1.0)
    Ao = oracle.HMatrix(T, oracle.KERNEL_INVQ, 1e-8, prec32=True)
    far, near = sampled_far_near(T, 16, 4, seed=5, max_mn=128 * 128)
    worst = check_sampled(oracle, T, Ao, Ao, C1, EPS, 1.5 * EPS, far, near)
    C0 = H.hmat_multiply(A, A, EPS, mode=H.MODE_MIXED, seed=0)
    s0 = C0.stats()
    print({k: (s0[k], s1[k]) for k in ("sample_passes", "done_in_first_round", "rounds", "ms_sample", "groups")},
          f"worst {worst:.3g}")
    assert s1["done_in_first_round"] > s0["done_in_first_round"]
    assert s1["sample_passes"] < s0["sample_passes"]

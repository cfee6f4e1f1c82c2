"""Parity at the benchmark's full size on sampled blocks: the sphere workload (N = 32768 points
on S^2, A = exp(-r), B = 1/(1+r^2), leaf 64, eta 1, factors by ACA to 1e-8 stored in FP32,
eps = 1e-6) in the launch configuration the benchmark times, checked on far blocks stratified
by level and on near blocks against the oracle's exact blocks A|tau x I * B|I x sigma."""
import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs
from parity_util import check_sampled, sampled_far_near

pytestmark = pytest.mark.gpu

N, LEAF, ACA, EPS = 32768, 64, 1e-8, 1e-6


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


@pytest.fixture(scope="module")
def workload(H, oracle):
    P = inputs.points(inputs.PTS_SPHERE, 3, N, 0)
    T = oracle.Tree(P, LEAF, 1.0)
    Ao = oracle.HMatrix(T, oracle.KERNEL_EXP, ACA, prec32=True)
    Bo = oracle.HMatrix(T, oracle.KERNEL_INVQ, ACA, prec32=True)
    A = H.hmat_build(P, H.K_EXP, leaf_size=LEAF, eta=1.0, aca_eps=ACA, factor_prec=32)
    B = H.hmat_build(P, H.K_INVQ, leaf_size=LEAF, eta=1.0, aca_eps=ACA, factor_prec=32, tree_from=A)
    assert np.array_equal(A.permutation(), T.perm)
    return T, Ao, Bo, A, B


# Near blocks: FP32 contractions over N = 32768 inner indices leave relative errors of order
# sqrt(N) * 2^-24 ~ 1e-5 in single entries; the bar for a whole block is the product's own,
# 1.5 eps in relative Frobenius norm. The FP64 path is held to 1e-10.
@pytest.mark.parametrize("mode,near_rtol", [("mixed", 1.5 * EPS), ("f64", 1e-10)])
def test_sphere_n32768_sampled(H, oracle, workload, mode, near_rtol):
    T, Ao, Bo, A, B = workload
    md = H.MODE_MIXED if mode == "mixed" else H.MODE_F64
    C = H.hmat_multiply(A, B, EPS, mode=md, block_width=8, seed=0)
    assert C.last_status == H.HMAT_OK
    far, near = sampled_far_near(T, 48, 16, seed=7)
    worst = check_sampled(oracle, T, Ao, Bo, C, EPS, near_rtol, far, near)
    print(f"{mode}: {len(far)} far blocks, worst relative error {worst:.3g}; {len(near)} near blocks")

"""The H-matrix matvec (Alg. 2 over all leaves) against the dense matrix, and the paper's
estimator of a product's relative error (subspace iterations with C v - A (B v)) against the
exact error from the dense oracle product."""
import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs
from parity_util import _oracle_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


@pytest.mark.parametrize("prec,kind", [(64, 0), (32, 1)])
def test_matvec_matches_dense(H, prec, kind):
    P = inputs.points(inputs.PTS_CUBE, 2, 1200, 3)
    A = H.hmat_build(P, kind, leaf_size=32, aca_eps=1e-10, factor_prec=prec)
    D = A.to_dense()
    x = (inputs.uniform01(9, 1200 * 21).reshape(21, 1200).T - 0.5).copy()
    y = H.hmat_matvec(A, x)
    ref = D @ x
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    y1 = H.hmat_matvec(A, x[:, 4])
    assert np.abs(y1 - ref[:, 4]).max() <= 1e-12 * np.abs(ref[:, 4]).max()


def test_product_error_estimate(H, oracle):
    P = inputs.points(inputs.PTS_CUBE, 2, 2048, 0)
    T, Ao, _ = _oracle_pair(oracle, P, 32, 1.0, 0, 0, 1e-10)
    A = H.hmat_build(P, H.K_EXP, leaf_size=32, eta=1.0, aca_eps=1e-10)
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    perm = T.perm
    DCo = np.empty_like(DC)
    DCo[np.ix_(perm, perm)] = DC
    for eps in (1e-4, 1e-6):
        C = H.hmat_multiply(A, A, eps, seed=1)
        exact = np.linalg.norm(C.to_dense() - DCo) / np.linalg.norm(DCo)
        est = H.hmat_product_error(A, A, C, iters=10, size=100, seed=2)
        print(f"eps {eps}: estimate {est:.3g}, exact {exact:.3g}")
        # the block spans the dominant error directions: a lower estimate that captures most of it
        assert 0.3 * exact <= est <= 1.05 * exact

"""The H-matrix matvec (Alg. 2 over all leaves) against the dense matrix and the oracle, and the
paper's estimator of a product's relative error (subspace iterations with C v - A (B v), every
step on the device) against the exact error from the dense oracle product."""
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
    """Alg. 2 on the device against the library's own dense view of the same H-matrix (the
    matvec kernel is the only difference): agreement to rounding, for FP64 and FP32 factors."""
    P = inputs.points(inputs.PTS_CUBE, 2, 1200, 3)
    A = H.hmat_build(P, kind, leaf_size=32, aca_eps=1e-10, factor_prec=prec)
    D = A.to_dense()
    x = (inputs.uniform01(9, 1200 * 21).reshape(21, 1200).T - 0.5).copy()
    y = H.hmat_matvec(A, x)
    ref = D @ x
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    y1 = H.hmat_matvec(A, x[:, 4])
    assert np.abs(y1 - ref[:, 4]).max() <= 1e-12 * np.abs(ref[:, 4]).max()


@pytest.mark.parametrize("kind,dim,n,leaf,eta", [(0, 2, 1500, 32, 1.0), (1, 3, 1200, 16, 1.0), (0, 2, 700, 16, 1e-9)])
def test_matvec_matches_oracle(H, oracle, kind, dim, n, leaf, eta):
    """Alg. 2 on the device against the oracle's dense H-matrix on the same points, built by the
    oracle's own tree and ACA (to 1e-14, so that the two sides' far factors agree far below the
    bar), and, for eta -> 0 (no far blocks: every leaf dense and exact), against the kernel
    matrix evaluated entry by entry."""
    P = inputs.points(kind, dim, n, 5)
    T = oracle.Tree(P, leaf, eta)
    Ao = oracle.HMatrix(T, oracle.KERNEL_EXP, 1e-14)
    D = np.empty((n, n))
    D[np.ix_(T.perm, T.perm)] = Ao.dense()   # original point order
    A = H.hmat_build(P, H.K_EXP, leaf_size=leaf, eta=eta, aca_eps=1e-14)
    x = (inputs.uniform01(17, n * 10).reshape(10, n).T - 0.5).copy()
    y = H.hmat_matvec(A, x)
    ref = D @ x
    assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max()
    if eta < 1e-6:
        K = np.exp(-np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)))
        assert np.abs(y - K @ x).max() <= 1e-12 * np.abs(K @ x).max()


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
    # the exact product (eta -> 0: every block dense and exact) has no error to find
    A0 = H.hmat_build(P[:600], H.K_EXP, leaf_size=32, eta=1e-9)
    C0 = H.hmat_multiply(A0, A0, 1e-6)
    assert H.hmat_product_error(A0, A0, C0, iters=3, size=20, seed=4) <= 1e-13
    with pytest.raises(H.HmatError) as e:
        H.hmat_product_error(A0, A0, C0, iters=1, size=129, seed=4)
    assert e.value.status == H.HMAT_EINVAL

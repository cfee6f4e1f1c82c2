"""A product run in groups (a memory budget forces the block tree to be cut into subtrees that
run one after another) against the full dense oracle: the same bar as a product in one pass."""
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


# FP32 near blocks: entries are sums over N = 3000 inner indices, relative error up to about
# sqrt(N) * 2^-24 ~ 3.3e-6 of the block's largest entry
@pytest.mark.parametrize("mode,near_rtol", [("f64", 1e-11), ("mixed", 4e-6)])
def test_grouped_product_dense_oracle(H, oracle, monkeypatch, mode, near_rtol):
    P = inputs.points(inputs.PTS_CUBE, 3, 3000, 4)
    prec = 64 if mode == "f64" else 32
    T, Ao, _ = _oracle_pair(oracle, P, 32, 1.0, 0, 0, 1e-10, prec32=(prec == 32))
    A = H.hmat_build(P, H.K_EXP, leaf_size=32, eta=1.0, aca_eps=1e-10, factor_prec=prec)
    md = H.MODE_F64 if mode == "f64" else H.MODE_MIXED
    monkeypatch.setenv("HMAT_MEMORY_BUDGET_GB", "0.05")
    C = H.hmat_multiply(A, A, 1e-6, mode=md, seed=2)
    monkeypatch.delenv("HMAT_MEMORY_BUDGET_GB")
    assert C.last_status == H.HMAT_OK
    assert C.stats()["groups"] > 1
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    _check_product(oracle, T, C, DC, 1e-6, near_rtol=near_rtol)
    # the same product in one pass agrees with the grouped one block by block
    C1 = H.hmat_multiply(A, A, 1e-6, mode=md, seed=2)
    la, lb = H.leaf_arrays(C), H.leaf_arrays(C1)
    assert np.array_equal(la.far, lb.far) and np.mean(la.rank == lb.rank) >= 0.95

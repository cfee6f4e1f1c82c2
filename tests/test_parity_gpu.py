"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Bars (from the method's statement of the result):
  * integer / index work bit-exact: cluster permutation, leaf geometry, sum-expression counts;
  * every far block of C = A B within relative Frobenius error 1.5 * eps of the exact block of
    the product of the stored inputs, with rank <= eps-rank + 2;
  * near blocks equal the exact product block to rounding, measured as the largest entry error
    relative to the block's largest entry: 1e-11 in FP64 (the two sides sum up to N products
    per entry in different orders, and an entry much smaller than the block's largest carries
    that rounding too), 2e-6 with FP32 contractions.
The oracle builds its own A and B from the same seeded points (its own trees and ACA); the
two sides' inputs differ by at most rounding of the same ACA steps, far below eps.
"""
import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs
from parity_util import _check_product, _check_structure, _gpu_pair, _oracle_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


def test_build_parity(H, oracle):
    """Tree, permutation and leaf geometry bit-exact; near leaves equal to rounding; far leaves
    agree with the oracle's ACA to the ACA tolerance."""
    P = inputs.points(0, 2, 1000, 7)
    T, A, _ = _oracle_pair(oracle, P, 16, 1.0, 0, 0, 1e-10)
    G = H.hmat_build(P, 0, leaf_size=16, eta=1.0, aca_eps=1e-10)
    la = _check_structure(H, T, G)
    same_rank = 0
    for l in range(T.nleaf):
        if la.far[l]:
            U, V = G.leaf_get(l)
            Uo, Vo = A.leaf(l)
            ref = Uo @ Vo.T
            assert np.linalg.norm(U @ V.T - ref) <= 1e-8 * np.linalg.norm(ref)
            same_rank += int(U.shape[1] == Uo.shape[1])
        else:
            assert np.abs(G.leaf_get(l) - A.leaf(l)).max() <= 4e-16
    assert same_rank >= 0.95 * la.far.sum()
    st = G.stats()
    assert st["n_far"] == la.far.sum() and st["csp"] == T.csp()


def test_sumexpr_counts_bit_exact(H, oracle):
    """a1: the library's restriction plan (Algorithm 3) has, for every leaf, exactly the oracle's
    number of low-rank terms and H-pairs."""
    for kind, dim, n, leaf in [(0, 2, 2048, 32), (1, 3, 3000, 32), (0, 3, 1531, 16)]:
        P = inputs.points(kind, dim, n, 1)
        T = oracle.Tree(P, leaf, 1.0)
        G = H.hmat_build(P, 0, leaf_size=leaf, eta=1.0, aca_eps=1e-6)
        lr, hp = H.hmat_sumexpr_counts(G, G)
        lr_o, hp_o, _ = T.sumexpr_counts()
        assert np.array_equal(lr, lr_o) and np.array_equal(hp, hp_o)


@pytest.mark.parametrize("kind,dim,n,leaf,kA,kB,eps", [
    (0, 2, 512, 16, 0, 0, 1e-6),
    (0, 2, 777, 16, 0, 1, 1e-6),     # ragged size, two kernels
    (1, 3, 1200, 32, 0, 1, 1e-6),    # sphere
    (0, 3, 1000, 32, 1, 1, 1e-4),
    (0, 2, 1000, 16, 0, 0, 1e-8),
])
def test_multiply_f64_dense_oracle(H, oracle, kind, dim, n, leaf, kA, kB, eps):
    P = inputs.points(kind, dim, n, 3)
    T, Ao, Bo = _oracle_pair(oracle, P, leaf, 1.0, kA, kB, 1e-12)
    A, B = _gpu_pair(H, P, leaf, 1.0, kA, kB, 1e-12)
    C = H.hmat_multiply(A, B, eps, mode=H.MODE_F64, seed=11)
    assert C.last_status == H.HMAT_OK
    _check_structure(H, T, C)
    DC = oracle.matmul(Ao.dense(), Bo.dense())
    worst, worst_near, nf = _check_product(oracle, T, C, DC, eps, near_rtol=1e-11)
    assert nf > 0


def test_multiply_config_n2048(H, oracle):
    """The N=2048 case: U[0,1]^2 (seed 0), exp(-r), leaf 32, eta 1, A = B by ACA to 1e-10,
    eps = 1e-6, every block against the full dense oracle."""
    P = inputs.points(0, 2, 2048, 0)
    T, Ao, _ = _oracle_pair(oracle, P, 32, 1.0, 0, 0, 1e-10)
    A = H.hmat_build(P, 0, leaf_size=32, eta=1.0, aca_eps=1e-10)
    C = H.hmat_multiply(A, A, 1e-6, mode=H.MODE_F64, seed=0)
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    worst, worst_near, nf = _check_product(oracle, T, C, DC, 1e-6, near_rtol=1e-11)
    assert nf == int((T.leaf_blocks[:, 2] == 1).sum())
    # Thm. 4.1: the global relative error follows from the blockwise bound
    Cd = C.to_dense()
    perm = T.perm
    DCo = np.empty_like(DC)
    DCo[np.ix_(perm, perm)] = DC
    assert np.linalg.norm(Cd - DCo) <= 1.5e-6 * np.linalg.norm(DCo)


@pytest.mark.parametrize("kind,dim,n,leaf,kA,kB,eps", [
    (0, 2, 2048, 32, 0, 0, 1e-10),
    (0, 2, 2048, 32, 0, 0, 1e-12),   # the truncation tolerance of the paper's experiments (Sec. 6)
    (1, 3, 1500, 32, 0, 1, 1e-12),   # sphere, two kernels
])
def test_multiply_f64_paper_eps(H, oracle, kind, dim, n, leaf, kA, kB, eps):
    """Every block against the full dense oracle at eps down to 1e-12, where the eps-tail
    (eps^2 = 1e-24 of a block's energy) lies far below the rounding of a Gram matrix of W.
    Both sides build their inputs by ACA to 1e-14, so the two sides' inputs agree far below eps."""
    P = inputs.points(kind, dim, n, 0)
    T, Ao, Bo = _oracle_pair(oracle, P, leaf, 1.0, kA, kB, 1e-14)
    A, B = _gpu_pair(H, P, leaf, 1.0, kA, kB, 1e-14)
    C = H.hmat_multiply(A, B, eps, mode=H.MODE_F64, seed=0)
    assert C.last_status == H.HMAT_OK
    DC = oracle.matmul(Ao.dense(), Bo.dense())
    worst, worst_near, nf = _check_product(oracle, T, C, DC, eps, near_rtol=1e-11)
    assert nf == int((T.leaf_blocks[:, 2] == 1).sum())
    print(f"eps {eps}: {nf} far blocks, worst relative error {worst / eps:.3f} eps, "
          f"largest rank {H.leaf_arrays(C).rank.max()}")


def test_multiply_mixed_fp32(H, oracle):
    """FP32 factors and FP32 contractions, FP64 orthogonalisation and core truncation,
    against the oracle on the same FP32-rounded inputs."""
    P = inputs.points(1, 3, 1500, 0)
    T, Ao, Bo = _oracle_pair(oracle, P, 32, 1.0, 0, 1, 1e-8, prec32=True)
    A, B = _gpu_pair(H, P, 32, 1.0, 0, 1, 1e-8, prec=32)
    C = H.hmat_multiply(A, B, 1e-6, mode=H.MODE_MIXED, seed=5)
    assert C.stats()["factor_prec"] == 32
    DC = oracle.matmul(Ao.dense(), Bo.dense())
    _check_product(oracle, T, C, DC, 1e-6, near_rtol=2e-6)


def test_multiply_f64_on_fp32_inputs(H, oracle):
    """mode F64 on FP32-stored inputs widens them exactly and computes in FP64."""
    P = inputs.points(0, 2, 700, 4)
    T, Ao, _ = _oracle_pair(oracle, P, 16, 1.0, 0, 0, 1e-8, prec32=True)
    A = H.hmat_build(P, 0, leaf_size=16, eta=1.0, aca_eps=1e-8, factor_prec=32)
    C = H.hmat_multiply(A, A, 1e-7, mode=H.MODE_F64)
    assert C.stats()["factor_prec"] == 64
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    _check_product(oracle, T, C, DC, 1e-7, near_rtol=1e-11)


def test_separable_kernel_closed_form(H, oracle):
    """(1 + x.y)^2 in 2-D: every product block has rank <= 6; at eps = 1e-10 the GPU returns
    rank <= 6 (+2 slack) with error below 1.5 eps."""
    P = inputs.points(0, 2, 600, 2)
    T, Ao, _ = _oracle_pair(oracle, P, 16, 1.0, 2, 2, 1e-13)
    A = H.hmat_build(P, 2, leaf_size=16, eta=1.0, aca_eps=1e-13)
    C = H.hmat_multiply(A, A, 1e-10, mode=H.MODE_F64)
    la = H.leaf_arrays(C)
    assert la.rank[la.far == 1].max() <= 8
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    _check_product(oracle, T, C, DC, 1e-10, near_rtol=1e-11)


def test_edge_cases(H, oracle):
    # n <= leaf size: the root is a near leaf; C is the dense product
    P = inputs.points(0, 2, 20, 1)
    A = H.hmat_build(P, 0, leaf_size=32)
    C = H.hmat_multiply(A, A, 1e-6)
    Pp = P
    K = np.exp(-np.sqrt(((Pp[:, None] - Pp[None]) ** 2).sum(-1)))
    assert np.abs(C.to_dense() - K @ K).max() <= 1e-12 * np.abs(K @ K).max()
    # a single point
    P1 = inputs.points(0, 3, 1, 0)
    A1 = H.hmat_build(P1, 1, leaf_size=4)
    assert abs(H.hmat_multiply(A1, A1, 1e-6).to_dense()[0, 0] - 1.0) <= 1e-15
    # eta -> 0: no far blocks, exact product
    P = inputs.points(0, 2, 300, 2)
    A = H.hmat_build(P, 0, leaf_size=16, eta=1e-9)
    C = H.hmat_multiply(A, A, 1e-6)
    assert C.stats()["n_far"] == 0
    K = np.exp(-np.sqrt(((P[:, None] - P[None]) ** 2).sum(-1)))
    assert np.abs(C.to_dense() - K @ K).max() <= 1e-11 * np.abs(K @ K).max()
    # a coarse eps keeps tiny ranks and still meets the bound
    P = inputs.points(0, 2, 800, 5)
    T, Ao, _ = _oracle_pair(oracle, P, 16, 1.0, 0, 0, 1e-10)
    A = H.hmat_build(P, 0, leaf_size=16, aca_eps=1e-10)
    C = H.hmat_multiply(A, A, 0.3)
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    _check_product(oracle, T, C, DC, 0.3, near_rtol=1e-11)


def test_rank_cap_reports_notconv(H):
    """A rank cap below the eps-rank ends with HMAT_ENOTCONV and a complete, usable C."""
    P = inputs.points(0, 2, 1024, 0)
    A = H.hmat_build(P, 0, leaf_size=32, aca_eps=1e-12)
    C = H.hmat_multiply(A, A, 1e-12, max_rank=8, block_width=8)
    assert C.last_status == H.HMAT_ENOTCONV
    st = C.stats()
    assert st["not_converged"] > 0 and st["max_rank"] <= 8
    with pytest.raises(H.HmatError) as e:
        H.hmat_multiply(A, A, 1e-12, max_rank=8, block_width=8, allow_notconv=False)
    assert e.value.status == H.HMAT_ENOTCONV


def test_mismatch_and_invalid(H):
    P = inputs.points(0, 2, 300, 0)
    Q = inputs.points(0, 2, 300, 1)
    A = H.hmat_build(P, 0, leaf_size=16)
    B = H.hmat_build(Q, 0, leaf_size=16)
    with pytest.raises(H.HmatError) as e:
        H.hmat_multiply(A, B, 1e-6)
    assert e.value.status == H.HMAT_EMISMATCH
    with pytest.raises(H.HmatError) as e:
        H.hmat_build(Q, 1, leaf_size=16, tree_from=A)
    assert e.value.status == H.HMAT_EMISMATCH
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(H.HmatError) as e:
            H.hmat_multiply(A, A, bad)
        assert e.value.status == H.HMAT_EINVAL
    # same points built twice: same tree, product allowed
    A2 = H.hmat_build(P, 1, leaf_size=16)
    H.hmat_multiply(A, A2, 1e-6)


def test_reproducible(H):
    """Two products with the same seed agree on what is unique: the blocks U V^T (the factors
    themselves are not unique, and the FP32 sums are accumulated in varying order) and, but for
    ties at the truncation threshold, the ranks."""
    P = inputs.points(1, 3, 1500, 3)
    A = H.hmat_build(P, 0, leaf_size=32, aca_eps=1e-8, factor_prec=32)
    C1 = H.hmat_multiply(A, A, 1e-6, mode=H.MODE_MIXED, seed=3)
    C2 = H.hmat_multiply(A, A, 1e-6, mode=H.MODE_MIXED, seed=3)
    same = total = 0
    for l in range(0, C1.leaf_count(), 3):
        a, b = C1.leaf_get(l), C2.leaf_get(l)
        if isinstance(a, tuple):
            Ma, Mb = a[0] @ a[1].T, b[0] @ b[1].T
            assert np.linalg.norm(Ma - Mb) <= 3e-6 * np.linalg.norm(Ma)
            same += int(a[0].shape[1] == b[0].shape[1])
            total += 1
        else:
            assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
    assert same >= 0.98 * total

"""The compressors of sum-expressions that work one vector at a time -- cross approximation
(Algorithm 6, then a QR of L and the eps truncation) and Lanczos bidiagonalization (Algorithm 7
with full reorthogonalization, then the truncation of Q (S^T Q)^T) -- against the dense oracle
product: every far block within 1.5 eps of the exact block with rank at most k_eps + 2, near
blocks exact, in FP64 and in the FP32 mixed mode, on one grouped (memory-bounded) product and in
a batch."""
import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs
from parity_util import _check_product, _gpu_pair, _oracle_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


COMPRESSORS = ["aca", "lanczos"]


def _comp(H, name):
    return {"aca": H.COMP_ACA, "lanczos": H.COMP_LANCZOS}[name]


@pytest.mark.parametrize("comp", COMPRESSORS)
def test_n2048_f64(H, oracle, comp):
    """U[0,1]^2 (seed 0), exp(-r), leaf 32, A = B by ACA to 1e-10, eps = 1e-6, FP64."""
    P = inputs.points(0, 2, 2048, 0)
    T, Ao, _ = _oracle_pair(oracle, P, 32, 1.0, 0, 0, 1e-10)
    A = H.hmat_build(P, 0, leaf_size=32, eta=1.0, aca_eps=1e-10)
    C = H.hmat_multiply(A, A, 1e-6, mode=H.MODE_F64, compressor=_comp(H, comp))
    assert C.last_status == H.HMAT_OK
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    worst, _, nf = _check_product(oracle, T, C, DC, 1e-6, near_rtol=1e-11)
    assert nf == int((T.leaf_blocks[:, 2] == 1).sum())
    st = C.stats()
    # one step per cross or Lanczos step: at least two per block (the stop needs two that pass)
    assert st["sample_passes"] >= 2 * nf
    Cd = C.to_dense()
    perm = T.perm
    DCo = np.empty_like(DC)
    DCo[np.ix_(perm, perm)] = DC
    assert np.linalg.norm(Cd - DCo) <= 1.5e-6 * np.linalg.norm(DCo)


def test_aca_steps_match_oracle(H, oracle):
    """The device cross approximation takes the oracle's steps: on the N = 2048 FP64 product the
    crosses summed over all far blocks (the library's sample_passes) match those of the oracle's
    Algorithm 6 run on the exact dense blocks with the same pivoting and stop rule (two
    consecutive crosses at eps/8); a pivot can differ only where two entries tie to rounding."""
    from oracle import compressors as X
    P = inputs.points(0, 2, 2048, 0)
    T, Ao, _ = _oracle_pair(oracle, P, 32, 1.0, 0, 0, 1e-10)
    A = H.hmat_build(P, 0, leaf_size=32, eta=1.0, aca_eps=1e-10)
    eps = 1e-6
    C = H.hmat_multiply(A, A, eps, mode=H.MODE_F64, compressor=H.COMP_ACA)
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    total = 0
    for l in range(T.nleaf):
        if T.leaf_blocks[l, 2] == 1:
            r0, m, c0, n = T.leaf_ranges(l)
            total += X.aca(DC[r0:r0 + m, c0:c0 + n], eps / 8, 95)[2]
    assert abs(C.stats()["sample_passes"] - total) <= 0.01 * total, (C.stats()["sample_passes"], total)


@pytest.mark.parametrize("comp", COMPRESSORS)
@pytest.mark.parametrize("eps", [1e-4, 1e-8])
def test_3d_two_kernels(H, oracle, eps, comp):
    """U[0,1]^3 (seed 5), A = exp(-r), B = 1/(1+r^2): the 3-D blocks on which a single
    eq. (truncaca) test at eps/4 stops early on some blocks."""
    P = inputs.points(0, 3, 3000, 5)
    T, Ao, Bo = _oracle_pair(oracle, P, 32, 1.0, 0, 1, 1e-10)
    A, B = _gpu_pair(H, P, 32, 1.0, 0, 1, 1e-10)
    C = H.hmat_multiply(A, B, eps, mode=H.MODE_F64, compressor=_comp(H, comp))
    DC = oracle.matmul(Ao.dense(), Bo.dense())
    _check_product(oracle, T, C, DC, eps, near_rtol=1e-11)


@pytest.mark.parametrize("comp", COMPRESSORS)
def test_mixed_fp32(H, oracle, comp):
    """FP32 factors and contractions (rows and columns of S in FP32), FP64 cross updates, QR and
    core truncation, against the oracle on the same FP32-rounded inputs."""
    P = inputs.points(1, 3, 1500, 0)
    T, Ao, Bo = _oracle_pair(oracle, P, 32, 1.0, 0, 1, 1e-8, prec32=True)
    A, B = _gpu_pair(H, P, 32, 1.0, 0, 1, 1e-8, prec=32)
    C = H.hmat_multiply(A, B, 1e-6, mode=H.MODE_MIXED, compressor=_comp(H, comp))
    assert C.last_status == H.HMAT_OK
    DC = oracle.matmul(Ao.dense(), Bo.dense())
    _check_product(oracle, T, C, DC, 1e-6, near_rtol=2e-6)


@pytest.mark.parametrize("comp", COMPRESSORS)
def test_closed_forms(H, oracle, comp):
    """(1 + x.y)^2 in 2-D: every product block has rank <= 6, so the crosses (or the Krylov
    space) exhaust it and the blocks come out at rank <= 6 (+2) to 1e-10; a coarse eps keeps tiny
    ranks within bound."""
    P = inputs.points(0, 2, 600, 2)
    T, Ao, _ = _oracle_pair(oracle, P, 16, 1.0, 2, 2, 1e-13)
    A = H.hmat_build(P, 2, leaf_size=16, eta=1.0, aca_eps=1e-13)
    C = H.hmat_multiply(A, A, 1e-10, mode=H.MODE_F64, compressor=_comp(H, comp))
    la = H.leaf_arrays(C)
    assert la.rank[la.far == 1].max() <= 8
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    _check_product(oracle, T, C, DC, 1e-10, near_rtol=1e-11)
    P = inputs.points(0, 2, 800, 5)
    T, Ao, _ = _oracle_pair(oracle, P, 16, 1.0, 0, 0, 1e-10)
    A = H.hmat_build(P, 0, leaf_size=16, aca_eps=1e-10)
    C = H.hmat_multiply(A, A, 0.3, compressor=_comp(H, comp))
    DC = oracle.matmul(Ao.dense(), Ao.dense())
    _check_product(oracle, T, C, DC, 0.3, near_rtol=1e-11)


@pytest.mark.parametrize("comp", COMPRESSORS)
def test_cap_and_invalid(H, comp):
    """A rank cap below the eps-rank ends with HMAT_ENOTCONV (ranks <= max_rank - 1: the cross
    approximation keeps the used-row flags in the last basis column, Lanczos the next w there);
    neither compressor takes fixed_rank or a rank proposal."""
    P = inputs.points(0, 2, 1024, 0)
    A = H.hmat_build(P, 0, leaf_size=32, aca_eps=1e-12)
    C = H.hmat_multiply(A, A, 1e-12, max_rank=8, compressor=_comp(H, comp))
    assert C.last_status == H.HMAT_ENOTCONV
    st = C.stats()
    assert st["not_converged"] > 0 and st["max_rank"] <= 7
    for kw in ({"fixed_rank": 4}, {"rank_proposal": 2}, {"compressor": 3}, {"compressor": -1}):
        args = {"compressor": _comp(H, comp), **kw}
        with pytest.raises(H.HmatError) as e:
            H.hmat_multiply(A, A, 1e-6, **args)
        assert e.value.status == H.HMAT_EINVAL


@pytest.mark.parametrize("comp", COMPRESSORS)
def test_batched_matches_single(H, comp):
    """Three products in one batched call give the blocks of three single calls (the same seed
    draws the same Lanczos start vectors), but sums accumulated by atomics may round differently
    and move a pivot or a stop, so the blocks agree to the sum of the two results' bounds
    (3 eps), ranks mostly exactly."""
    As, Bs = [], []
    for i, n in enumerate((900, 1300, 700)):
        P = inputs.points(0, 3, n, 40 + i)
        A, B = _gpu_pair(H, P, 32, 1.0, 0, 1, 1e-9)
        As.append(A)
        Bs.append(B)
    Cb = H.hmat_multiply_batched(As, Bs, 1e-6, compressor=_comp(H, comp))
    same = total = 0
    for A, B, C in zip(As, Bs, Cb):
        Cs = H.hmat_multiply(A, B, 1e-6, compressor=_comp(H, comp))
        for l in range(Cs.leaf_count()):
            a, b = Cs.leaf_get(l), C.leaf_get(l)
            if isinstance(a, tuple):
                Ma, Mb = a[0] @ a[1].T, b[0] @ b[1].T
                assert np.linalg.norm(Ma - Mb) <= 3e-6 * np.linalg.norm(Ma)
                same += int(a[0].shape[1] == b[0].shape[1])
                total += 1
            else:
                assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    assert same >= 0.95 * total


@pytest.mark.parametrize("comp", COMPRESSORS)
def test_grouped(H, oracle, monkeypatch, comp):
    """A memory budget that splits the product into groups: every group runs its own steps; the
    blocks still meet the bound."""
    P = inputs.points(0, 3, 3000, 1)
    T, Ao, Bo = _oracle_pair(oracle, P, 32, 1.0, 0, 1, 1e-10)
    A, B = _gpu_pair(H, P, 32, 1.0, 0, 1, 1e-10)
    monkeypatch.setenv("HMAT_MEMORY_BUDGET_GB", "0.05")
    C = H.hmat_multiply(A, B, 1e-6, compressor=_comp(H, comp))
    monkeypatch.delenv("HMAT_MEMORY_BUDGET_GB")
    assert C.stats()["groups"] > 1
    DC = oracle.matmul(Ao.dense(), Bo.dense())
    _check_product(oracle, T, C, DC, 1e-6, near_rtol=1e-11)

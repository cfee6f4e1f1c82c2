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


@pytest.fixture(scope="module")
def largest_blocks(workload, oracle):
    """Sixteen of the far blocks of the top size class (1024 x 1024, level 5; 180 of them), chosen
    with a seeded generator, and the oracle's exact blocks A|tau x I * B|I x sigma."""
    T, Ao, Bo, _, _ = workload
    sizes = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    far = np.nonzero(T.leaf_blocks[:, 2] == 1)[0]
    top = far[sizes[far, 1] == sizes[far, 1].max()]
    assert sizes[top[0], 1] >= 1024 and len(top) >= 16
    pick = np.random.default_rng(5).choice(top, size=16, replace=False)
    blocks = {}
    for l in pick.tolist():
        r0, m, c0, n = T.leaf_ranges(l)
        blocks[l] = oracle.block_product_blas(Ao, Bo, r0, m, c0, n)
    return blocks


@pytest.mark.parametrize("mode", ["mixed", "f64"])
def test_sphere_n32768_largest_blocks(H, oracle, workload, largest_blocks, mode):
    """The largest far blocks, whose sum-expressions carry the most terms (Lemma 5.3), against the
    oracle at 1.5 eps and rank <= eps-rank + 2, in the launch configuration the benchmark times.
    Mixed form: the 1024-row targets' applications are split over several thread blocks each
    (the per-class counts of the product say so). FP64 path: their panels do not fit in shared
    memory and are staged in global memory."""
    T, Ao, Bo, A, B = workload
    md = H.MODE_MIXED if mode == "mixed" else H.MODE_F64
    C = H.hmat_multiply(A, B, EPS, mode=md, block_width=8, seed=0)
    assert C.last_status == H.HMAT_OK
    st = C.stats()
    if mode == "mixed":
        assert st["apply_split_targets"] >= len(largest_blocks) and st["apply_max_split"] >= 4, st
    else:
        assert st["apply_gstage_targets"] >= 180, st
    # the unique bytes of the passes are at most their per-use bytes, and include the panels
    assert 0 < st["bytes_apply_unique"] <= st["bytes_apply_use"]
    worst = 0.0
    for l, blk in largest_blocks.items():
        U, V = C.leaf_get(l)
        nb = np.linalg.norm(blk)
        err = np.linalg.norm(blk - U @ V.T) / nb
        tr = oracle.truth_for_block(blk, EPS, l)
        assert err <= 1.5 * EPS, (l, err, U.shape[1], tr.k_eps)
        assert U.shape[1] <= tr.k_eps + 2, (l, U.shape[1], tr.k_eps)
        # Eckart-Young: no rank-k approximation beats the singular-value tail at k
        assert err * nb >= np.sqrt(np.sum(tr.s[U.shape[1]:] ** 2)) * (1 - 1e-3) - 1e-13 * nb
        worst = max(worst, err)
    print(f"{mode}: {len(largest_blocks)} blocks of {U.shape[0]} rows, worst relative error {worst / EPS:.3f} eps; "
          f"split targets {st['apply_split_targets']} (max {st['apply_max_split']}), "
          f"global-staging targets {st['apply_gstage_targets']}, "
          f"unique/use bytes {st['bytes_apply_unique'] / st['bytes_apply_use']:.3f}")

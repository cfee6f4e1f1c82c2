"""The large sweep: N = 524288 points on S^2 (seed 0), exp(-r), leaf 64, eta 1, factors by ACA
to 1e-8 stored in FP32, C = A A at eps = 1e-4 and 1e-6 (FP32 contractions) and 1e-8 (the FP64
path on the same inputs). The product runs in subtree groups (its device memory estimate is
about 0.5 TB). Checked on sampled blocks against the oracle's exact blocks A|tau x I * A|I x sigma,
computed once and reused for the three tolerances."""
import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, LEAF, ACA = 524288, 64, 1e-8
# 256 far blocks stratified by level (the block sizes are 512, 256, 128 and 64 rows: exact
# oracle blocks cost 2 m n N flops each, so the larger levels get fewer) and 16 near blocks
PER_LEVEL = {10: 4, 11: 12, 12: 120, 13: 120}
N_NEAR = 16


def sample_levels(T, per_level, n_near, seed):
    rng = np.random.default_rng(seed)
    lv, kind = T.leaf_blocks[:, 3], T.leaf_blocks[:, 2]
    far = []
    for level, k in sorted(per_level.items()):
        cand = np.nonzero((lv == level) & (kind == 1))[0]
        far += rng.choice(cand, size=min(k, len(cand)), replace=False).tolist()
    near = rng.choice(np.nonzero(kind != 1)[0], size=n_near, replace=False).tolist()
    return far, near


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


@pytest.fixture(scope="module")
def sweep(H, oracle):
    P = inputs.points(inputs.PTS_SPHERE, 3, N, 0)
    T = oracle.Tree(P, LEAF, 1.0)
    Ao = oracle.HMatrix(T, oracle.KERNEL_EXP, ACA, prec32=True)
    A = H.hmat_build(P, H.K_EXP, leaf_size=LEAF, eta=1.0, aca_eps=ACA, factor_prec=32)
    assert np.array_equal(A.permutation(), T.perm)
    far, near = sample_levels(T, PER_LEVEL, N_NEAR, seed=11)
    blocks = {}
    for l in far + near:
        r0, m, c0, n = T.leaf_ranges(l)
        blocks[l] = oracle.block_product_blas(Ao, Ao, r0, m, c0, n)
    return T, A, far, near, blocks


@pytest.mark.parametrize("eps,mode,near_rtol", [(1e-4, "mixed", 1.5e-4), (1e-6, "mixed", 1.5e-6),
                                                 (1e-8, "f64", 1e-10)])
def test_sweep_n524288(H, oracle, sweep, eps, mode, near_rtol):
    T, A, far, near, blocks = sweep
    assert len(far) == sum(PER_LEVEL.values()) == 256
    C = H.hmat_multiply(A, A, eps, mode=H.MODE_MIXED if mode == "mixed" else H.MODE_F64, seed=1)
    assert C.last_status == H.HMAT_OK
    assert C.stats()["groups"] > 1
    worst = 0.0
    for l in far:
        blk = blocks[l]
        U, V = C.leaf_get(l)
        nb = np.linalg.norm(blk)
        err = np.linalg.norm(blk - U @ V.T) / nb
        tr = oracle.truth_for_block(blk, eps, l)
        assert err <= 1.5 * eps, (l, err, U.shape[1], tr.k_eps)
        assert U.shape[1] <= tr.k_eps + 2, (l, U.shape[1], tr.k_eps)
        worst = max(worst, err)
    for l in near:
        D = C.leaf_get(l)
        e = np.linalg.norm(D - blocks[l]) / np.linalg.norm(blocks[l])
        assert e <= near_rtol, (l, e)
    print(f"eps {eps} {mode}: {len(far)} far blocks, worst relative error {worst:.3g}")
    if eps == 1e-6:  # the paper's global check (Sec. 6): subspace iterations on C v - A (A v)
        est = H.hmat_product_error(A, A, C, iters=10, size=100, seed=3)
        print(f"eps {eps}: estimated global relative error {est:.3g}")
        assert est <= 1.5 * eps

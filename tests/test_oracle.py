"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test targets a mistake the oracle could plausibly contain (a dropped term, a wrong
index, a transposed operand, an off-by-one rank) and checks it against something other
than the oracle itself: brute force, closed forms, an independent library routine, or a
theorem of the paper.
"""
import os

import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs


def _kernel(kind, X, Y):
    if kind == 0:
        r = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
        return np.exp(-r)
    if kind == 1:
        r2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
        return 1.0 / (1.0 + r2)
    ip = X @ Y.T
    return (1.0 + ip) ** 2


def _bbox(P):
    return P.min(0), P.max(0)


# ---------------------------------------------------------------- trees (Def. 2.2, 2.3, Alg. 1)

@pytest.mark.parametrize("kind,dim,n,leaf", [(0, 2, 300, 8), (1, 3, 517, 16), (0, 3, 64, 64), (0, 1, 1, 4),
                                             (0, 2, 101, 2), (0, 2, 5, 2)])
def test_cluster_tree_definition(oracle, kind, dim, n, leaf):
    """Def. 2.2: root = I, children partition the parent, all non-empty; leaves <= n_min;
    depth = ceil(log2(n / leaf)); each split puts the smaller coordinates on the first child."""
    P = inputs.points(kind, dim, n, 5)
    T = oracle.Tree(P, leaf, 1.0)
    assert sorted(T.perm.tolist()) == list(range(n))
    cl = T.cl
    assert cl[0, 1] == 0 and cl[0, 2] == n
    D = 0
    while -(-n // 2 ** D) > leaf:
        D += 1
    assert T.depth == D
    Pp = P[T.perm]
    for c in range(T.ncl):
        lvl, b, s, c0, c1 = (int(x) for x in cl[c])
        assert s >= 1
        if c0 < 0:
            assert lvl == D and s <= leaf
            continue
        assert cl[c0, 1] == b and cl[c0, 2] == s // 2
        assert cl[c1, 1] == b + s // 2 and cl[c0, 2] + cl[c1, 2] == s
        lo, hi = _bbox(Pp[b:b + s])
        ax = int(np.argmax(hi - lo))
        left, right = Pp[b:b + s // 2, ax], Pp[b + s // 2:b + s, ax]
        if len(left) and len(right):
            assert left.max() <= right.min()


def test_cluster_tree_rejects_leaf_size_one(oracle):
    """Def. 2.2 (iii): clusters are non-empty. With every leaf on one level, n_min = 1 would split
    a one-point cluster above the leaf level into an empty and a one-point child (N = 5: level 2
    holds clusters of 1 and 2 points), so the tree requires n_min >= 2."""
    with pytest.raises(ValueError):
        oracle.Tree(inputs.points(0, 2, 5, 4), 1, 1.0)


def _adm(Pt, Ps, eta):
    lt, ht = _bbox(Pt)
    ls, hs = _bbox(Ps)
    dt, ds = np.linalg.norm(ht - lt), np.linalg.norm(hs - ls)
    gap = np.maximum(0, np.maximum(ls - ht, lt - hs))
    dist = np.linalg.norm(gap)
    return dist > 0 and max(dt, ds) <= eta * dist


@pytest.mark.parametrize("kind,dim,n,leaf,eta", [(0, 2, 400, 8, 1.0), (1, 3, 700, 16, 1.0), (0, 3, 333, 10, 2.0)])
def test_block_tree_partition_and_admissibility(oracle, kind, dim, n, leaf, eta):
    """Alg. 1: leaves partition I x I; far leaves admissible, near leaves and inner blocks
    not; inner blocks have exactly the 4 children tau' x sigma'; the tree is level-conserving."""
    P = inputs.points(kind, dim, n, 11)
    T = oracle.Tree(P, leaf, eta)
    Pp = P[T.perm]
    cover = np.zeros((n, n), np.int32)
    for b in range(T.nbl):
        tau, sig, k, lvl, leafid, nch = (int(x) for x in T.bl[b])
        tb, ts = T.cl[tau, 1:3]
        sb, ss = T.cl[sig, 1:3]
        assert T.cl[tau, 0] == lvl == T.cl[sig, 0]
        a = _adm(Pp[tb:tb + ts], Pp[sb:sb + ss], eta)
        if k == 1:
            assert a and leafid >= 0
            cover[tb:tb + ts, sb:sb + ss] += 1
        elif k == 2:
            assert not a and leafid >= 0 and T.cl[tau, 3] < 0
            cover[tb:tb + ts, sb:sb + ss] += 1
        else:
            assert not a and nch == 4
            kids = {(int(T.bl[c, 0]), int(T.bl[c, 1])) for c in T.bl_child[b]}
            want = {(int(x), int(y)) for x in T.cl[tau, 3:5] for y in T.cl[sig, 3:5]}
            assert kids == want
    assert (cover == 1).all()


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_points_1d_n16():
    """The points of tests/golden/tree_1d_n16_leaf2_eta1.txt: x_i = ((5 i + 3) mod 16) / 16."""
    return (((5 * np.arange(16) + 3) % 16) / 16.0).reshape(16, 1)


def test_hand_derived_example_tree_and_counts(oracle):
    """Def. 2.2, Def. 2.3, Algorithm 1 and Algorithm 3 against a worked example derived by hand
    (16 points on a line, leaf 2, eta 1): permutation, block and leaf counts, C_sp, every leaf's
    level and admissibility (including the equality case of the <= test), and its low-rank
    terms, H-pairs and the level each low-rank term is created on. A wrong split, a strict
    inequality, a dropped inherited term or an H-pair kept as low rank each change a line."""
    from parity_util import read_tree_golden
    perm, counts, leaves = read_tree_golden(os.path.join(GOLDEN, "tree_1d_n16_leaf2_eta1.txt"))
    T = oracle.Tree(golden_points_1d_n16(), 2, 1.0)
    assert np.array_equal(T.perm, perm)
    assert (T.ncl, T.nbl, T.nleaf, T.depth, T.csp()) == (counts["clusters"], counts["blocks"], counts["leaves"],
                                                         counts["depth"], counts["csp"])
    assert len(T.far_leaves()) == counts["far"] and len(T.near_leaves()) == counts["near"]
    lr, hp, at = T.sumexpr_counts()
    seen = set()
    for l in range(T.nleaf):
        key = T.leaf_ranges(l)
        lev, far, n_lr, n_hp, created = leaves[key]
        seen.add(key)
        assert int(T.leaf_blocks[l, 3]) == lev and (T.leaf_blocks[l, 2] == 1) == far, key
        assert (int(lr[l]), int(hp[l])) == (n_lr, n_hp), key
        assert [int(x) for x in at[l, 2:2 + len(created)]] == created and at[l, :2].sum() == 0, key
    assert seen == set(leaves)


def test_admissibility_symmetric(oracle):
    """Def. 2.3: adm(tau, sigma) = adm(sigma, tau), so the leaf pattern is symmetric."""
    P = inputs.points(1, 3, 900, 2)
    T = oracle.Tree(P, 16, 1.0)
    kinds = {(int(a), int(b)): int(k) for a, b, k in T.bl[:, :3]}
    for (a, b), k in kinds.items():
        assert kinds[(b, a)] == k


# ---------------------------------------------------------------- assembly (Alg. 6)

@pytest.mark.parametrize("kernel,kind,dim", [(0, 0, 2), (1, 1, 3), (0, 1, 3)])
def test_aca_accuracy_against_brute_force(oracle, kernel, kind, dim):
    """Far leaves by ACA match the kernel block evaluated entry by entry (eq. (ACAblockerror)
    with a modest constant); near leaves are the kernel block exactly."""
    P = inputs.points(kind, dim, 600, 4)
    T = oracle.Tree(P, 16, 1.0)
    H = oracle.HMatrix(T, kernel, 1e-8)
    Pp = P[T.perm]
    for l in range(T.nleaf):
        r0, m, c0, n = T.leaf_ranges(l)
        K = _kernel(kernel, Pp[r0:r0 + m], Pp[c0:c0 + n])
        if H.ranks[l] < 0:
            assert np.array_equal(H.leaf(l), K) or np.abs(H.leaf(l) - K).max() <= 1e-15 * np.abs(K).max()
        else:
            U, V = H.leaf(l)
            err = np.linalg.norm(K - U @ V.T) / np.linalg.norm(K)
            assert err <= 1e-6, (l, err)


def test_aca_exact_on_separable_kernel(oracle):
    """The kernel (1 + x.y)^2 in 2-D has rank <= 6 on every block: ACA reproduces the block
    to rounding after 6 terms; the 7th (rounding-level) term is the one the stop test
    measures and is kept, so the stored rank is at most 7."""
    P = inputs.points(0, 2, 500, 9)
    T = oracle.Tree(P, 16, 1.0)
    H = oracle.HMatrix(T, oracle.KERNEL_POLY2, 1e-12)
    Pp = P[T.perm]
    for l in T.far_leaves():
        U, V = H.leaf(int(l))
        assert U.shape[1] <= 7
        r0, m, c0, n = T.leaf_ranges(int(l))
        K = _kernel(2, Pp[r0:r0 + m], Pp[c0:c0 + n])
        assert np.linalg.norm(K - U @ V.T) <= 1e-12 * np.linalg.norm(K)


def test_fp32_storage_is_exact_rounding(oracle):
    """prec32 stores every factor entry rounded to float once."""
    P = inputs.points(0, 2, 300, 1)
    T = oracle.Tree(P, 16, 1.0)
    H64 = oracle.HMatrix(T, 0, 1e-8)
    H32 = oracle.HMatrix(T, 0, 1e-8, prec32=True)
    for l in range(T.nleaf):
        a, b = H64.leaf(l), H32.leaf(l)
        if H64.ranks[l] < 0:
            assert np.array_equal(a.astype(np.float32).astype(np.float64), b)
        else:
            assert np.array_equal(a[0].astype(np.float32).astype(np.float64), b[0])
            assert np.array_equal(a[1].astype(np.float32).astype(np.float64), b[1])


def test_dense_sub_matches_leaves(oracle):
    """The dense view of the H-matrix places each leaf at its (tau, sigma) position."""
    P = inputs.points(0, 2, 256, 3)
    T = oracle.Tree(P, 16, 1.0)
    H = oracle.HMatrix(T, 0, 1e-9)
    D = H.dense()
    for l in range(T.nleaf):
        r0, m, c0, n = T.leaf_ranges(l)
        blk = H.leaf(l) if H.ranks[l] < 0 else H.leaf(l)[0] @ H.leaf(l)[1].T
        assert np.allclose(D[r0:r0 + m, c0:c0 + n], blk, rtol=0, atol=1e-15)
    sub = H.dense_sub(10, 50, 100, 77)
    assert np.array_equal(sub, D[10:60, 100:177])


# ---------------------------------------------------------------- dense product

def test_matmul_brute_force(oracle):
    """The product against a brute-force triple loop (tiny) and an independent BLAS call."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((7, 5))
    B = rng.standard_normal((5, 9))
    C = oracle.matmul(A, B)
    ref = np.zeros((7, 9))
    for i in range(7):
        for j in range(9):
            for k in range(5):
                ref[i, j] += A[i, k] * B[k, j]
    assert np.abs(C - ref).max() <= 1e-14
    A = rng.standard_normal((130, 70))
    B = rng.standard_normal((70, 90))
    assert np.abs(oracle.matmul(A, B) - A @ B).max() <= 1e-12


def test_block_product_matches_dense(oracle):
    """C|tau x sigma = A|tau x I * B|I x sigma equals the block of the full product."""
    P = inputs.points(1, 3, 400, 6)
    T = oracle.Tree(P, 16, 1.0)
    A = oracle.HMatrix(T, 0, 1e-9)
    B = oracle.HMatrix(T, 1, 1e-9)
    DC = oracle.matmul(A.dense(), B.dense())
    for l in list(T.far_leaves()[:5]) + list(T.near_leaves()[:3]):
        r0, m, c0, n = T.leaf_ranges(int(l))
        Cb = oracle.block_product(A, B, r0, m, c0, n, chunk=37)
        assert np.abs(Cb - DC[r0:r0 + m, c0:c0 + n]).max() <= 1e-12 * np.abs(DC).max()


def test_eta_to_zero_gives_dense_kernel(oracle):
    """Closed form: with eta -> 0 nothing is admissible, every leaf is dense, and the H-matrix
    and its product are the kernel matrix and its square exactly."""
    P = inputs.points(0, 2, 128, 8)
    T = oracle.Tree(P, 16, 1e-9)
    assert len(T.far_leaves()) == 0
    H = oracle.HMatrix(T, 0, 1e-9)
    Pp = P[T.perm]
    K = _kernel(0, Pp, Pp)
    assert np.abs(H.dense() - K).max() <= 1e-15
    assert np.abs(oracle.matmul(H.dense(), H.dense()) - K @ K).max() <= 1e-12


# ---------------------------------------------------------------- SVD and eps-rank

@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (3, 5), (40, 40), (64, 20), (17, 90)])
def test_svd_against_lapack_and_identities(oracle, m, n):
    rng = np.random.default_rng(m * 100 + n)
    M = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, -12, n))
    s, U, V = oracle.svd(M)
    s_ref = np.linalg.svd(M, compute_uv=False)
    assert np.abs(s - s_ref).max() <= 1e-13 * s_ref[0]
    p = min(m, n)
    assert np.abs(U.T @ U - np.eye(p)).max() <= 1e-12 or s_ref[-1] < 1e-13 * s_ref[0]
    assert np.abs(V.T @ V - np.eye(p)).max() <= 1e-12
    assert np.abs(U * s @ V.T - M).max() <= 1e-13 * s[0]
    # Eckart-Young: the rank-k truncation error is the tail of the singular values
    for k in range(p + 1):
        err = np.linalg.norm(M - (U[:, :k] * s[:k]) @ V[:, :k].T)
        tail = np.sqrt(np.sum(s[k:] ** 2))
        assert abs(err - tail) <= 1e-12 * s[0] + 1e-10 * tail


def test_svd_rank_deficient_and_zero(oracle):
    rng = np.random.default_rng(3)
    M = rng.standard_normal((30, 4)) @ rng.standard_normal((4, 25))
    s, _, _ = oracle.svd(M, vectors=False)
    assert (s[4:] <= 1e-12 * s[0]).all() and s[3] > 1e-3 * s[0]
    s, _, _ = oracle.svd(np.zeros((6, 4)), vectors=False)
    assert (s == 0).all()


def _with_spectrum(rng, m, n, s):
    """An m x n matrix with the given singular values (random orthonormal factors)."""
    k = len(s)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return (U * s) @ V.T


@pytest.mark.parametrize("m,n", [(200, 150), (150, 200), (257, 257)])
def test_svd_values_qrcp_against_jacobi_and_lapack(oracle, m, n):
    """The pivoted-QR singular values: equal to the full one-sided Jacobi's and to LAPACK's above
    the stopping level; the undetermined remainder bounds the dropped energy (the best rank-k
    error cannot exceed that of the truncated factorisation)."""
    rng = np.random.default_rng(m + 7 * n)
    sv = np.logspace(0, -15, 40)
    M = _with_spectrum(rng, m, n, sv) + 1e-16 * rng.standard_normal((m, n))
    s, resid = oracle.svd_values_lowrank(M, tol=1e-13)
    s_full, _, _ = oracle.svd(M, vectors=False)
    s_ref = np.linalg.svd(M, compute_uv=False)
    k = len(s)
    assert 0 < k < 40
    assert np.abs(s - s_full[:k]).max() <= 1e-13 * s_full[0]
    assert np.abs(s - s_ref[:k]).max() <= 1e-13 * s_ref[0]
    nf = np.linalg.norm(M)
    assert resid <= 1e-13 * nf
    assert np.sum(s_ref[k:] ** 2) <= resid ** 2 * (1 + 1e-6) + 1e-30
    # the remainder is the part the pivoted factorisation could not yet drop: it is not much
    # below the stopping level (the step before met none of it)
    assert s[-1] >= 1e-13 * nf * 1e-3


def test_svd_values_qrcp_exact_rank_zero_and_full(oracle):
    rng = np.random.default_rng(11)
    sv = np.array([5.0, 2.0, 1.0, 1e-3, 1e-6])
    M = _with_spectrum(rng, 90, 70, sv)
    s, resid = oracle.svd_values_lowrank(M, tol=1e-13)
    assert len(s) == 5 and np.abs(s - sv).max() <= 1e-13 * sv[0] and resid <= 1e-13 * np.linalg.norm(M)
    s, resid = oracle.svd_values_lowrank(np.zeros((20, 30)))
    assert len(s) == 0 and resid == 0.0
    # tol = 0: every step runs (up to an exactly zero remainder); the values are the full SVD's
    M = rng.standard_normal((25, 12))
    s, resid = oracle.svd_values_lowrank(M, tol=0.0)
    assert len(s) == 12 and resid == 0.0
    assert np.abs(s - np.linalg.svd(M, compute_uv=False)).max() <= 1e-13 * s[0]
    # column pivoting matters: a tiny column first and a dominant one last
    M = np.zeros((10, 3))
    M[:, 0] = 1e-9 * rng.standard_normal(10)
    M[:, 2] = rng.standard_normal(10)
    s, resid = oracle.svd_values_lowrank(M, tol=1e-6)
    assert len(s) == 1 and abs(s[0] - np.linalg.norm(M[:, 2])) <= 1e-14 * s[0]


def test_block_product_blas_matches_plain_loop(oracle):
    """The BLAS-chunked exact block equals the oracle's plain loop and the dense product."""
    P = inputs.points(1, 3, 3000, 2)
    T = oracle.Tree(P, 32, 1.0)
    A = oracle.HMatrix(T, oracle.KERNEL_EXP, 1e-8)
    B = oracle.HMatrix(T, oracle.KERNEL_INVQ, 1e-8)
    DC = oracle.matmul(A.dense(), B.dense())
    sizes = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    far = np.nonzero(T.leaf_blocks[:, 2] == 1)[0]
    for l in [far[0], far[len(far) // 2], far[np.argmax(sizes[far, 1])], int(np.nonzero(T.leaf_blocks[:, 2] == 2)[0][0])]:
        r0, m, c0, n = T.leaf_ranges(int(l))
        ref = oracle.block_product(A, B, r0, m, c0, n)
        got = oracle.block_product_blas(A, B, r0, m, c0, n, chunk=700)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(got - DC[r0:r0 + m, c0:c0 + n]).max() <= 1e-13 * np.abs(ref).max()


def test_truth_for_large_block_matches_full_svd(oracle):
    """truth_for_block on a block above QRCP_MIN: the eps-rank and tail equal those of the
    full one-sided Jacobi SVD of the same exact product block."""
    P = inputs.points(1, 3, 8192, 5)
    T = oracle.Tree(P, 64, 1.0)
    A = oracle.HMatrix(T, oracle.KERNEL_EXP, 1e-10)
    sizes = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    big = [l for l in range(T.nleaf) if T.leaf_blocks[l, 2] == 1 and min(sizes[l, 1], sizes[l, 3]) >= oracle.QRCP_MIN]
    assert big
    l = big[0]
    r0, m, c0, n = T.leaf_ranges(l)
    blk = oracle.block_product(A, A, r0, m, c0, n)
    s_full, _, _ = oracle.svd(blk, vectors=False)
    for eps in (1e-4, 1e-6, 1e-8, 1e-10):
        tr = oracle.truth_for_block(blk, eps, l)
        assert len(tr.s) < min(m, n)          # the pivoted QR path was taken
        assert tr.k_eps == oracle.eps_rank(s_full, eps)
        assert abs(tr.tail - np.sqrt(np.sum(s_full[tr.k_eps:] ** 2))) <= 1e-12 * tr.norm
        assert abs(tr.norm - np.linalg.norm(blk)) <= 1e-13 * tr.norm


def test_eps_rank_closed_forms(oracle):
    s = np.array([1.0, 1e-3, 1e-7])
    tot = np.sqrt(np.sum(s ** 2))
    assert oracle.eps_rank(s, 1e-6) == 2          # tail 1e-7 <= 1e-6 * tot
    assert oracle.eps_rank(s, 1e-8) == 3
    assert oracle.eps_rank(s, 2e-3) == 1          # tail ~1e-3 <= 2e-3
    assert oracle.eps_rank(s, 1.0) == 0
    assert oracle.eps_rank(np.zeros(4), 1e-6) == 0
    # boundary: tail exactly eps * norm counts as within ("<=")
    s = np.array([3.0, 4.0])
    assert oracle.eps_rank(s, 4.0 / 5.0) == 1
    assert oracle.eps_rank(s, np.nextafter(4.0 / 5.0, 0)) == 2
    _ = tot


def test_eps_rank_monotone(oracle):
    rng = np.random.default_rng(5)
    s = np.sort(np.abs(rng.standard_normal(50)) * np.logspace(0, -14, 50))[::-1]
    ks = [oracle.eps_rank(s, e) for e in np.logspace(-16, 0, 60)]
    assert all(a >= b for a, b in zip(ks, ks[1:]))
    assert ks[0] == 50


# ---------------------------------------------------------------- product truth & sum-expressions

def test_product_of_separable_kernels_has_low_rank(oracle):
    """Closed form: (1 + x.y)^2 has global rank <= 6 in 2-D, so every block of the product
    of two such H-matrices has eps-rank <= 6 even at eps = 1e-12."""
    P = inputs.points(0, 2, 512, 2)
    T = oracle.Tree(P, 16, 1.0)
    A = oracle.HMatrix(T, oracle.KERNEL_POLY2, 1e-14)
    _, truths = oracle.product_truth(A, A, 1e-12)
    assert max(t.k_eps for t in truths.values()) <= 6


def test_identity_factor_gives_best_approx_of_other(oracle):
    """Closed form: with A = diag (near leaves diagonal, far leaves zero) the product's far
    blocks are diag * B|b, whose eps-rank is that of B|b scaled by the rows."""
    P = inputs.points(0, 2, 256, 4)
    T = oracle.Tree(P, 16, 1.0)
    B = oracle.HMatrix(T, 0, 1e-12)
    DB = B.dense()
    d = 1.0 + inputs.uniform01(77, 256)
    DA = np.diag(d)
    DC = oracle.matmul(DA, DB)
    assert np.abs(DC - d[:, None] * DB).max() <= 1e-15 * np.abs(DB).max() * 2


def test_sumexpr_reproduces_product_blocks(oracle):
    """Alg. 3 restriction from S(I,I) = HK (Alg. 4): for every leaf, the low-rank terms plus
    the H-pairs of its sum-expression add up to the exact product block (Sec. 3.2), and the
    number of low-rank terms matches the symbolic count."""
    P = inputs.points(1, 3, 700, 12)
    T = oracle.Tree(P, 16, 1.0)
    A = oracle.HMatrix(T, 0, 1e-10)
    B = oracle.HMatrix(T, 1, 1e-10)
    DC = oracle.matmul(A.dense(), B.dense())
    lr, hp, at = T.sumexpr_counts()
    assert np.array_equal(at.sum(1), lr)
    for l in range(T.nleaf):
        r0, m, c0, n = T.leaf_ranges(l)
        S, nt = oracle.sumexpr_eval(A, B, l)
        assert nt == lr[l]
        blk = DC[r0:r0 + m, c0:c0 + n]
        assert np.linalg.norm(S - blk) <= 1e-13 * max(np.linalg.norm(blk), 1e-300)


def test_lemma_5_3_term_bound(oracle):
    """Lemma 5.3: S(tau, sigma) holds at most C_sp * level(tau x sigma) low-rank terms, and
    terms are only created at levels where the target's ancestor has a far neighbour."""
    for kind, dim, n, leaf in [(0, 2, 2048, 32), (1, 3, 4096, 32)]:
        P = inputs.points(kind, dim, n, 0)
        T = oracle.Tree(P, leaf, 1.0)
        lr, hp, at = T.sumexpr_counts()
        csp = T.csp()
        lvl = T.leaf_blocks[:, 3]
        assert (lr <= csp * lvl).all()
        assert (hp <= csp).all()
        assert (at[:, 0] == 0).all()     # S(I, I) holds no low-rank terms
        # near leaves sit on the last level; their H-pairs are leaf x leaf pairs
        near = T.leaf_blocks[:, 2] == 2
        assert (lvl[near] == T.depth).all()


def test_truth_eckart_young_invariant(oracle):
    """For the truth of a product block: err of the best rank-k_eps approximation equals the
    SVD tail and is <= eps * ||block||; rank k_eps - 1 would exceed eps."""
    P = inputs.points(0, 2, 512, 0)
    T = oracle.Tree(P, 16, 1.0)
    A = oracle.HMatrix(T, 0, 1e-10)
    DC = oracle.matmul(A.dense(), A.dense())
    for l in T.far_leaves()[:40]:
        r0, m, c0, n = T.leaf_ranges(int(l))
        blk = DC[r0:r0 + m, c0:c0 + n]
        L, R = oracle.best_approx(blk, 1e-6)
        k = L.shape[1]
        err = np.linalg.norm(blk - L @ R.T)
        nb = np.linalg.norm(blk)
        assert err <= 1e-6 * nb * (1 + 1e-10)
        s = np.linalg.svd(blk, compute_uv=False)
        if k > 0:
            assert np.sqrt(np.sum(s[k - 1:] ** 2)) > 1e-6 * nb * (1 - 1e-10)


# ---------------------------------------------------------------- learned rank proposal network

def _mlp_params(seed, scale=0.3):
    from oracle import rank_mlp as R
    return (inputs.uniform01(seed, R.N_PARAMS) * 2.0 - 1.0) * scale


def test_mlp_gradient_finite_differences():
    """Backpropagation against central differences of the loss, on every parameter group (a
    transposed weight, a dropped ReLU mask or a missing 1/count factor all fail here)."""
    from oracle import rank_mlp as R
    w = _mlp_params(11)
    X = (inputs.uniform01(12, 37 * R.F).reshape(37, R.F) * 2.0 - 1.0) * 2.0
    t = inputs.uniform01(13, 37) * 5.0
    L, g = R.loss_grad(w, X, t)
    assert L == pytest.approx(R.loss(w, X, t), rel=1e-15)
    idx = np.concatenate([np.arange(0, 40), np.arange(R.H * R.F, R.H * R.F + 8),
                          np.arange(R.H * R.F + R.H + 100, R.H * R.F + R.H + 140),
                          np.arange(R.N_PARAMS - 2 * R.H - 1, R.N_PARAMS)])
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (R.loss(wp, X, t) - R.loss(wm, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), i


def test_mlp_zero_weights_closed_form():
    """All weights zero: the output is b3 for every sample; the only non-zero gradient entry is
    d/db3 = 2 mean(b3 - t)."""
    from oracle import rank_mlp as R
    w = np.zeros(R.N_PARAMS)
    w[-1] = 1.75
    X = inputs.uniform01(21, 10 * R.F).reshape(10, R.F)
    t = inputs.uniform01(22, 10) * 4.0
    assert np.all(R.forward(w, X) == 1.75)
    L, g = R.loss_grad(w, X, t)
    assert L == pytest.approx(np.mean((1.75 - t) ** 2), rel=1e-14)
    assert g[-1] == pytest.approx(2.0 * np.mean(1.75 - t), rel=1e-14)
    assert np.all(g[:-1] == 0.0)


def test_mlp_linear_regime_is_affine_map():
    """With positive inputs, non-negative weights and positive biases every ReLU passes its
    input, so the network is the composed affine map w3.(W2 (W1 x + b1) + b2) + b3; and its
    gradient with respect to w3 is 2/count * sum_s e_s h2_s."""
    from oracle import rank_mlp as R
    w = inputs.uniform01(31, R.N_PARAMS) * 0.2 + 0.01
    W1, b1, W2, b2, w3, b3 = R.unpack(w)
    X = inputs.uniform01(32, 9 * R.F).reshape(9, R.F)
    t = inputs.uniform01(33, 9)
    y = np.array([w3 @ (W2 @ (W1 @ x + b1) + b2) + b3 for x in X])
    np.testing.assert_allclose(R.forward(w, X), y, rtol=1e-14)
    _, g = R.loss_grad(w, X, t)
    h2 = np.array([W2 @ (W1 @ x + b1) + b2 for x in X])
    gw3 = 2.0 / 9 * ((y - t)[:, None] * h2).sum(0)
    np.testing.assert_allclose(g[R.N_PARAMS - R.H - 1:R.N_PARAMS - 1], gw3, rtol=1e-12)


def test_mlp_target_round_trip():
    from oracle import rank_mlp as R
    r = np.array([0, 1, 3, 7, 15, 96, -2], np.float64)
    np.testing.assert_allclose(R.predicted_rank(R.target(r)), np.maximum(r, 0), atol=1e-12)
    assert R.target(np.array([0.0]))[0] == 0.0 and R.target(np.array([3.0]))[0] == 2.0


# ---------------------------------------------------------------- one-vector compressors (Sec. 4)

def _lowrank(seed, m, n, r):
    u = inputs.uniform01(seed, m * r).reshape(m, r) - 0.5
    v = inputs.uniform01(seed + 1, n * r).reshape(n, r) - 0.5
    return u @ v.T


def test_aca_interpolates_pivots_and_recovers_low_rank():
    """Algorithm 6: the cross approximation reproduces D exactly on every pivot row and column
    (the Schur complement vanishes there), and a rank-5 matrix exactly after 5 crosses (the
    next crosses are rounding noise). A dropped correction term or a transposed index breaks
    both."""
    from oracle import compressors as X
    D = _lowrank(31, 40, 30, 5)
    L, U, k = X.aca(D, 1e-14, 50)
    assert 5 <= k <= 7
    assert np.linalg.norm(D - L @ U.T) <= 1e-12 * np.linalg.norm(D)
    # a full-rank matrix stopped early: exact on the pivot rows and columns only
    G = inputs.uniform01(33, 24 * 20).reshape(24, 20)
    L, U, k = X.aca(G, 0.2, 50, need=1)
    assert 1 <= k < 20
    R = G - L @ U.T
    rows = [i for i in range(24) if np.abs(L[i, :]).max() > 0 and np.abs(R[i, :]).max() <= 1e-12]
    cols = [j for j in range(20) if np.abs(R[:, j]).max() <= 1e-12]
    assert len(rows) >= k and len(cols) >= k
    # u_r is 1 at its pivot column and 0 at earlier pivot columns (unit triangular structure)
    piv = [int(np.flatnonzero(np.isclose(U[:, r], 1.0))[0]) for r in range(k)]
    for r in range(k):
        assert abs(U[piv[r], r] - 1.0) <= 1e-14
        for s in range(r):
            assert abs(U[piv[s], r]) <= 1e-12


def test_aca_skips_zero_row():
    """An exactly zero first row is marked used and the next unused row starts the crosses."""
    from oracle import compressors as X
    D = _lowrank(35, 20, 16, 3)
    D[0, :] = 0.0
    L, U, k = X.aca(D, 1e-14, 30)
    assert np.linalg.norm(D - L @ U.T) <= 1e-12 * np.linalg.norm(D)
    Z = np.zeros((6, 5))
    L, U, k = X.aca(Z, 1e-6, 10)
    assert k == 0 and L.shape == (6, 0)


def test_lanczos_bidiagonal_form():
    """Algorithm 7: Q and W orthonormal and Q^T D W_k upper bidiagonal with alpha on the diagonal
    and beta above it; run to full length, the singular values of that bidiagonal matrix are
    D's (numpy's SVD)."""
    from oracle import compressors as X
    D = inputs.uniform01(41, 18 * 12).reshape(18, 12) - 0.3
    w1 = inputs.uniform01(42, 12) - 0.5
    Q, W, a, b, k = X.lanczos(D, w1, 0.0, 100)
    assert k == 12
    assert np.abs(Q.T @ Q - np.eye(k)).max() <= 1e-12
    Wk = W[:, :k]
    assert np.abs(Wk.T @ Wk - np.eye(k)).max() <= 1e-12
    Bm = Q.T @ D @ Wk
    ref = np.diag(a) + np.diag(b[:k - 1], 1)
    assert np.abs(Bm - ref).max() <= 1e-12 * np.abs(D).max()
    sv = np.linalg.svd(ref, compute_uv=False)
    assert np.allclose(sv, np.linalg.svd(D, compute_uv=False), rtol=1e-12, atol=1e-12)
    # a rank-4 matrix: the Krylov space is exhausted after 4 steps and Q Q^T D = D
    R4 = _lowrank(43, 30, 25, 4)
    Q, W, a, b, k = X.lanczos(R4, inputs.uniform01(44, 25) - 0.5, 1e-12, 100)
    assert 4 <= k <= 6 and a[4] <= 1e-10 * a[0]
    assert np.linalg.norm(R4 - Q @ (Q.T @ R4)) <= 1e-12 * np.linalg.norm(R4)


def test_truncate_is_eckart_young():
    """Algorithm 5: the truncated L U^T has the eps-rank of L U^T and its error is the tail of
    the singular values (numpy's SVD of the product)."""
    from oracle import compressors as X
    L = inputs.uniform01(51, 40 * 9).reshape(40, 9) - 0.5
    U = (inputs.uniform01(52, 30 * 9).reshape(30, 9) - 0.5) * (0.1 ** np.arange(9))
    M = L @ U.T
    s = np.linalg.svd(M, compute_uv=False)
    for eps in (1e-1, 1e-3, 1e-6):
        A, B = X.truncate(L, U, eps)
        k = A.shape[1]
        tail = np.sqrt(np.cumsum((s * s)[::-1])[::-1])
        kref = int(np.argmax(tail <= eps * tail[0])) if np.any(tail <= eps * tail[0]) else len(s)
        assert k == kref
        assert abs(np.linalg.norm(M - A @ B.T) - np.sqrt(np.sum(s[k:] ** 2))) <= 1e-12 * np.linalg.norm(M)


def test_compressors_meet_bound_on_product_blocks(oracle):
    """The stop rule (two consecutive steps meeting eq. (truncaca) at eps/8) followed by the
    truncation meets the blockwise bound 1.5 eps with rank <= k_eps + 2 on the exact far blocks
    of a 3-D product (e^{-r} times 1/(1+r^2))."""
    from oracle import compressors as X
    from parity_util import _oracle_pair
    P = inputs.points(0, 3, 2000, 5)
    T, Ao, Bo = _oracle_pair(oracle, P, 32, 1.0, 0, 1, 1e-10)
    DC = oracle.matmul(Ao.dense(), Bo.dense())
    eps = 1e-6
    far = [l for l in range(T.nleaf) if T.leaf_blocks[l, 2] == 1]
    assert len(far) > 500
    for l in far:
        r0, m, c0, n = T.leaf_ranges(l)
        blk = DC[r0:r0 + m, c0:c0 + n]
        tr = oracle.truth_for_block(blk, eps, l)
        L, U, _ = X.aca(blk, eps / 8, 95)
        Q, _, _, _, _ = X.lanczos(blk, inputs.uniform01(l, n) - 0.5, eps / 8, 95)
        for A, B in (X.truncate(L, U, eps), X.truncate(Q, blk.T @ Q, eps)):
            err = np.linalg.norm(blk - A @ B.T) / tr.norm
            assert err <= 1.5 * eps, (l, err)
            assert A.shape[1] <= tr.k_eps + 2, (l, A.shape[1], tr.k_eps)


def _with_singular_values(seed, m, n, s):
    """A matrix U diag(s) V^T with orthonormal U, V from seeded uniforms (numpy QR)."""
    U, _ = np.linalg.qr(inputs.uniform01(seed, m * len(s)).reshape(m, len(s)) - 0.5)
    V, _ = np.linalg.qr(inputs.uniform01(seed + 1, n * len(s)).reshape(n, len(s)) - 0.5)
    return (U * s) @ V.T


def test_randomized_range_finder():
    """Algorithm 8, blocked: a rank-5 matrix is captured in one round by exactly 5 orthonormal
    columns (the other 3 samples fall below the drop threshold), and the next round keeps none;
    on singular values 2^-i the truncated result meets 1.5 eps at rank <= k_eps + 2."""
    from oracle import compressors as X
    D = _lowrank(61, 40, 30, 5)
    om = np.random.default_rng(62).standard_normal((30, 24))
    Q, W, rounds = X.randomized(D, om, 1e-10, 8, 64)
    assert Q.shape[1] == 5 and rounds == 2
    assert np.abs(Q.T @ Q - np.eye(5)).max() <= 1e-13
    assert np.linalg.norm(D - Q @ W.T) <= 1e-12 * np.linalg.norm(D)
    s = 2.0 ** -np.arange(30)
    G = _with_singular_values(63, 50, 40, s)
    om = np.random.default_rng(64).standard_normal((40, 80))
    for eps in (1e-2, 1e-4, 1e-7):
        Q, W, _ = X.randomized(G, om, eps, 8, 80)
        A, B = X.truncate(Q, W, eps)
        tail = np.sqrt(np.cumsum((s * s)[::-1])[::-1])
        k_eps = int(np.argmax(tail <= eps * tail[0]))
        err = np.linalg.norm(G - A @ B.T) / np.linalg.norm(G)
        assert err <= 1.5 * eps and A.shape[1] <= k_eps + 2, (eps, err, A.shape[1], k_eps)


def test_fixed_rank_subspace_iteration():
    """Algorithm 9: rank <= k, and with a spectral gap after k (singular values 1..0.5, then
    1e-4 and below) one subspace iteration comes within 1 % of the best rank-k error."""
    from oracle import compressors as X
    s = np.concatenate([np.linspace(1.0, 0.5, 6), 1e-4 * 0.5 ** np.arange(20)])
    G = _with_singular_values(71, 60, 45, s)
    om = np.random.default_rng(72).standard_normal((45, 6))
    best = np.sqrt(np.sum(s[6:] ** 2))
    for q in (1, 2):
        L, U = X.fixed_rank(G, om, q)
        assert L.shape[1] <= 6
        assert np.abs(L.T @ L - np.eye(L.shape[1])).max() <= 1e-12
        err = np.linalg.norm(G - L @ U.T)
        assert best <= err * (1 + 1e-12) and err <= 1.01 * best, (q, err, best)


def test_randomized_meets_paper_eps_on_product_blocks(oracle):
    """The blocked Alg. 8 at the paper's eps = 1e-12 (Sec. 6) on exact far blocks of a product of
    ACA inputs (N = 2048 in 2-D, exp(-r), ACA to 1e-14): every block within 1.5 eps of the block
    at rank <= eps-rank + 2 (numpy's SVD). Without the final projection of a column that kept
    little of its norm against the whole basis, the basis loses orthogonality at this eps and
    190 of these 1262 blocks miss the bar."""
    from oracle import compressors as CO
    P = inputs.points(0, 2, 2048, 0)
    T = oracle.Tree(P, 32, 1.0)
    A = oracle.HMatrix(T, oracle.KERNEL_EXP, 1e-14)
    DC = oracle.matmul(A.dense(), A.dense())
    eps = 1e-12
    far = T.far_leaves()
    for l in far[::4]:
        l = int(l)
        r0, m, c0, n = T.leaf_ranges(l)
        D = DC[r0:r0 + m, c0:c0 + n]
        om = np.random.default_rng(1000 + l).standard_normal((n, 400))
        Q, W, _ = CO.randomized(D, om, eps, 8, 96)
        L, U = CO.truncate(Q, W, eps)
        s = np.linalg.svd(D, compute_uv=False)
        err = np.linalg.norm(D - L @ U.T) / np.linalg.norm(D)
        assert err <= 1.5 * eps, (l, err)
        assert L.shape[1] <= oracle.eps_rank(s, eps) + 2


def test_gaussian_test_matrix_generator():
    """The oracle-side Gaussian generator: its stream is the published splitmix64 (checked
    against the independent stream of the input module at the counters it names), its entries
    are standard normal (Kolmogorov-Smirnov against N(0, 1) on 200 000 draws), and different
    leaves, rounds and columns draw uncorrelated samples."""
    import math
    from scipy import stats
    from oracle import gaussian
    seed = 12345
    G = gaussian.omega(seed, 7, 2, 300, 5)
    assert G.shape == (300, 5) and np.array_equal(G, G.astype(np.float32).astype(np.float64))
    for i, c in ((0, 0), (299, 4), (17, 3)):
        t = (((7 * 64 + 2) * 64 + c) << 24) + i
        z1, z2 = (int(v) for v in inputs.splitmix64(seed, 2, 2 * t))
        u1 = ((z1 >> 40) + 1) * 2.0 ** -24
        u2 = (z2 >> 40) * 2.0 ** -24
        assert G[i, c] == float(np.float32(math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)))
    big = gaussian.omega(3, 11, 0, 40000, 5).ravel()
    assert stats.kstest(big, "norm").pvalue > 1e-3
    assert abs(big.mean()) < 0.02 and abs(big.var() - 1.0) < 0.02
    cols = np.hstack([gaussian.omega(3, leaf, rd, 20000, 2) for leaf, rd in ((0, 0), (1, 0), (0, 1))])
    cc = np.corrcoef(cols.T)
    assert np.abs(cc - np.eye(6)).max() < 0.05
    with pytest.raises(ValueError):
        gaussian.omega(3, 0, 64, 10, 2)

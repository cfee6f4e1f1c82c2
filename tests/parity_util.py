"""Comparison helpers shared by the GPU parity tests: the oracle's and the library's input pair
on the same seeded points, structure checks and the per-leaf comparison of a product with the
dense oracle product."""
import numpy as np


def _oracle_pair(oracle, P, leaf, eta, kA, kB, aca_eps, prec32=False):
    T = oracle.Tree(P, leaf, eta)
    A = oracle.HMatrix(T, kA, aca_eps, prec32=prec32)
    B = A if (kB == kA) else oracle.HMatrix(T, kB, aca_eps, prec32=prec32)
    return T, A, B


def _gpu_pair(H, P, leaf, eta, kA, kB, aca_eps, prec=64):
    A = H.hmat_build(P, kA, leaf_size=leaf, eta=eta, aca_eps=aca_eps, factor_prec=prec)
    B = A if kB == kA else H.hmat_build(P, kB, leaf_size=leaf, eta=eta, aca_eps=aca_eps, factor_prec=prec,
                                        tree_from=A)
    return A, B


def _check_structure(H, T, Hm):
    la = H.leaf_arrays(Hm)
    assert np.array_equal(Hm.permutation(), T.perm)
    ref = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    assert len(la.far) == T.nleaf
    assert np.array_equal(la.row_begin, ref[:, 0]) and np.array_equal(la.row_size, ref[:, 1])
    assert np.array_equal(la.col_begin, ref[:, 2]) and np.array_equal(la.col_size, ref[:, 3])
    assert np.array_equal(la.far, (T.leaf_blocks[:, 2] == 1).astype(np.int64))
    assert np.array_equal(la.level, T.leaf_blocks[:, 3])
    return la


def _check_product(oracle, T, C, DC, eps, near_rtol, tol_factor=1.5, rank_slack=2):
    """Compare every leaf of C with the dense oracle product DC (permuted order)."""
    worst = 0.0
    worst_near = 0.0
    n_far = 0
    for l in range(T.nleaf):
        r0, m, c0, n = T.leaf_ranges(l)
        blk = DC[r0:r0 + m, c0:c0 + n]
        if T.leaf_blocks[l, 2] == 1:
            U, V = C.leaf_get(l)
            nb = np.linalg.norm(blk)
            err = np.linalg.norm(blk - U @ V.T) / nb if nb > 0 else np.linalg.norm(U @ V.T)
            tr = oracle.truth_for_block(blk, eps, l)
            assert err <= tol_factor * eps, (l, err, U.shape[1], tr.k_eps)
            assert U.shape[1] <= tr.k_eps + rank_slack, (l, U.shape[1], tr.k_eps)
            # Eckart-Young: no rank-k approximation beats the SVD tail
            k = U.shape[1]
            assert err * nb >= np.sqrt(np.sum(tr.s[k:] ** 2)) * (1 - 1e-3) - 1e-13 * nb
            worst = max(worst, err)
            n_far += 1
        else:
            D = C.leaf_get(l)
            e = np.abs(D - blk).max() / max(np.abs(blk).max(), 1e-300)
            assert e <= near_rtol, (l, e)
            worst_near = max(worst_near, e)
    return worst, worst_near, n_far


def sampled_far_near(T, n_far, n_near, seed, max_mn=512 * 512):
    """Far leaves stratified by level (at most m*n = max_mn entries each) and near leaves, drawn
    with a seeded generator: the blocks a large product is checked on."""
    rng = np.random.default_rng(seed)
    lv = T.leaf_blocks[:, 3]
    kind = T.leaf_blocks[:, 2]
    sizes = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    mn = sizes[:, 1] * sizes[:, 3]
    far = []
    cands = [np.nonzero((lv == level) & (kind == 1) & (mn <= max_mn))[0] for level in sorted(set(lv.tolist()))]
    cands = [c for c in cands if len(c)]
    per = max(1, n_far // max(1, len(cands)))
    for cand in cands:
        far += rng.choice(cand, size=min(per, len(cand)), replace=False).tolist()
    near_c = np.nonzero(kind != 1)[0]
    near = rng.choice(near_c, size=min(n_near, len(near_c)), replace=False).tolist()
    return far, near


def check_sampled(oracle, T, Ao, Bo, C, eps, near_rtol, far, near, tol_factor=1.5, rank_slack=2):
    """The sampled leaves of C against the exact blocks A|tau x I * B|I x sigma of the oracle's
    inputs: far leaves within tol_factor * eps with rank <= eps-rank + rank_slack, near leaves
    within near_rtol in relative Frobenius norm."""
    worst = 0.0
    for l in far:
        r0, m, c0, n = T.leaf_ranges(l)
        blk = oracle.block_product_blas(Ao, Bo, r0, m, c0, n)
        U, V = C.leaf_get(l)
        nb = np.linalg.norm(blk)
        err = np.linalg.norm(blk - U @ V.T) / nb if nb > 0 else np.linalg.norm(U @ V.T)
        tr = oracle.truth_for_block(blk, eps, l)
        assert err <= tol_factor * eps, (l, err, U.shape[1], tr.k_eps)
        assert U.shape[1] <= tr.k_eps + rank_slack, (l, U.shape[1], tr.k_eps)
        worst = max(worst, err)
    for l in near:
        r0, m, c0, n = T.leaf_ranges(l)
        blk = oracle.block_product_blas(Ao, Bo, r0, m, c0, n)
        D = C.leaf_get(l)
        e = np.linalg.norm(D - blk) / max(np.linalg.norm(blk), 1e-300)
        assert e <= near_rtol, (l, e)
    return worst


def read_tree_golden(path):
    """Parse a hand-derived tree fixture of tests/golden/: the points' closed form is in its
    header; returns (perm, counts dict, leaves dict keyed by (row_begin, row_size, col_begin,
    col_size) -> (level, far, n_lowrank, n_hpairs, [low-rank terms created per level ...]))."""
    perm, counts, leaves = None, {}, {}
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "perm":
            perm = np.array([int(x) for x in f[1:]], np.int64)
        elif f[0] == "counts":
            counts = {f[i]: int(f[i + 1]) for i in range(1, len(f), 2)}
        elif f[0] == "leaf":
            r0, m, c0, n, lev = (int(x) for x in f[1:6])
            leaves[(r0, m, c0, n)] = (lev, f[6] == "F", int(f[7]), int(f[8]), [int(x) for x in f[9:]])
    return perm, counts, leaves

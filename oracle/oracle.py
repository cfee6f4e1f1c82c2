"""FP64 CPU oracle for the H-matrix product with blockwise eps-best truncation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the CUDA library never does, and the two share no code.
The only thing both sides use is the seeded point generator (``paper_1805_08998_gb300.inputs``),
which holds none of the method's arithmetic.

The oracle computes the result the paper targets, by its plain definition:
  * the stored inputs A_H, B_H are built from the points (cluster tree Def. 2.2, admissibility
    Def. 2.3, block tree Algorithm 1, near leaves dense, far leaves by ACA Algorithm 6 stopped
    by eq. (truncaca)), all in hmat_oracle.c;
  * the exact product D_C = D_A D_B of the stored H-matrices (Sec. 3.1: L = HK);
  * for every far leaf b of the product's block tree (the same tree, Sec. 3: all matrices on
    one block tree) the SVD of D_C|b and the eps-rank: the smallest k with relative Frobenius
    truncation error <= eps (Sec. 6, definition of the eps-rank); Eckart-Young gives the best
    approximation and its error;
  * near leaves are exact (Algorithm 4: near leaves are evaluated, not truncated).
For large products the exact block C|b = A|tau x I * B|I x sigma is computed for sampled
blocks only (`block_product`).

Every function is pinned by tests/test_oracle.py (brute force at tiny N, closed forms,
Eckart-Young, rank monotonicity in eps, an independent library SVD at small sizes, the
structure theorems of Sec. 5). Readings of points the paper leaves open are listed in
hmat_oracle.c beside the code that takes them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmat_oracle.c")
_LIB = os.path.join(_HERE, "libhmat_oracle.so")

KERNEL_EXP = 0   # exp(-|x-y|)
KERNEL_INVQ = 1  # 1 / (1 + |x-y|^2)
KERNEL_POLY2 = 2  # (1 + x.y)^2, separable: global rank <= (d+1)(d+2)/2

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)


def build() -> str:
    """Compile hmat_oracle.c with gcc (no FMA contraction, OpenMP)."""
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_tree_build.restype = _P
        L.or_tree_build.argtypes = [_PD, _I64, ctypes.c_int, ctypes.c_int, _D]
        L.or_tree_free.argtypes = [_P]
        L.or_tree_counts.argtypes = [_P, _PI64]
        L.or_tree_export.argtypes = [_P, _PI64, _PI64, _PI64, _PI64]
        L.or_hmat_build.restype = _P
        L.or_hmat_build.argtypes = [_P, ctypes.c_int, _D, ctypes.c_int, ctypes.c_int]
        L.or_hmat_free.argtypes = [_P]
        L.or_hmat_ranks.argtypes = [_P, _PI64]
        L.or_hmat_leaf.argtypes = [_P, ctypes.c_int, _PD, _PD]
        L.or_hmat_dense_sub.argtypes = [_P, _I64, _I64, _I64, _I64, _PD, _I64]
        L.or_matmul.argtypes = [_PD, _PD, _PD, _I64, _I64, _I64]
        L.or_block_product.argtypes = [_P, _P, _I64, _I64, _I64, _I64, _I64, _PD]
        L.or_svd.restype = ctypes.c_int
        L.or_svd.argtypes = [_PD, _I64, _I64, _PD, _PD, _PD]
        L.or_eps_rank.restype = _I64
        L.or_eps_rank.argtypes = [_PD, _I64, _D]
        L.or_svd_values_qrcp.restype = _I64
        L.or_svd_values_qrcp.argtypes = [_PD, _I64, _I64, _D, _PD, _PD]
        L.or_sumexpr_counts.argtypes = [_P, _PI64, _PI64, _PI64]
        L.or_sumexpr_eval.restype = ctypes.c_int
        L.or_sumexpr_eval.argtypes = [_P, _P, ctypes.c_int, _PD]
        L.or_num_threads.restype = ctypes.c_int
        L.or_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _pd(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _pi(a: np.ndarray):
    return a.ctypes.data_as(_PI64)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def num_threads() -> int:
    return int(lib().or_num_threads())


class Tree:
    """Cluster tree (Def. 2.2) + block-cluster tree (Algorithm 1) on the given points."""

    def __init__(self, pts: np.ndarray, leaf_size: int, eta: float):
        pts = np.ascontiguousarray(pts, dtype=np.float64)
        self.pts = pts
        self.n, self.dim = pts.shape
        self.leaf_size, self.eta = leaf_size, eta
        self._h = lib().or_tree_build(_pd(pts), self.n, self.dim, leaf_size, float(eta))
        if not self._h:
            raise ValueError("invalid tree parameters")
        cnt = np.zeros(4, np.int64)
        lib().or_tree_counts(self._h, _pi(cnt))
        self.ncl, self.nbl, self.nleaf, self.depth = (int(x) for x in cnt)
        self.perm = np.zeros(self.n, np.int64)
        self.cl = np.zeros((self.ncl, 5), np.int64)     # level, begin, size, child0, child1
        self.bl = np.zeros((self.nbl, 6), np.int64)     # tau, sigma, kind, level, leaf, nchild
        self.bl_child = np.zeros((self.nbl, 4), np.int64)
        lib().or_tree_export(self._h, _pi(self.perm), _pi(self.cl), _pi(self.bl), _pi(self.bl_child))
        leaves = self.bl[self.bl[:, 4] >= 0]
        order = np.argsort(leaves[:, 4])
        self.leaf_blocks = leaves[order]                # per leaf: tau, sigma, kind, level, leaf, nchild

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_tree_free(self._h)
            self._h = None

    def leaf_ranges(self, leaf: int):
        tau, sigma = int(self.leaf_blocks[leaf, 0]), int(self.leaf_blocks[leaf, 1])
        return (int(self.cl[tau, 1]), int(self.cl[tau, 2]), int(self.cl[sigma, 1]), int(self.cl[sigma, 2]))

    def far_leaves(self):
        return np.nonzero(self.leaf_blocks[:, 2] == 1)[0]

    def near_leaves(self):
        return np.nonzero(self.leaf_blocks[:, 2] == 2)[0]

    def sumexpr_counts(self):
        """Per leaf: (#low-rank terms, #H-pairs, low-rank terms created per level), by Alg. 3/4."""
        L = self.nleaf
        lr = np.zeros(L, np.int64)
        hp = np.zeros(L, np.int64)
        at = np.zeros(L * (self.depth + 1), np.int64)
        lib().or_sumexpr_counts(self._h, _pi(lr), _pi(hp), _pi(at))
        return lr, hp, at.reshape(L, self.depth + 1)

    def csp(self) -> int:
        """C_sp (Sec. 2): the largest number of blocks tau x sigma in the tree for one tau."""
        cnt = np.bincount(self.bl[:, 0], minlength=self.ncl)
        return int(cnt.max())


class HMatrix:
    """Kernel matrix assembled on a Tree: near leaves dense, far leaves by ACA (Alg. 6)."""

    def __init__(self, tree: Tree, kernel: int, aca_eps: float, aca_kmax: int = 256, prec32: bool = False):
        self.tree = tree
        self.kernel = kernel
        self.prec32 = bool(prec32)
        self._h = lib().or_hmat_build(tree._h, int(kernel), float(aca_eps), int(aca_kmax), int(self.prec32))
        self.ranks = np.zeros(tree.nleaf, np.int64)
        lib().or_hmat_ranks(self._h, _pi(self.ranks))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_hmat_free(self._h)
            self._h = None

    def leaf(self, l: int):
        r0, m, c0, n = self.tree.leaf_ranges(l)
        k = int(self.ranks[l])
        if k < 0:
            D = np.zeros((n, m), np.float64)  # column-major m x n stored as (n, m) rows
            lib().or_hmat_leaf(self._h, l, _pd(D), _pd(D))
            return D.T.copy()
        U = np.zeros((k, m), np.float64)
        V = np.zeros((k, n), np.float64)
        if k > 0:
            lib().or_hmat_leaf(self._h, l, _pd(U), _pd(V))
        return U.T.copy(), V.T.copy()

    def dense_sub(self, r0: int, m: int, c0: int, n: int) -> np.ndarray:
        """Dense block of the stored H-matrix, permuted order, as an (m, n) array."""
        out = np.zeros((n, m), np.float64)
        lib().or_hmat_dense_sub(self._h, r0, m, c0, n, _pd(out), m)
        return out.T.copy()

    def dense(self) -> np.ndarray:
        N = self.tree.n
        return self.dense_sub(0, N, 0, N)


def matmul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Plain triple-loop product (ascending inner index), FP64."""
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    Af = np.asfortranarray(A, dtype=np.float64)
    Bf = np.asfortranarray(B, dtype=np.float64)
    C = np.zeros((m, n), np.float64, order="F")
    lib().or_matmul(Af.ctypes.data_as(_PD), Bf.ctypes.data_as(_PD), C.ctypes.data_as(_PD), m, k, n)
    return np.ascontiguousarray(C)


def sumexpr_eval(A: HMatrix, B: HMatrix, leaf: int):
    """Dense S(leaf) built by Algorithm 3 along the root-to-leaf path, and its #low-rank terms."""
    r0, m, c0, n = A.tree.leaf_ranges(leaf)
    out = np.zeros((n, m), np.float64)
    nt = lib().or_sumexpr_eval(A._h, B._h, int(leaf), _pd(out))
    if nt < 0:
        raise RuntimeError("leaf not reachable")
    return out.T.copy(), nt


def block_product(A: HMatrix, B: HMatrix, r0: int, m: int, c0: int, n: int, chunk: int = 512) -> np.ndarray:
    """Exact C|tau x sigma = A|tau x I * B|I x sigma (permuted ranges)."""
    out = np.zeros((n, m), np.float64)
    lib().or_block_product(A._h, B._h, r0, m, c0, n, chunk, _pd(out))
    return out.T.copy()


def block_product_blas(A: HMatrix, B: HMatrix, r0: int, m: int, c0: int, n: int, chunk: int = 0) -> np.ndarray:
    """The exact block C|tau x sigma = A|tau x I * B|I x sigma, as block_product computes it, with
    the row slab of A and the column slab of B densified chunk by chunk by the oracle's own leaf
    evaluation and each chunk's product taken by numpy's matmul (BLAS) as a library primitive.
    For the samples of the largest products (N = 524288), where the plain loop takes seconds
    per block. The default chunk keeps each slab near 256 MB."""
    N = A.tree.n
    if chunk <= 0:
        chunk = max(8192, min(N, (1 << 25) // max(m, n, 1)))
    chunk = min(chunk, max(N, 1))
    out = np.zeros((m, n), np.float64)
    Ab = np.empty((m, chunk), np.float64, order="F")   # column-major, leading dimension m
    for k0 in range(0, N, chunk):
        kc = min(chunk, N - k0)
        Bb = np.empty((kc, n), np.float64, order="F")  # column-major, leading dimension kc
        lib().or_hmat_dense_sub(A._h, r0, m, k0, kc, Ab.ctypes.data_as(_PD), m)
        lib().or_hmat_dense_sub(B._h, k0, kc, c0, n, Bb.ctypes.data_as(_PD), kc)
        out += Ab[:, :kc] @ Bb
    return out


def svd(M: np.ndarray, vectors: bool = True):
    """One-sided Jacobi SVD (own code). Returns (s, U, V) with M = U diag(s) V^T."""
    M = np.asfortranarray(M, dtype=np.float64)
    m, n = M.shape
    p = min(m, n)
    s = np.zeros(p, np.float64)
    if p == 0:
        return s, np.zeros((m, 0)), np.zeros((n, 0))
    U = np.zeros((m, p), np.float64, order="F") if vectors else None
    V = np.zeros((n, p), np.float64, order="F") if vectors else None
    rc = lib().or_svd(M.ctypes.data_as(_PD), m, n, _pd(s),
                      U.ctypes.data_as(_PD) if vectors else None,
                      V.ctypes.data_as(_PD) if vectors else None)
    if rc < 0:
        raise RuntimeError("Jacobi SVD did not converge")
    return s, U, V


def eps_rank(s: np.ndarray, eps: float) -> int:
    """Smallest k with ||s[k:]||_2 <= eps * ||s||_2 (Sec. 6 eps-rank, reading: '<=')."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    return int(lib().or_eps_rank(_pd(s), len(s), float(eps)))


# Blocks with min(m, n) >= QRCP_MIN take their singular values from the pivoted QR (one-sided
# Jacobi on the triangular factor) when eps >= 1e3 * QRCP_TOL: the dropped energy, at most
# QRCP_TOL * ||block||_F, is then at most a thousandth of the eps-tail. The full one-sided Jacobi
# costs O(n^3) per sweep (about 40 s for a 1024 x 1024 block on one core).
QRCP_MIN = 129
QRCP_TOL = 1e-13


def svd_values_lowrank(M: np.ndarray, tol: float = QRCP_TOL):
    """Singular values of a block of low numerical rank by Householder QR with column pivoting,
    stopped once the remaining columns have norm <= tol * ||M||_F, then the one-sided Jacobi on
    the triangular factor. Returns (s, resid): the k values found (descending) and the remaining
    block's Frobenius norm, which bounds the energy of the values not returned."""
    M = np.asfortranarray(M, dtype=np.float64)
    m, n = M.shape
    s = np.zeros(max(min(m, n), 1), np.float64)
    resid = ctypes.c_double(0.0)
    k = lib().or_svd_values_qrcp(M.ctypes.data_as(_PD), m, n, float(tol), _pd(s), ctypes.byref(resid))
    return s[:k].copy(), resid.value


@dataclass
class BlockTruth:
    leaf: int
    norm: float             # ||D_C|b||_F
    s: np.ndarray           # singular values of D_C|b
    k_eps: int              # eps-rank
    tail: float             # sqrt(sum_{i >= k_eps} s_i^2)


def truth_for_block(Cb: np.ndarray, eps: float, leaf: int = -1) -> BlockTruth:
    """The block's singular values, eps-rank and eps-tail. Large blocks (min(m, n) >= QRCP_MIN)
    at eps >= 1e3 * QRCP_TOL use svd_values_lowrank and count the undetermined remainder in the
    tail and the norm."""
    if min(Cb.shape) >= QRCP_MIN and eps >= 1e3 * QRCP_TOL:
        s, resid = svd_values_lowrank(Cb)
        se = np.append(s, resid) if resid > 0.0 else s
        k = min(eps_rank(se, eps), len(s))
        return BlockTruth(leaf, float(np.sqrt(np.sum(se * se))), s, k, float(np.sqrt(np.sum(se[k:] ** 2))))
    s, _, _ = svd(Cb, vectors=False)
    k = eps_rank(s, eps)
    return BlockTruth(leaf, float(np.sqrt(np.sum(s * s))), s, k, float(np.sqrt(np.sum(s[k:] ** 2))))


def best_approx(Cb: np.ndarray, eps: float):
    """Eckart-Young best approximation at the eps-rank: (U_k diag(s_k), V_k)."""
    s, U, V = svd(Cb, vectors=True)
    k = eps_rank(s, eps)
    return U[:, :k] * s[:k], V[:, :k]


def product_truth(A: HMatrix, B: HMatrix, eps: float):
    """Full dense oracle (small N): D_C and the per-far-leaf truth."""
    DA, DB = A.dense(), B.dense()
    DC = matmul(DA, DB)
    t = A.tree
    truths = {}
    for l in t.far_leaves():
        r0, m, c0, n = t.leaf_ranges(int(l))
        truths[int(l)] = truth_for_block(DC[r0:r0 + m, c0:c0 + n], eps, int(l))
    return DC, truths

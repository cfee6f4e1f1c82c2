"""Thin ctypes binding of libhmat.so: the same names as the C-ABI in include/hmat.h.

Argument marshalling only; every step of the product runs in the library's CUDA kernels.
Loading fails loudly (ImportError) when the library has not been built, and every call that
fails raises HmatError with the library's status and message -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhmat.so")

HMAT_OK, HMAT_EINVAL, HMAT_ENOMEM, HMAT_ECUDA, HMAT_ENOTCONV, HMAT_ETIMEOUT, HMAT_EMISMATCH = range(7)
STATUS_NAMES = {0: "HMAT_OK", 1: "HMAT_EINVAL", 2: "HMAT_ENOMEM", 3: "HMAT_ECUDA", 4: "HMAT_ENOTCONV",
                5: "HMAT_ETIMEOUT", 6: "HMAT_EMISMATCH"}

K_EXP, K_INVQ, K_POLY2 = 0, 1, 2
PTS_CUBE, PTS_SPHERE = 0, 1
MODE_F64, MODE_MIXED = 0, 1
# compressor of the sum-expressions: Algorithm 8 / Algorithm 6 / Algorithm 7
COMP_RANDOMIZED, COMP_ACA, COMP_LANCZOS = 0, 1, 2

# every symbol include/hmat.h declares
EXPORTS = ["hmat_points", "hmat_build", "hmat_plan_host", "hmat_multiply", "hmat_multiply_batched", "hmat_to_dense",
           "hmat_leaf_count", "hmat_leaf_info",
           "hmat_leaf_get", "hmat_permutation", "hmat_stats", "hmat_sumexpr_counts", "hmat_destroy",
           "hmat_data_bytes", "hmat_data_get", "hmat_rank_features", "hmat_rankmodel_train",
           "hmat_rankmodel_predict", "hmat_rankmodel_get", "hmat_rankmodel_create", "hmat_rankmodel_grad",
           "hmat_rankmodel_grad_noalloc", "hmat_rankmodel_destroy", "hmat_matvec", "hmat_product_error", "hmat_last_error", "hmat_set_allocator",
           "hmat_check_bounded_wait"]

RANK_FEATURES = 12
RANK_PARAMS = 5057
RANKGRAD_NOALLOC_MAX = 16384
PROP_NONE, PROP_LEARNED, PROP_HEURISTIC = 0, 1, 2


class HmatError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class BuildOpts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("eta", ctypes.c_double), ("aca_eps", ctypes.c_double),
                ("factor_prec", ctypes.c_int), ("aca_kmax", ctypes.c_int)]


class MultOpts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("mode", ctypes.c_int), ("rank_proposal", ctypes.c_int),
                ("max_rank", ctypes.c_int), ("max_rounds", ctypes.c_int), ("block_width", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("rank_model", ctypes.c_void_p), ("fixed_rank", ctypes.c_int),
                ("power_iters", ctypes.c_int), ("compressor", ctypes.c_int)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("lr", ctypes.c_float), ("seed", ctypes.c_uint64)]


class Leaf(ctypes.Structure):
    _fields_ = [("row_begin", ctypes.c_int64), ("row_size", ctypes.c_int64), ("col_begin", ctypes.c_int64),
                ("col_size", ctypes.c_int64), ("level", ctypes.c_int), ("far", ctypes.c_int),
                ("rank", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("depth", ctypes.c_int), ("csp", ctypes.c_int),
                ("n_far", ctypes.c_int64), ("n_near", ctypes.c_int64), ("storage_bytes", ctypes.c_int64),
                ("factor_prec", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("n_terms", ctypes.c_int64), ("n_lr_refs", ctypes.c_int64), ("n_hpairs", ctypes.c_int64),
                ("rounds", ctypes.c_int), ("not_converged", ctypes.c_int64),
                ("flops_apply", ctypes.c_double), ("flops_terms", ctypes.c_double),
                ("flops_near", ctypes.c_double), ("bytes_apply", ctypes.c_double),
                ("ms_plan", ctypes.c_double), ("ms_terms", ctypes.c_double), ("ms_near", ctypes.c_double),
                ("ms_sample", ctypes.c_double), ("ms_final", ctypes.c_double),
                ("ms_apply", ctypes.c_double), ("apply_launches", ctypes.c_int64),
                ("bytes_apply_use", ctypes.c_double), ("launches", ctypes.c_int64),
                ("n_ff_jobs", ctypes.c_int64), ("n_panels", ctypes.c_int64),
                ("first_round_cols", ctypes.c_int64), ("done_in_first_round", ctypes.c_int64),
                ("sample_passes", ctypes.c_int64), ("groups", ctypes.c_int64),
                ("bytes_apply_unique", ctypes.c_double), ("apply_gstage_targets", ctypes.c_int64),
                ("apply_split_targets", ctypes.c_int64), ("apply_max_split", ctypes.c_int),
                ("bytes_terms_use", ctypes.c_double), ("ms_near_kernel", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PF = ctypes.POINTER(ctypes.c_float)
_lib = None


def lib():
    """Load libhmat.so (built by __graft_entry__.build() / build_lib.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (paper_1805_08998_gb300.build_lib)")
    L = ctypes.CDLL(LIB_PATH)
    L.hmat_points.argtypes = [ctypes.c_int, ctypes.c_int, _I64, ctypes.c_uint64, _PD]
    L.hmat_build.argtypes = [_PD, _I64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(BuildOpts), _P, _P,
                             ctypes.POINTER(_P)]
    L.hmat_multiply.argtypes = [_P, _P, ctypes.POINTER(MultOpts), _P, ctypes.POINTER(_P)]
    L.hmat_multiply_batched.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int,
                                        ctypes.POINTER(MultOpts), _P, ctypes.POINTER(_P)]
    L.hmat_to_dense.argtypes = [_P, _PD, _I64]
    L.hmat_leaf_count.argtypes = [_P, _PI64]
    L.hmat_leaf_info.argtypes = [_P, _I64, ctypes.POINTER(Leaf)]
    L.hmat_leaf_get.argtypes = [_P, _I64, _PD, _PD]
    L.hmat_permutation.argtypes = [_P, _PI64]
    L.hmat_stats.argtypes = [_P, ctypes.POINTER(Stats)]
    L.hmat_sumexpr_counts.argtypes = [_P, _P, _PI64, _PI64]
    L.hmat_plan_host.argtypes = [_PD, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_double, _PI64, _PI64,
                                 ctypes.POINTER(Leaf), _PI64, _PI64, _I64, ctypes.POINTER(ctypes.c_int)]
    L.hmat_data_bytes.argtypes = [_P, _PI64]
    L.hmat_data_get.argtypes = [_P, _P, _I64]
    L.hmat_rank_features.argtypes = [_P, _P, ctypes.c_double, _P, _PF, _PF, _PI64]
    L.hmat_rankmodel_train.argtypes = [_PF, _PF, _I64, ctypes.POINTER(TrainOpts), _P, ctypes.POINTER(_P)]
    L.hmat_rankmodel_predict.argtypes = [_P, _PF, _I64, _PF]
    L.hmat_rankmodel_get.argtypes = [_P, _PF, _PF, _PF, _PF]
    L.hmat_rankmodel_create.argtypes = [_PF, _PF, _PF, ctypes.POINTER(_P)]
    L.hmat_rankmodel_grad.argtypes = [_P, _PF, _PF, _I64, _PF, _PF]
    L.hmat_rankmodel_grad_noalloc.argtypes = [_P, _PF, _PF, _I64, _PF, _PF, _P]
    L.hmat_matvec.argtypes = [_P, _PD, _PD, _I64, _P]
    L.hmat_product_error.argtypes = [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _PD]
    L.hmat_check_bounded_wait.argtypes = [ctypes.c_int]
    L.hmat_rankmodel_destroy.argtypes = [_P]
    L.hmat_rankmodel_destroy.restype = None
    L.hmat_destroy.argtypes = [_P]
    L.hmat_destroy.restype = None
    L.hmat_last_error.restype = ctypes.c_char_p
    for name in ["hmat_points", "hmat_build", "hmat_plan_host", "hmat_multiply", "hmat_multiply_batched", "hmat_to_dense",
                 "hmat_leaf_count",
                 "hmat_leaf_info", "hmat_leaf_get", "hmat_permutation", "hmat_stats", "hmat_sumexpr_counts",
                 "hmat_set_allocator", "hmat_data_bytes", "hmat_data_get", "hmat_rank_features",
                 "hmat_rankmodel_train", "hmat_rankmodel_predict", "hmat_rankmodel_get", "hmat_rankmodel_create",
                 "hmat_rankmodel_grad", "hmat_rankmodel_grad_noalloc", "hmat_matvec", "hmat_product_error",
                 "hmat_check_bounded_wait"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int, allow=()):
    if status != HMAT_OK and status not in allow:
        raise HmatError(status, lib().hmat_last_error().decode())
    return status


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class HMatrix:
    """Owner of an hmat_t; released with hmat_destroy."""

    def __init__(self, handle: int):
        self._h = handle
        self.last_status = HMAT_OK

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "_h", None):
            lib().hmat_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def leaf_count(self) -> int:
        n = ctypes.c_int64()
        _check(lib().hmat_leaf_count(self._h, ctypes.byref(n)))
        return n.value

    def leaf_info(self, i: int) -> Leaf:
        info = Leaf()
        _check(lib().hmat_leaf_info(self._h, i, ctypes.byref(info)))
        return info

    def leaf_get(self, i: int):
        info = self.leaf_info(i)
        m, n = info.row_size, info.col_size
        if not info.far:
            D = np.zeros((n, m), np.float64)
            _check(lib().hmat_leaf_get(self._h, i, D.ctypes.data_as(_PD), None))
            return D.T.copy()
        k = info.rank
        U = np.zeros((k, m), np.float64)
        V = np.zeros((k, n), np.float64)
        if k > 0:
            _check(lib().hmat_leaf_get(self._h, i, U.ctypes.data_as(_PD), V.ctypes.data_as(_PD)))
        return U.T.copy(), V.T.copy()

    def leaves(self):
        return [self.leaf_info(i) for i in range(self.leaf_count())]

    def to_dense(self) -> np.ndarray:
        n = self.stats()["n"]
        out = np.zeros((n, n), np.float64)  # filled column-major -> transpose view
        _check(lib().hmat_to_dense(self._h, out.ctypes.data_as(_PD), n))
        return out.T.copy()

    def permutation(self) -> np.ndarray:
        n = self.stats()["n"]
        perm = np.zeros(n, np.int64)
        _check(lib().hmat_permutation(self._h, perm.ctypes.data_as(_PI64)))
        return perm

    def data_bytes(self) -> int:
        n = ctypes.c_int64()
        _check(lib().hmat_data_bytes(self._h, ctypes.byref(n)))
        return n.value

    def data_get(self, out) -> None:
        """Copy the packed factor buffer into `out` (a host buffer: numpy array or a pinned
        torch tensor's data_ptr() with its byte size given as a (ptr, nbytes) tuple)."""
        if isinstance(out, tuple):
            ptr, nbytes = out
        else:
            ptr, nbytes = out.ctypes.data, out.nbytes
        _check(lib().hmat_data_get(self._h, ctypes.c_void_p(ptr), nbytes))

    def stats(self) -> dict:
        s = Stats()
        _check(lib().hmat_stats(self._h, ctypes.byref(s)))
        return s.as_dict()


def hmat_points(dist: int, dim: int, n: int, seed: int) -> np.ndarray:
    out = np.zeros((n, dim), np.float64)
    _check(lib().hmat_points(dist, dim, n, seed, out.ctypes.data_as(_PD)))
    return out


def hmat_build(xyz: np.ndarray, kernel: int, leaf_size: int = 32, eta: float = 1.0, aca_eps: float = 1e-10,
               factor_prec: int = 64, aca_kmax: int = 0, tree_from: HMatrix | None = None, stream=None) -> HMatrix:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n, dim = xyz.shape
    opts = BuildOpts(leaf_size, eta, aca_eps, factor_prec, aca_kmax)
    h = _P()
    _check(lib().hmat_build(xyz.ctypes.data_as(_PD), n, dim, kernel, ctypes.byref(opts),
                            tree_from.handle if tree_from is not None else None, _stream_ptr(stream),
                            ctypes.byref(h)))
    return HMatrix(h.value)


def hmat_multiply(A: HMatrix, B: HMatrix, eps: float, mode: int = MODE_F64, rank_proposal: int = 0,
                  max_rank: int = 0, max_rounds: int = 0, block_width: int = 0, seed: int = 0,
                  stream=None, allow_notconv: bool = True, rank_model: "RankModel | None" = None,
                  fixed_rank: int = 0, power_iters: int = -1, compressor: int = COMP_RANDOMIZED) -> HMatrix:
    opts = MultOpts(eps, mode, rank_proposal, max_rank, max_rounds, block_width, seed,
                    rank_model.handle if rank_model is not None else None, fixed_rank, power_iters, compressor)
    h = _P()
    st = lib().hmat_multiply(A.handle, B.handle, ctypes.byref(opts), _stream_ptr(stream), ctypes.byref(h))
    _check(st, allow=(HMAT_ENOTCONV,) if allow_notconv else ())
    C = HMatrix(h.value)
    C.last_status = st
    return C


def hmat_multiply_batched(As, Bs, eps: float, mode: int = MODE_F64, rank_proposal: int = 0, max_rank: int = 0,
                          max_rounds: int = 0, block_width: int = 0, seed: int = 0, stream=None,
                          allow_notconv: bool = True, rank_model: "RankModel | None" = None,
                          compressor: int = COMP_RANDOMIZED):
    """Products As[i] Bs[i] in one call; returns the list of outputs."""
    n = len(As)
    if len(Bs) != n:
        raise _shape_error(f"{n} left factors but {len(Bs)} right factors")
    opts = MultOpts(eps, mode, rank_proposal, max_rank, max_rounds, block_width, seed,
                    rank_model.handle if rank_model is not None else None, 0, -1, compressor)
    a = (_P * max(n, 1))(*[x.handle for x in As])
    b = (_P * max(n, 1))(*[x.handle for x in Bs])
    c = (_P * max(n, 1))()
    st = lib().hmat_multiply_batched(a, b, n, ctypes.byref(opts), _stream_ptr(stream), c)
    _check(st, allow=(HMAT_ENOTCONV,) if allow_notconv else ())
    out = []
    for i in range(n):
        h = HMatrix(c[i])
        h.last_status = st
        out.append(h)
    return out


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None  # the callbacks handed to the library, kept alive while it may call them


def hmat_set_allocator(alloc=None, free=None) -> None:
    """Route the library's device allocations through alloc(nbytes, stream) -> device pointer
    (int; 0 or None for failure) and free(ptr); both None restores the default pool. The callables
    must not raise (an exception inside a C callback is printed and ignored)."""
    global _allocator_refs
    if (alloc is None) != (free is None):
        raise _shape_error("alloc and free must both be given or both be None")
    if alloc is None:
        _check(lib().hmat_set_allocator(None, None, None))
        _allocator_refs = None
        return
    a = ALLOC_FN(lambda nbytes, stream, ctx: alloc(nbytes, stream) or None)
    f = FREE_FN(lambda ptr, ctx: free(ptr))
    _check(lib().hmat_set_allocator(a, f, None))
    _allocator_refs = (a, f)


def hmat_matvec(Hm: HMatrix, x, stream=None) -> np.ndarray:
    """y = H x for x of shape (n,) or (n, ncols), original point order."""
    x = np.asarray(x, np.float64)
    vec = x.ndim == 1
    if x.ndim not in (1, 2) or x.shape[0] != Hm.stats()["n"]:
        raise _shape_error(f"x must have shape (n,) or (n, ncols) with n = {Hm.stats()['n']}, got {x.shape}")
    X = np.asfortranarray(x.reshape(x.shape[0], -1))
    Y = np.zeros_like(X, order="F")
    _check(lib().hmat_matvec(Hm.handle, X.ctypes.data_as(_PD), Y.ctypes.data_as(_PD), X.shape[1], _stream_ptr(stream)))
    return Y[:, 0].copy() if vec else np.ascontiguousarray(Y)


def hmat_check_bounded_wait(polls: int) -> int:
    """Status of the library's bounded-wait check (HMAT_ETIMEOUT when the wait gave up)."""
    return lib().hmat_check_bounded_wait(polls)


def hmat_product_error(A: HMatrix, B: HMatrix, C: HMatrix, iters: int = 10, size: int = 100, seed: int = 0) -> float:
    out = ctypes.c_double()
    _check(lib().hmat_product_error(A.handle, B.handle, C.handle, iters, size, seed, ctypes.byref(out)))
    return out.value


@dataclass
class PlanHost:
    perm: np.ndarray
    leaves: "LeafArrays"
    n_lowrank: np.ndarray
    n_hpairs: np.ndarray
    csp: int


def hmat_plan_host(points, leaf_size: int = 64, eta: float = 1.0) -> PlanHost:
    """Cluster tree, block tree and per-leaf sum-expression counts on the host (no GPU)."""
    P = np.ascontiguousarray(points, np.float64)
    if P.ndim == 1:
        P = P[:, None]
    n, dim = P.shape
    L = lib()
    nl = ctypes.c_int64()
    _check(L.hmat_plan_host(P.ctypes.data_as(_PD), n, dim, leaf_size, eta, None, ctypes.byref(nl), None, None,
                            None, 0, None))
    k = nl.value
    perm = np.zeros(n, np.int64)
    lv = (Leaf * max(k, 1))()
    lr = np.zeros(k, np.int64)
    hp = np.zeros(k, np.int64)
    csp = ctypes.c_int()
    _check(L.hmat_plan_host(P.ctypes.data_as(_PD), n, dim, leaf_size, eta, perm.ctypes.data_as(_PI64),
                            ctypes.byref(nl), lv, lr.ctypes.data_as(_PI64), hp.ctypes.data_as(_PI64), k,
                            ctypes.byref(csp)))
    rec = np.ctypeslib.as_array(lv)[:k]  # the hmat_leaf records as a structured array (no copy)
    cols = {f: rec[f].astype(np.int64) for f in ("row_begin", "row_size", "col_begin", "col_size", "level", "far",
                                                 "rank")}
    return PlanHost(perm, LeafArrays(**cols), lr, hp, int(csp.value))


def hmat_sumexpr_counts(A: HMatrix, B: HMatrix):
    L = A.leaf_count()
    lr = np.zeros(L, np.int64)
    hp = np.zeros(L, np.int64)
    _check(lib().hmat_sumexpr_counts(A.handle, B.handle, lr.ctypes.data_as(_PI64), hp.ctypes.data_as(_PI64)))
    return lr, hp


@dataclass
class LeafArrays:
    """Leaf geometry of an H-matrix as numpy arrays (permuted ranges)."""
    row_begin: np.ndarray
    row_size: np.ndarray
    col_begin: np.ndarray
    col_size: np.ndarray
    far: np.ndarray
    rank: np.ndarray
    level: np.ndarray


def leaf_arrays(H: HMatrix) -> LeafArrays:
    infos = H.leaves()
    f = lambda k: np.array([getattr(x, k) for x in infos], np.int64)
    return LeafArrays(f("row_begin"), f("row_size"), f("col_begin"), f("col_size"), f("far"), f("rank"), f("level"))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _shape_error(msg: str) -> HmatError:
    # the C side sees only pointers and counts, so array shapes are checked here
    return HmatError(HMAT_EINVAL, msg)


def _samples(features, ranks=None):
    """features as a (count, RANK_FEATURES) float32 array; ranks, if given, as count float32."""
    X = _f32(features)
    if X.ndim != 2 or X.shape[1] != RANK_FEATURES:
        raise _shape_error(f"features must have shape (count, {RANK_FEATURES}), got {X.shape}")
    if ranks is None:
        return X
    y = _f32(ranks).reshape(-1)
    if y.shape[0] != X.shape[0]:
        raise _shape_error(f"{X.shape[0]} feature rows but {y.shape[0]} ranks")
    return X, y


class RankModel:
    """Owner of an hmat_rankmodel_t (the learned rank proposal); released with
    hmat_rankmodel_destroy."""

    def __init__(self, handle: int):
        self._h = handle

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "_h", None):
            lib().hmat_rankmodel_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def predict(self, features) -> np.ndarray:
        X = _samples(features)
        out = np.zeros(X.shape[0], np.float32)
        _check(lib().hmat_rankmodel_predict(self._h, X.ctypes.data_as(_PF), X.shape[0], out.ctypes.data_as(_PF)))
        return out

    def get(self):
        """(weights, mean, dev, loss): the FP16 weights widened to float32, the feature
        normalisation and the final training loss."""
        w = np.zeros(RANK_PARAMS, np.float32)
        mu = np.zeros(RANK_FEATURES, np.float32)
        dv = np.zeros(RANK_FEATURES, np.float32)
        loss = ctypes.c_float()
        _check(lib().hmat_rankmodel_get(self._h, w.ctypes.data_as(_PF), mu.ctypes.data_as(_PF),
                                        dv.ctypes.data_as(_PF), ctypes.byref(loss)))
        return w, mu, dv, loss.value

    def grad(self, features, ranks):
        X, y = _samples(features, ranks)
        g = np.zeros(RANK_PARAMS, np.float32)
        loss = ctypes.c_float()
        _check(lib().hmat_rankmodel_grad(self._h, X.ctypes.data_as(_PF), y.ctypes.data_as(_PF), X.shape[0],
                                         g.ctypes.data_as(_PF), ctypes.byref(loss)))
        return g, loss.value


def hmat_rankmodel_grad_noalloc(model: RankModel, features, ranks, stream=None, want_loss: bool = True):
    """hmat_rankmodel_grad without device allocation (fixed scratch; at most
    RANKGRAD_NOALLOC_MAX samples; concurrent calls on one device race). With want_loss=False the
    loss pointer is NULL and the loss returned is None."""
    X, y = _samples(features, ranks)
    g = np.zeros(RANK_PARAMS, np.float32)
    loss = ctypes.c_float()
    _check(lib().hmat_rankmodel_grad_noalloc(model.handle, X.ctypes.data_as(_PF), y.ctypes.data_as(_PF), X.shape[0],
                                             g.ctypes.data_as(_PF), ctypes.byref(loss) if want_loss else None,
                                             _stream_ptr(stream)))
    return g, (loss.value if want_loss else None)


def hmat_rank_features(A: HMatrix, B: HMatrix, eps: float, C: HMatrix | None = None):
    """(features n_far x RANK_FEATURES, ranks of C on those blocks or zeros)."""
    n = ctypes.c_int64()
    _check(lib().hmat_rank_features(A.handle, B.handle, eps, None, None, None, ctypes.byref(n)))
    F = np.zeros((n.value, RANK_FEATURES), np.float32)
    r = np.zeros(n.value, np.float32)
    _check(lib().hmat_rank_features(A.handle, B.handle, eps, C.handle if C is not None else None,
                                    F.ctypes.data_as(_PF), r.ctypes.data_as(_PF), ctypes.byref(n)))
    return F, r


def hmat_rankmodel_train(features, ranks, epochs: int = 0, lr: float = 0.0, seed: int = 0,
                         stream=None) -> RankModel:
    X, y = _samples(features, ranks)
    opts = TrainOpts(epochs, lr, seed)
    h = _P()
    _check(lib().hmat_rankmodel_train(X.ctypes.data_as(_PF), y.ctypes.data_as(_PF), X.shape[0], ctypes.byref(opts),
                                      _stream_ptr(stream), ctypes.byref(h)))
    return RankModel(h.value)


def hmat_rankmodel_create(weights, mean, dev) -> RankModel:
    w, mu, dv = _f32(weights).reshape(-1), _f32(mean).reshape(-1), _f32(dev).reshape(-1)
    if w.shape[0] != RANK_PARAMS or mu.shape[0] != RANK_FEATURES or dv.shape[0] != RANK_FEATURES:
        raise _shape_error(f"need {RANK_PARAMS} weights and {RANK_FEATURES} means and deviations, got "
                           f"{w.shape[0]}, {mu.shape[0]}, {dv.shape[0]}")
    h = _P()
    _check(lib().hmat_rankmodel_create(w.ctypes.data_as(_PF), mu.ctypes.data_as(_PF), dv.ctypes.data_as(_PF),
                                       ctypes.byref(h)))
    return RankModel(h.value)

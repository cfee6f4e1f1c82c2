"""Host-side checks of the C-ABI library that need no GPU: it builds, loads, exports every
symbol include/hmat.h declares, validates its arguments, and its point generator matches
the shared seeded generator."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1805_08998_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "hmat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmat_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(H):
    declared = _declared_symbols()
    assert "hmat_multiply" in declared and "hmat_build" in declared
    L = H.lib()
    for name in declared:
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value
    assert sorted(H.EXPORTS) == declared


def test_header_is_plain_c(H, tmp_path):
    """include/hmat.h is a C header: a C99 program that includes it compiles without warnings
    under -Wall -Wextra -pedantic, links against libhmat.so and calls it."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text("""#include "hmat.h"
#include <stdio.h>
int main(void) {
  hmat_build_opts b = {32, 1.0, 1e-10, 64, 0};
  hmat_mult_opts m = {0};
  hmat_stats_t st;
  hmat_leaf lf;
  double xyz[6];
  hmat_status s = hmat_points(HMAT_PTS_SPHERE, 3, 2, 7, xyz);
  (void)b; (void)m; (void)st; (void)lf;
  printf("%d %.17g\\n", (int)s, xyz[5]);
  return s == HMAT_OK ? 0 : 1;
}
""")
    lib_dir = os.path.dirname(H.LIB_PATH)
    exe = tmp_path / "abi"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", lib_dir, "-lhmat",
                        "-Wl,-rpath," + lib_dir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    st, z = r.stdout.split()
    assert int(st) == 0 and float(z) == inputs.points(1, 3, 2, 7)[1, 2]


@pytest.mark.parametrize("dist,dim,n,seed", [(0, 1, 17, 3), (0, 2, 1000, 0), (0, 3, 333, 9), (1, 3, 500, 0)])
def test_points_match_shared_generator(H, dist, dim, n, seed):
    a = H.hmat_points(dist, dim, n, seed)
    b = inputs.points(dist, dim, n, seed)
    if dist == 0:
        assert np.array_equal(a, b)
    else:  # cos/sin of two math libraries may differ in the last bit
        assert np.abs(a - b).max() <= 4e-16


def test_generator_matches_published_splitmix64(H):
    """The seeded stream behind every synthetic input is splitmix64: the shared module's outputs
    and the library's cube points (u = (output >> 11) 2^-53, one draw per coordinate) reproduce the
    generator's published outputs for seeds 0 and 1234567."""
    ref = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "splitmix64.txt")):
        f = line.split()
        if f and f[0] == "seed":
            ref[int(f[1])] = [int(x) for x in f[2:]]
    for seed, outs in ref.items():
        got = inputs.splitmix64(seed, len(outs))
        assert [int(x) for x in got] == outs
        u = H.hmat_points(0, 1, len(outs), seed)[:, 0]
        assert [int(x) for x in (u * 2.0 ** 53).astype(np.uint64)] == [o >> 11 for o in outs]


def test_argument_validation(H):
    xyz = inputs.points(0, 2, 100, 0)
    with pytest.raises(H.HmatError) as e:
        H.hmat_build(xyz, 0, leaf_size=0)
    assert e.value.status == H.HMAT_EINVAL
    with pytest.raises(H.HmatError) as e:  # n_min = 1 would make empty clusters (Def. 2.2)
        H.hmat_build(xyz, 0, leaf_size=1)
    assert e.value.status == H.HMAT_EINVAL
    with pytest.raises(H.HmatError) as e:  # the kernels' shared-memory layouts hold leaves of <= 64 points
        H.hmat_build(xyz, 0, leaf_size=65)
    assert e.value.status == H.HMAT_EINVAL
    with pytest.raises(H.HmatError) as e:
        H.hmat_build(xyz, 0, leaf_size=16, eta=-1.0)
    assert e.value.status == H.HMAT_EINVAL
    with pytest.raises(H.HmatError) as e:
        H.hmat_build(xyz, 0, leaf_size=16, factor_prec=16)
    assert e.value.status == H.HMAT_EINVAL
    with pytest.raises(H.HmatError) as e:
        H.hmat_build(xyz, 7, leaf_size=16)
    assert e.value.status == H.HMAT_EINVAL
    bad = xyz.copy()
    bad[3, 1] = np.nan
    with pytest.raises(H.HmatError) as e:
        H.hmat_build(bad, 0, leaf_size=16)
    assert e.value.status == H.HMAT_EINVAL
    assert "non-finite" in str(e.value)
    # NULL handles
    L = H.lib()
    out = ctypes.c_void_p()
    opts = H.MultOpts(1e-6, 0, 0, 0, 0, 0, 0)
    assert L.hmat_multiply(None, None, ctypes.byref(opts), None, ctypes.byref(out)) == H.HMAT_EINVAL
    assert out.value is None
    assert L.hmat_leaf_count(None, None) == H.HMAT_EINVAL
    assert L.hmat_set_allocator(ctypes.c_void_p(1), None, None) == H.HMAT_EINVAL
    with pytest.raises(H.HmatError):
        H.hmat_points(1, 2, 10, 0)
    for dist in (2, -1, 1 << 30):  # enum arguments outside the enumeration
        with pytest.raises(H.HmatError) as e:
            H.hmat_points(dist, 3, 10, 0)
        assert e.value.status == H.HMAT_EINVAL
    for kernel in (-1, 3, 1 << 30):
        with pytest.raises(H.HmatError) as e:
            H.hmat_build(xyz, kernel, leaf_size=16)
        assert e.value.status == H.HMAT_EINVAL


def test_binding_checks_array_shapes(H):
    """The C-ABI sees only pointers and counts, so the binding checks array shapes before a call:
    a wrongly shaped array raises HMAT_EINVAL instead of letting the library read or write past
    its end. (These checks run before any device is touched.)"""
    F = H.RANK_FEATURES
    bad = [lambda: H.hmat_rankmodel_create(np.zeros(10), np.zeros(F), np.ones(F)),
           lambda: H.hmat_rankmodel_create(np.zeros(H.RANK_PARAMS), np.zeros(F - 1), np.ones(F)),
           lambda: H.hmat_rankmodel_train(np.zeros((10, F - 5)), np.ones(10)),
           lambda: H.hmat_rankmodel_train(np.zeros((10, F)), np.ones(9)),
           lambda: H.RankModel(None).predict(np.zeros((3, F + 1))),
           lambda: H.RankModel(None).grad(np.zeros((3, F)), np.zeros(4)),
           lambda: H.hmat_rankmodel_grad_noalloc(H.RankModel(None), np.zeros(F), np.zeros(1)),
           lambda: H.hmat_multiply_batched([], [None], 1e-6)]
    for call in bad:
        with pytest.raises(H.HmatError) as e:
            call()
        assert e.value.status == H.HMAT_EINVAL


def test_last_error_is_thread_local(H):
    import threading
    L = H.lib()
    assert L.hmat_leaf_count(None, None) == H.HMAT_EINVAL
    msg_main = L.hmat_last_error().decode()
    seen = {}

    def worker():
        seen["t"] = L.hmat_last_error().decode()

    th = threading.Thread(target=worker)
    th.start()
    th.join()
    assert msg_main and seen["t"] == ""


@pytest.mark.skipif(any(os.path.exists(f"/dev/nvidia{i}") for i in range(16)),
                    reason="checks the behaviour without a CUDA device")
def test_no_device_returns_status(H):
    """Without a usable CUDA device, the entry points that need one return HMAT_ECUDA with a
    message and leave their output handle NULL; nothing aborts across the ABI, and the library
    stays usable for host-only calls."""
    F = H.RANK_FEATURES
    P = inputs.points(0, 2, 300, 0)
    calls = [lambda: H.hmat_build(P, 0, leaf_size=16),
             lambda: H.hmat_rankmodel_create(np.zeros(H.RANK_PARAMS, np.float32), np.zeros(F), np.ones(F)),
             lambda: H.hmat_rankmodel_train(np.zeros((10, F), np.float32), np.ones(10, np.float32))]
    for call in calls:
        with pytest.raises(H.HmatError) as e:
            call()
        assert e.value.status == H.HMAT_ECUDA and H.lib().hmat_last_error()
    L = H.lib()
    out = ctypes.c_void_p(1)
    opts = H.BuildOpts(16, 1.0, 1e-8, 64, 0)
    assert L.hmat_build(P.ctypes.data_as(H._PD), 300, 2, 0, ctypes.byref(opts), None, None,
                        ctypes.byref(out)) == H.HMAT_ECUDA
    assert out.value is None
    ph = H.hmat_plan_host(P, leaf_size=16)
    assert len(ph.perm) == 300 and H.lib().hmat_last_error() == b""


@pytest.mark.parametrize("kind,dim,n,leaf,eta", [(0, 2, 2048, 32, 1.0), (1, 3, 3000, 32, 1.0), (0, 3, 1531, 16, 1.0),
                                                 (0, 1, 777, 8, 0.5), (0, 2, 300, 16, 2.0), (0, 3, 1, 4, 1.0),
                                                 (0, 2, 101, 2, 1.0), (0, 3, 5, 2, 1.0)])
def test_plan_host_matches_oracle(H, oracle, kind, dim, n, leaf, eta):
    """a0/a1 host logic without a GPU: the library's cluster tree (Def. 2.2), block tree
    (Algorithm 1, Def. 2.3) and restriction plan (Algorithm 3) give, bit for bit, the oracle's
    permutation, leaf geometry, admissibility, levels, C_sp and per-leaf counts of low-rank terms
    and H-pairs."""
    P = inputs.points(kind, dim, n, 11)
    T = oracle.Tree(P, leaf, eta)
    ph = H.hmat_plan_host(P, leaf_size=leaf, eta=eta)
    assert np.array_equal(ph.perm, T.perm)
    la = ph.leaves
    assert len(la.far) == T.nleaf
    ref = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    assert np.array_equal(la.row_begin, ref[:, 0]) and np.array_equal(la.row_size, ref[:, 1])
    assert np.array_equal(la.col_begin, ref[:, 2]) and np.array_equal(la.col_size, ref[:, 3])
    assert np.array_equal(la.far, (T.leaf_blocks[:, 2] == 1).astype(np.int64))
    assert np.array_equal(la.level, T.leaf_blocks[:, 3])
    assert np.array_equal(la.rank, np.where(la.far == 1, 0, -1))
    assert ph.csp == T.csp()
    lr, hp, _ = T.sumexpr_counts()
    assert np.array_equal(ph.n_lowrank, lr) and np.array_equal(ph.n_hpairs, hp)


def _degenerate_points(case):
    if case == "duplicates":   # 40 distinct points, each 25 times: ties everywhere
        return np.repeat(inputs.points(0, 3, 40, 1), 25, axis=0)
    if case == "identical":    # one point 500 times: zero boxes, nothing admissible
        return np.zeros((500, 2))
    if case == "collinear":    # a segment in 3-D: two box sides stay proportional
        t = inputs.uniform01(6, 1000)
        return np.stack([t, 2 * t, -t], 1)
    if case == "two_clusters":  # two well separated squares
        return np.concatenate([inputs.points(0, 2, 500, 2), inputs.points(0, 2, 500, 3) + 10.0])
    g = np.arange(12.0)         # integer grid: equal box sides and tied coordinates
    X, Y = np.meshgrid(g, g)
    return np.stack([X.ravel(), Y.ravel()], 1)


@pytest.mark.parametrize("case,leaf", [("duplicates", 16), ("identical", 8), ("collinear", 16),
                                       ("two_clusters", 16), ("grid", 4)])
def test_plan_host_degenerate_geometry(H, oracle, case, leaf):
    """Ties, zero-size boxes and collinear points: the library's trees and plan still equal the
    oracle's bit for bit (split ties by original index, first longest side, distance 0 never
    admissible)."""
    P = _degenerate_points(case)
    T = oracle.Tree(P, leaf, 1.0)
    ph = H.hmat_plan_host(P, leaf_size=leaf, eta=1.0)
    assert np.array_equal(ph.perm, T.perm)
    la = ph.leaves
    ref = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    assert len(la.far) == T.nleaf
    assert np.array_equal(la.row_begin, ref[:, 0]) and np.array_equal(la.col_begin, ref[:, 2])
    assert np.array_equal(la.far, (T.leaf_blocks[:, 2] == 1).astype(np.int64))
    assert ph.csp == T.csp()
    lr, hp, _ = T.sumexpr_counts()
    assert np.array_equal(ph.n_lowrank, lr) and np.array_equal(ph.n_hpairs, hp)
    if case == "identical":
        assert la.far.sum() == 0


def test_plan_host_arguments(H):
    P = inputs.points(0, 2, 100, 0)
    L = H.lib()
    for args in [(None, 100, 2, 16, 1.0), (P, 0, 2, 16, 1.0), (P, 100, 4, 16, 1.0), (P, 100, 2, 0, 1.0),
                 (P, 100, 2, 1, 1.0), (P, 100, 2, 129, 1.0), (P, 100, 2, 16, 0.0), (P, 100, 2, 16, float("nan"))]:
        pts, n, dim, leaf, eta = args
        ptr = pts.ctypes.data_as(H._PD) if pts is not None else None
        assert L.hmat_plan_host(ptr, n, dim, leaf, eta, None, None, None, None, None, 0, None) == H.HMAT_EINVAL
    bad = P.copy()
    bad[7, 0] = np.inf
    assert L.hmat_plan_host(bad.ctypes.data_as(H._PD), 100, 2, 16, 1.0, None, None, None, None, None, 0,
                            None) == H.HMAT_EINVAL
    # a partial leaf buffer: only the first max_leaves entries are written
    full = H.hmat_plan_host(P, leaf_size=8)
    lr = np.full(5, -7, np.int64)
    nl = ctypes.c_int64()
    assert L.hmat_plan_host(P.ctypes.data_as(H._PD), 100, 2, 8, 1.0, None, ctypes.byref(nl), None,
                            lr[:3].ctypes.data_as(H._PI64), None, 3, None) == H.HMAT_OK
    assert nl.value == len(full.n_lowrank) and np.array_equal(lr[:3], full.n_lowrank[:3]) and np.all(lr[3:] == -7)


def test_bounded_wait_check_arguments(H):
    """The bounded-wait check rejects poll counts outside 1..2^22 before it touches a device."""
    for bad in (0, -1, (1 << 22) + 1):
        assert H.hmat_check_bounded_wait(bad) == H.HMAT_EINVAL
        assert b"polls" in H.lib().hmat_last_error()


def test_plan_host_matches_hand_derived_example(H):
    """The library's trees and restriction plan against the worked example derived by hand in
    tests/golden/tree_1d_n16_leaf2_eta1.txt (Def. 2.2, Def. 2.3, Algorithms 1 and 3)."""
    from parity_util import read_tree_golden
    perm, counts, leaves = read_tree_golden(os.path.join(ROOT, "tests", "golden", "tree_1d_n16_leaf2_eta1.txt"))
    P = (((5 * np.arange(16) + 3) % 16) / 16.0).reshape(16, 1)
    ph = H.hmat_plan_host(P, leaf_size=2, eta=1.0)
    assert np.array_equal(ph.perm, perm)
    assert ph.csp == counts["csp"]
    la = ph.leaves
    assert len(la.far) == counts["leaves"] and int(la.far.sum()) == counts["far"]
    got = {}
    for l in range(len(la.far)):
        key = (int(la.row_begin[l]), int(la.row_size[l]), int(la.col_begin[l]), int(la.col_size[l]))
        got[key] = (int(la.level[l]), bool(la.far[l]), int(ph.n_lowrank[l]), int(ph.n_hpairs[l]))
    assert got == {k: v[:4] for k, v in leaves.items()}


@pytest.mark.parametrize("kind,n", [(1, 32768), (0, 131072)])
def test_plan_host_full_size(H, oracle, kind, n):
    """Integer work at full size, bit-exact: the benchmark's sphere workload (N = 32768) and the
    3-D workload of the learned proposal (N = 131072), leaf 64, eta 1: permutation, leaf
    geometry and admissibility, C_sp and every leaf's term and H-pair counts."""
    dim = 3
    P = inputs.points(kind, dim, n, 0)
    T = oracle.Tree(P, 64, 1.0)
    ph = H.hmat_plan_host(P, leaf_size=64, eta=1.0)
    assert np.array_equal(ph.perm, T.perm)
    la = ph.leaves
    assert len(la.far) == T.nleaf
    assert np.array_equal(la.far, (T.leaf_blocks[:, 2] == 1).astype(np.int64))
    assert np.array_equal(la.level, T.leaf_blocks[:, 3])
    ref = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    assert np.array_equal(la.row_begin, ref[:, 0]) and np.array_equal(la.col_size, ref[:, 3])
    assert ph.csp == T.csp()
    lr, hp, _ = T.sumexpr_counts()
    assert np.array_equal(ph.n_lowrank, lr) and np.array_equal(ph.n_hpairs, hp)

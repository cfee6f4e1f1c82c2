#!/usr/bin/env python
"""Benchmark of the H x H product with blockwise eps-best truncation on one GB300.

Workload (the paper's setting, Sec. 6.1, with synthetic stand-ins for its Galerkin sphere
matrices): N = 32768 points uniform on the unit sphere (seed 0), A with k = exp(-r), B with
k = 1/(1+r^2), cardinality-balanced bisection with leaf size 64, eta = 1, far leaves by ACA
to 1e-8 stored in FP32, C = A B truncated to relative Frobenius error eps = 1e-6 per block.

One step = one hmat_multiply (all of the hot path: symbolic restriction, low-rank products,
adaptive randomized sampling + FP64 orthogonalisation, core truncation, near field). The
"chosen form" is MODE_MIXED (FP32 contractions, FP64 orthogonalisation and core SVD); the
plain FP64 GPU path (MODE_F64) is timed beside it.

value = degrees of freedom per second (N / product time; the paper reports seconds per
degree of freedom), summed over ranks. Inputs (A, B: ~0.7 GB of FP32 factors) exceed the
129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1805_08998_gb300 import inputs  # noqa: E402

METRIC = "H×H product time & GFLOP/s at ε=1e-6: chosen form vs plain FP64 GPU; %roofline"
WORKLOAD = {
    "workload": "hxh_sphere_n32768_exp_x_invq_leaf64_eta1_fp32factors_eps1e-6",
    "n": 32768, "points": "uniform on unit sphere S^2, seed 0", "kernel_A": "exp(-r)",
    "kernel_B": "1/(1+r^2)", "leaf_size": 64, "eta": 1.0, "aca_eps": 1e-8, "factor_prec": 32,
    "eps": 1e-6, "block_width": 8, "inputs_exceed_l2": True,
}
UNIT = "DOF/s"
FP64_TFLOPS = 1.25  # nominal GB300 FP64 (non-tensor) rate


def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class Replicas:
    """Host side of an N-rank run of the benchmark: every rank computes the whole workload on its
    own GPU (the product does not shard across GPUs here), the ranks meet at barriers around the
    timed region, and the slowest rank's time is the job's time."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def replica_value(n_points: int, ms_max: float, world: int) -> float:
    """Whole-job throughput in degrees of freedom per second: every rank multiplies its own
    N-point product, so the job does world * N degrees of freedom in the slowest rank's time."""
    return world * n_points / (ms_max * 1e-3)


def reference_runs_here(rank: int, world: int) -> bool:
    """The oracle arm runs on rank 0 only; other ranks exit without work."""
    return world <= 1 or rank == 0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _tf32_peak():
    """Dense TF32 tensor rate: the measured sustained bf16 GEMM rate (the near-field kernel runs
    inside a long step) times the nominal TF32 : bf16 ratio of GB300 (1.1 : 2.25 PFLOP/s)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops_sustained" in d:
            return float(d["bf16_tflops_sustained"]) * 1.1 / 2.25, "measured sustained bf16 x 1.1/2.25"
    return 1700.0 * 1.1 / 2.25, "fallback sustained bf16 (1.7 PFLOP/s) x 1.1/2.25"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic_from_profile():
    """DRAM bytes (read + write) of one sum-expression application pass (all size classes)
    from the committed ncu summary, if it was taken on the current kernel source (the summary
    records the sha256 of hmat_apply.cuh); otherwise None."""
    prof = os.path.join(ROOT, "profiles", "k_apply_sphere_n32768.md")
    src = os.path.join(ROOT, "paper_1805_08998_gb300", "csrc", "hmat_apply.cuh")
    if not (os.path.exists(prof) and os.path.exists(src)):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    txt = open(prof).read()
    if f"kernel source sha256: {sha}" not in txt:
        return None
    for line in txt.splitlines():
        if line.startswith("dram_bytes_per_pass:"):
            return float(line.split(":")[1])
    return None


# ------------------------------------------------------------------------------------ CPU oracle

def oracle_sample(n_blocks_per_level=2, seed=0, threads=None, budget_s=25.0, min_s=0.0, setup=None):
    """Time the oracle on a stratified sample of target blocks of the workload and extrapolate
    to the whole product: exact block C|b = A|tau x I * B|I x sigma (cost ~ m n N) plus the
    SVD truncation of far blocks (cost ~ m n min(m, n)). Returns (estimated seconds for the full
    product, description, threads used, setup). Levels are visited in passes, n_blocks_per_level
    new blocks of each per pass, until at least min_s seconds of oracle work are done (or the
    candidates run out); no block starts after budget_s."""
    from oracle import oracle as O
    if threads:
        O.set_threads(threads)
    W = WORKLOAD
    if setup is None:
        P = inputs.points(inputs.PTS_SPHERE, 3, W["n"], 0)
        T = O.Tree(P, W["leaf_size"], W["eta"])
        A = O.HMatrix(T, O.KERNEL_EXP, W["aca_eps"], prec32=True)
        B = O.HMatrix(T, O.KERNEL_INVQ, W["aca_eps"], prec32=True)
        setup = (T, A, B)
    T, A, B = setup
    N = T.n
    rng = np.random.default_rng(seed)
    lv = T.leaf_blocks[:, 3]
    far = T.leaf_blocks[:, 2] == 1
    sizes = np.array([T.leaf_ranges(l) for l in range(T.nleaf)])
    mn = sizes[:, 1] * sizes[:, 3]
    c_prod, c_svd = [], []
    t_start = time.perf_counter()
    done = 0
    pools = []
    for level in sorted(set(lv.tolist()), reverse=True):
        cand = np.nonzero((lv == level) & (mn <= 256 * 256))[0]
        if len(cand):
            pools.append(list(rng.permutation(cand)))
    while True:
        took = 0
        for pool in pools:
            for _ in range(n_blocks_per_level):
                if not pool or time.perf_counter() - t_start > budget_s:
                    break
                l = pool.pop()
                r0, m, c0, n = sizes[l]
                t0 = time.perf_counter()
                blk = O.block_product(A, B, r0, m, c0, n)
                t1 = time.perf_counter()
                c_prod.append((t1 - t0) / (m * n * N))
                if far[l]:
                    O.truth_for_block(blk, W["eps"])
                    c_svd.append((time.perf_counter() - t1) / (m * n * min(m, n)))
                done += 1
                took += 1
        elapsed = time.perf_counter() - t_start
        if took == 0 or elapsed >= min_s or elapsed > budget_s:
            break
    cp = float(np.mean(c_prod))
    cs = float(np.mean(c_svd)) if c_svd else 0.0
    svd_work = float(np.sum((mn * np.minimum(sizes[:, 1], sizes[:, 3]))[far]))
    t_est = cp * float(np.sum(mn)) * N + cs * svd_work
    desc = (f"{done} blocks (stratified by level, m*n <= 256^2; {time.perf_counter() - t_start:.1f} s of "
            f"oracle work) of the N={N} product: exact block products "
            f"and SVD truncations timed, extrapolated to all {T.nleaf} leaves by cost ~ m*n*N (+ m*n*min(m,n) "
            f"for the far-block SVDs)")
    return t_est, desc, O.num_threads(), setup


CONFIG1 = {"workload": "hxh_cube2d_n2048_exp_leaf32_eta1_aca1e-10_f64_eps1e-6", "n": 2048,
           "points": "uniform in [0,1]^2, seed 0", "kernel": "exp(-r)", "leaf_size": 32, "eta": 1.0,
           "aca_eps": 1e-10, "eps": 1e-6}


def oracle_config1(threads):
    """The full dense oracle on the N = 2048 case, measured rather than extrapolated: D_C = D_A D_B
    of the stored inputs and the SVD truncation of every far block. Returns (seconds, threads)."""
    from oracle import oracle as O
    O.set_threads(threads)
    C1 = CONFIG1
    P = inputs.points(inputs.PTS_CUBE, 2, C1["n"], 0)
    T = O.Tree(P, C1["leaf_size"], C1["eta"])
    A = O.HMatrix(T, O.KERNEL_EXP, C1["aca_eps"])
    t0 = time.perf_counter()
    O.product_truth(A, A, C1["eps"])
    return time.perf_counter() - t0, O.num_threads()


# ------------------------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, _, world = _rank_env()
    if not reference_runs_here(rank, world):
        return
    setup = None
    for w in range(args.warmup):
        _, _, _, setup = oracle_sample(n_blocks_per_level=1, seed=100 + w, budget_s=5.0, setup=setup)
    vals = []
    t0 = time.perf_counter()
    desc, thr = "", 0
    for k in range(args.steps):
        t_est, desc, thr, setup = oracle_sample(n_blocks_per_level=1, seed=k, budget_s=15.0, min_s=10.0,
                                                setup=setup)
        vals.append(WORKLOAD["n"] / t_est)
    wall = time.perf_counter() - t0
    v = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * WORKLOAD["n"] / v, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism="replicas" if world > 1 else "single"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": desc + "; one stratified sample per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat as H

    rank, local_rank, world = _rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    W = WORKLOAD
    P = inputs.points(inputs.PTS_SPHERE, 3, W["n"], 0)
    A = H.hmat_build(P, H.K_EXP, leaf_size=W["leaf_size"], eta=W["eta"], aca_eps=W["aca_eps"],
                     factor_prec=W["factor_prec"], stream=stream)
    B = H.hmat_build(P, H.K_INVQ, leaf_size=W["leaf_size"], eta=W["eta"], aca_eps=W["aca_eps"],
                     factor_prec=W["factor_prec"], tree_from=A, stream=stream)

    def mult(mode, seed):
        return H.hmat_multiply(A, B, W["eps"], mode=mode, block_width=W["block_width"], seed=seed, stream=stream)

    rep = Replicas(dist, dev)
    barrier, max_over_ranks = rep.barrier, rep.max

    # ---- warm-up (chosen form and plain FP64)
    for w in range(max(args.warmup, 3)):
        C = mult(H.MODE_MIXED, 1000 + w)
    del C
    C = mult(H.MODE_F64, 999)
    del C
    torch.cuda.synchronize()

    # ---- timed: chosen form
    stats = []
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        for k in range(args.steps):
            C = mult(H.MODE_MIXED, k)
            stats.append(C.stats())
            last_status = C.last_status
            del C
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)

    # ---- timed: plain FP64 GPU path (same workload, same number of steps)
    k64 = args.steps
    s64 = []
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(k64):
        C = mult(H.MODE_F64, k)
        s64.append(C.stats())
        del C
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms64 = max_over_ranks(e0.elapsed_time(e1) / k64)

    # ---- end to end through the public API with host buffers: H2D of the points from pinned
    # memory, both builds (GPU ACA), the product, and D2H of C's packed factors to pinned memory
    pts_pinned = torch.from_numpy(P.copy()).pin_memory()
    C = mult(H.MODE_MIXED, 0)
    out_bytes = C.data_bytes()
    del C
    # C's packed size varies slightly with the test matrices (ranks differ by one here and
    # there): size the pinned buffer with a margin
    host_out = torch.empty(int(out_bytes * 1.5) + (1 << 20), dtype=torch.uint8).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0
    xyz = pts_pinned.numpy()  # pinned host buffer; hmat_build copies it to the device itself
    for k in range(e2e_steps):
        h2d += pts_pinned.numel() * 8
        Ae = H.hmat_build(xyz, H.K_EXP, leaf_size=W["leaf_size"], eta=W["eta"], aca_eps=W["aca_eps"],
                          factor_prec=W["factor_prec"], stream=stream)
        Be = H.hmat_build(xyz, H.K_INVQ, leaf_size=W["leaf_size"], eta=W["eta"], aca_eps=W["aca_eps"],
                          factor_prec=W["factor_prec"], tree_from=Ae, stream=stream)
        Ce = H.hmat_multiply(Ae, Be, W["eps"], mode=H.MODE_MIXED, block_width=W["block_width"], seed=k,
                             stream=stream)
        nb = Ce.data_bytes()
        Ce.data_get((host_out.data_ptr(), host_out.numel()))
        d2h += nb
        del Ae, Be, Ce
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps)

    # ---- the N = 2048 case on the GPU (FP64 path), for the measured CPU comparison
    C1 = CONFIG1
    P1 = inputs.points(inputs.PTS_CUBE, 2, C1["n"], 0)
    A1 = H.hmat_build(P1, H.K_EXP, leaf_size=C1["leaf_size"], eta=C1["eta"], aca_eps=C1["aca_eps"],
                      factor_prec=64, stream=stream)
    c1_ms = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C = H.hmat_multiply(A1, A1, C1["eps"], mode=H.MODE_F64, seed=k, stream=stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            c1_ms.append((time.perf_counter() - t0) * 1e3)
        del C
    c1_gpu_ms = max_over_ranks(float(np.median(c1_ms)))

    st = stats[-1]
    flops = st["flops_terms"] + st["flops_near"] + st["flops_apply"]
    gflops = flops / (ms * 1e-3) / 1e9
    st64 = s64[-1]
    flops64 = st64["flops_terms"] + st64["flops_near"] + st64["flops_apply"]
    # dominant kernel: the sum-expression application (k_apply), timed by CUDA events on the
    # call's stream inside the library
    apply_ms = np.mean([s["ms_apply"] for s in stats])
    apply_launches = np.mean([s["apply_launches"] for s in stats])
    apply_bytes = np.mean([s["bytes_apply_use"] for s in stats])
    apply_unique = np.mean([s["bytes_apply_unique"] for s in stats])
    per_launch_ms = apply_ms / max(apply_launches, 1)
    # primary basis: the unique bytes of a pass (every referenced factor element once, plus the
    # panels); secondary: per use (each target reads its whole sum-expression)
    achieved = (apply_unique / max(apply_launches, 1)) / (per_launch_ms * 1e-3) / 1e9
    achieved_use = (apply_bytes / max(apply_launches, 1)) / (per_launch_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    traffic = _traffic_from_profile()
    # the low-rank products (a2, panels and far x far products): per-use bytes over the phase's
    # device time (CUDA events on the call's stream around the phase)
    terms_ms = np.mean([s["ms_terms"] for s in stats])
    terms_bytes = np.mean([s["bytes_terms_use"] for s in stats])
    terms_gbs = terms_bytes / (terms_ms * 1e-3) / 1e9
    near_ms = np.mean([s["ms_near_kernel"] for s in stats])
    near_flops = 3.0 * np.mean([s["flops_near"] for s in stats])  # three TF32 products per product
    near_tf = near_flops / (near_ms * 1e-3) / 1e12
    tf32_peak, tf32_kind = _tf32_peak()
    # the FP64 path's application kernel against the FP64 pipe (nominal 1.25 TFLOP/s)
    apply64_ms = np.mean([s["ms_apply"] for s in s64])
    apply64_flops = np.mean([s["flops_apply"] for s in s64])
    fp64_tflops = apply64_flops / (apply64_ms * 1e-3) / 1e12
    launches = int(sum(s["launches"] for s in stats))
    value = replica_value(W["n"], ms, world)

    if rank == 0:
        # CPU oracle baseline on the host cores (bounded sample)
        t_est, desc, thr, _ = oracle_sample(n_blocks_per_level=2, budget_s=25.0, min_s=15.0)
        c1_all, c1_thr = oracle_config1(os.cpu_count() or 1)
        c1_one, _ = oracle_config1(1)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(W, parallelism="replicas" if world > 1 else "single"),
            "gflops": gflops,
            "plain_f64": {"ms_per_step": ms64, "value": replica_value(W["n"], ms64, world),
                          "gflops": flops64 / (ms64 * 1e-3) / 1e9, "steps": k64,
                          "roofline": {"kernel": "k_apply<double> (sum-expression application, FP64)",
                                       "bound": "fp64", "achieved": fp64_tflops, "peak": FP64_TFLOPS,
                                       "unit": "TFLOP/s", "frac": fp64_tflops / FP64_TFLOPS,
                                       "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)",
                                       "apply_ms_per_step": apply64_ms}},
            "speedup_vs_plain_f64": ms64 / ms,
            "status": int(last_status),
            "phases_ms": {k: st[k] for k in ("ms_plan", "ms_terms", "ms_sample", "ms_final", "ms_near", "ms_apply")},
            "max_rank": st["max_rank"], "rounds": st["rounds"],
            "roofline": {"kernel": "k_apply (sum-expression application)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_kind, "traffic": traffic,
                         "per_launch_ms": per_launch_ms, "launches_per_step": apply_launches,
                         "algorithmic_bytes_per_launch": apply_unique / max(apply_launches, 1),
                         "bytes_basis": "unique: per pass, every stored factor element an active target's "
                                        "sum-expression references counted once, plus the In/Out panels",
                         "achieved_use": achieved_use, "frac_use": achieved_use / peak,
                         "use_bytes_per_launch": apply_bytes / max(apply_launches, 1),
                         "use_basis": "per use: every active target's sum-expression read once per pass, "
                                      "plus its In/Out panels; terms shared by neighbouring targets count "
                                      "once per target",
                         # measured DRAM bytes of a pass (ncu) over its unique bytes: re-reads beyond
                         # the minimum; and the DRAM rate of the live pass
                         "traffic_over_unique": (traffic / (apply_unique / max(apply_launches, 1)))
                         if traffic else None,
                         "dram_gbs": (traffic / (per_launch_ms * 1e-3) / 1e9) if traffic else None,
                         "dram_frac": (traffic / (per_launch_ms * 1e-3) / 1e9 / peak) if traffic else None},
            "roofline_a2": {"kernel": "k_panel, k_panel_leaf, k_ff_warp, k_term_jobs (low-rank products)",
                            "bound": "hbm", "achieved": terms_gbs, "peak": peak, "unit": "GB/s",
                            "frac": terms_gbs / peak, "peak_source": peak_kind, "ms_per_step": terms_ms,
                            "bytes_per_step": terms_bytes,
                            "bytes_basis": "per use: every panel reads its H-block once plus its input and "
                                           "output columns; every far x far product its four factors and "
                                           "the new one"},
            "roofline_near": {"kernel": "k_near_tc (near field a8, tcgen05 kind::tf32, 3 x TF32 per FP32 product)",
                              "bound": "tensor", "achieved": near_tf, "peak": tf32_peak, "unit": "TFLOP/s",
                              "frac": near_tf / tf32_peak, "peak_source": tf32_kind, "ms_per_step": near_ms,
                              "flops_per_step": near_flops,
                              "flops_basis": "3 x (2 m n K summed over every near leaf's terms and leaf pairs): "
                                             "the TF32 products the tensor cores execute; timed with CUDA events "
                                             "on the kernel's own stream, concurrent with the sampling"},
            "cpu_baseline": {"value": W["n"] / t_est, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": desc},
            "config1_measured": {"config": CONFIG1, "gpu_f64_ms": c1_gpu_ms,
                                 "gpu_f64_value": CONFIG1["n"] / (c1_gpu_ms * 1e-3),
                                 "cpu_oracle_s": {"threads": c1_thr, "all_threads": c1_all, "one_thread": c1_one},
                                 "cpu_oracle_value": {"all_threads": CONFIG1["n"] / c1_all,
                                                      "one_thread": CONFIG1["n"] / c1_one},
                                 "unit": UNIT,
                                 "what": "GPU: hmat_multiply wall time (FP64 path, median of steps); CPU: the "
                                         "oracle's dense product of the stored inputs and the SVD truncation of "
                                         "every far block, timed in full"},
            "e2e": {"value": replica_value(W["n"], e2e_s * 1e3, world), "unit": UNIT, "h2d_bytes_per_step": h2d // e2e_steps,
                    "d2h_bytes_per_step": d2h // e2e_steps, "ms_per_step": e2e_s * 1e3,
                    "includes": "points H2D (pinned), hmat_build x2 (GPU ACA), hmat_multiply, C factors D2H (pinned)"},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

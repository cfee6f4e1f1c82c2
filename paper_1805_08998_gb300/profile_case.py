"""Run the sphere product workload at a chosen size: the driver used for ncu captures.

    python -m paper_1805_08998_gb300.profile_case --n 8192 --mode mixed --reps 2 [--compressor aca|lanczos]

Points uniform on the unit sphere (seed 0), A = exp(-r), B = 1/(1+r^2), leaf 64, eta 1,
ACA 1e-8, FP32 factors, eps 1e-6 (the benchmark's workload, scaled in N). Prints the
product's statistics as JSON, with the call's wall time (hmat_multiply synchronises at its end)
as wall_ms.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--mode", choices=["mixed", "f64"], default="mixed")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--block-width", type=int, default=8)
    ap.add_argument("--compressor", choices=["randomized", "aca", "lanczos"], default="randomized")
    args = ap.parse_args()
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat as H
    from paper_1805_08998_gb300 import inputs
    P = inputs.points(inputs.PTS_SPHERE, 3, args.n, 0)
    A = H.hmat_build(P, H.K_EXP, leaf_size=64, eta=1.0, aca_eps=1e-8, factor_prec=32)
    B = H.hmat_build(P, H.K_INVQ, leaf_size=64, eta=1.0, aca_eps=1e-8, factor_prec=32, tree_from=A)
    mode = H.MODE_MIXED if args.mode == "mixed" else H.MODE_F64
    comp = {"randomized": H.COMP_RANDOMIZED, "aca": H.COMP_ACA, "lanczos": H.COMP_LANCZOS}[args.compressor]
    for r in range(args.reps):
        t0 = time.perf_counter()
        C = H.hmat_multiply(A, B, args.eps, mode=mode, block_width=args.block_width, seed=r, compressor=comp)
        wall = (time.perf_counter() - t0) * 1e3
        st = C.stats()
        st["wall_ms"] = wall
        print(json.dumps({k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()}), flush=True)
        del C


if __name__ == "__main__":
    main()

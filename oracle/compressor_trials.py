"""Stop-rule trials of the one-vector compressors on exact product blocks -- test infrastructure.

    python -m oracle.compressor_trials [--quick]

For the exact far blocks of oracle products (the dense product of the stored inputs, restricted
to each far leaf), runs the cross approximation (Algorithm 6) and the Lanczos bidiagonalization
(Algorithm 7) of oracle/compressors.py under several readings of the stop test eq. (truncaca),
truncates the result to the eps-rank (Algorithm 5), and prints per reading how many blocks miss
the blockwise bound (error > 1.5 eps or rank > k_eps + 2), the worst error / eps and the mean
number of steps. The readings: one step meeting the test at eps/4, eps/10 or eps/32, or two
consecutive steps at eps/4 or eps/8. For comparison it also runs the blocked randomized range
finder (Algorithm 8: 8 columns per round, stop at eps/2, dropping at 0.1 eps) and reports its
rounds. Uses only the oracle, the seeded point generator and numpy's seeded Gaussians.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import compressors as X  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1805_08998_gb300 import inputs  # noqa: E402

CASES = [  # (label, points kind, dim, N, seed, leaf, kernel of A, kernel of B, eps)
    ("2-D e^-r squared", 0, 2, 2048, 0, 32, 0, 0, 1e-6),
    ("3-D e^-r x 1/(1+r^2)", 0, 3, 3000, 5, 32, 0, 1, 1e-6),
    ("3-D e^-r x 1/(1+r^2)", 0, 3, 3000, 5, 32, 0, 1, 1e-4),
    ("3-D e^-r x 1/(1+r^2)", 0, 3, 3000, 5, 32, 0, 1, 1e-8),
]
RULES = [("one at eps/4", 0.25, 1), ("one at eps/10", 0.1, 1), ("one at eps/32", 1 / 32, 1),
         ("two at eps/4", 0.25, 2), ("two at eps/8", 0.125, 2)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="first two cases only")
    args = ap.parse_args()
    O.build()
    cases = CASES[:2] if args.quick else CASES
    for label, kind, dim, n, seed, leaf, ka, kb, eps in cases:
        P = inputs.points(kind, dim, n, seed)
        T = O.Tree(P, leaf, 1.0)
        A = O.HMatrix(T, ka, 1e-10)
        B = A if kb == ka else O.HMatrix(T, kb, 1e-10)
        DC = O.matmul(A.dense(), B.dense())
        blocks = []
        for l in range(T.nleaf):
            if T.leaf_blocks[l, 2] == 1:
                r0, m, c0, nn = T.leaf_ranges(l)
                blk = DC[r0:r0 + m, c0:c0 + nn]
                blocks.append((l, blk, O.truth_for_block(blk, eps, l)))
        rng = np.random.default_rng(7)
        fails, worst, rounds = 0, 0.0, []
        for l, blk, tr in blocks:
            om = rng.standard_normal((blk.shape[1], 96))
            Q, W, rd = X.randomized(blk, om, eps, 8, 96)
            Uc, Vc = X.truncate(Q, W, eps)
            err = np.linalg.norm(blk - Uc @ Vc.T) / tr.norm
            worst = max(worst, err / eps)
            rounds.append(rd)
            if err > 1.5 * eps or Uc.shape[1] > tr.k_eps + 2:
                fails += 1
        print(f"{label:22s} N={n:5d} eps={eps:.0e} {'random':8s} {'8 per round':14s}: {fails:2d} of {len(blocks)} "
              f"blocks miss the bound, worst {worst:.2f} eps, mean rounds {np.mean(rounds):.1f}", flush=True)
        for comp in ("aca", "lanczos"):
            for name, fac, need in RULES:
                fails, worst, steps = 0, 0.0, []
                for l, blk, tr in blocks:
                    if comp == "aca":
                        L, U, k = X.aca(blk, fac * eps, 95, need)
                        Uc, Vc = X.truncate(L, U, eps)
                    else:
                        w1 = inputs.uniform01(1000 + l, blk.shape[1]) - 0.5
                        Q, _, _, _, k = X.lanczos(blk, w1, fac * eps, 95, need)
                        Uc, Vc = X.truncate(Q, blk.T @ Q, eps)
                    err = np.linalg.norm(blk - Uc @ Vc.T) / tr.norm
                    worst = max(worst, err / eps)
                    steps.append(k)
                    if err > 1.5 * eps or Uc.shape[1] > tr.k_eps + 2:
                        fails += 1
                print(f"{label:22s} N={n:5d} eps={eps:.0e} {comp:8s} {name:14s}: {fails:2d} of {len(blocks)} "
                      f"blocks miss the bound, worst {worst:.2f} eps, mean steps {np.mean(steps):.1f}", flush=True)


if __name__ == "__main__":
    main()

"""Truncation error of the m-step Krylov approximation at each workload's m.

TEST INFRASTRUCTURE ONLY: an oracle-side report, run by hand
(``python -m oracle.truncation``); nothing in the product imports it.

The m-step Lanczos result f_m is the parity target of the CUDA path; the
converged e^A 1 is a different quantity, and the gap between them is the
method's own error at the chosen depth, not the GPU's.  The converged value
is the oracle's Lanczos result with m grown in steps of 10 until
||f_{m+10} - f_m|| / ||f_m|| < 1e-13 (normwise), or until breakdown.
Reported per workload: the normwise relative error of f_m and the largest
relative error over the head (scores >= 1e-3 of the largest).
"""
import math
import sys

import numpy as np

from oracle.communicability import krylov_expv
from paper_1409_5000_gb300 import synth


def converged(n, rp, col, m0, tol=1e-13, m_max=400):
    th_a, y_a, me = krylov_expv(n, rp, col, m0)
    m = m0
    while m < m_max and me == m:
        m += 10
        th_b, y_b, me = krylov_expv(n, rp, col, m)
        a = y_a * math.exp(th_a - th_b)
        if np.linalg.norm(a - y_b) <= tol * np.linalg.norm(y_b):
            return th_b, y_b, m
        th_a, y_a = th_b, y_b
    return th_a, y_a, m


def errors(g, m):
    th_m, y_m, _ = krylov_expv(g.n, g.row_ptr, g.col, m)
    th_c, y_c, m_c = converged(g.n, g.row_ptr, g.col, m)
    a = y_m * math.exp(th_m - th_c)
    head = y_c >= 1e-3 * y_c.max()
    return (float(np.linalg.norm(a - y_c) / np.linalg.norm(y_c)),
            float(np.max(np.abs(a - y_c)[head] / y_c[head])), m_c)


def workloads():
    ens = synth.er_ensemble_small()
    yield "C1 ER(500, p=0.016) realisation 0 of 10", ens.graphs[0], 20
    for kind in ("er", "ba", "ws"):
        yield f"C2 {kind.upper()}(1e5) + 12-clique", synth.single_clique_100k(kind).graphs[0], 30
    sizes = synth.er_ensemble_uneven_sizes()
    for r in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        g = synth.er_ensemble_member(sizes, 20.0, 30, 15, 3, r)
        yield f"C3 ER(n={g.n}, d=20) realisation {r} of 256", g, 25
    yield "C4 stand-in BA(1e6, 8) + 20-clique (C4 is n = 1e7)", \
        synth.ba_clique_large(n=1_000_000).graphs[0], 40
    sizes5 = [100_000] * 64
    yield "C5 ER(1e5, d=16) realisation 0 of 64", \
        synth.er_ensemble_member(sizes5, 16.0, 25, 10, 5, 0), 30


def main():
    print("| workload | m | normwise rel. error of f_m | head max rel. error | m at convergence |")
    print("|---|---|---|---|---|")
    for name, g, m in workloads():
        nr, hd, mc = errors(g, m)
        print(f"| {name} | {m} | {nr:.2e} | {hd:.2e} | {mc} |", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Oracle work items for the full-size parity tests, run in a spawn pool.

Each item regenerates one realisation from the seeded generators (nothing
large crosses the process boundary) and evaluates the FP64 oracle on it.
This module imports neither torch nor the CUDA binding.
"""
import os

import numpy as np

import oracle.adjoint as oa
import oracle.communicability as oc
from paper_1409_5000_gb300 import synth


def ensemble_member_scores(args):
    """(r, theta_r, y_r): Krylov e^A 1 of realisation r of an ER ensemble."""
    sizes, dbar, k, extra, config, r, m = args
    g = synth.er_ensemble_member(sizes, dbar, k, extra, config, r)
    theta, y, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, m)
    return r, theta, y


def ensemble_member_grad(args):
    """(r, theta_r, g_r): Krylov edge gradient of realisation r for node set S."""
    sizes, dbar, k, extra, config, r, m, nodes = args
    g = synth.er_ensemble_member(sizes, dbar, k, extra, config, r)
    w = np.zeros(g.n)
    sel = np.asarray([x for x in nodes if x < g.n], dtype=np.int64)
    w[sel] = 1.0
    theta, gr = oa.krylov_edge_grad(g.n, g.row_ptr, g.col, w, m)
    return r, theta, gr


def pool_map(fn, items, procs=None):
    """fn over items in a spawn pool, single-threaded BLAS per worker."""
    import multiprocessing as mp

    procs = procs or min(16, os.cpu_count() or 1, len(items))
    keep = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in keep:
        os.environ[v] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            return pool.map(fn, items, chunksize=1)
    finally:
        for v, x in keep.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x

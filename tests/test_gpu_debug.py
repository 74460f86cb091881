"""The bounds-checked build (libcb_debug.so, -DCB_DEBUG) on every SpMV path.

In that build each indexed access of the SpMV kernels is checked on the
device before it happens: column-blocked stream elements and fill positions,
tiled-CSR columns, the two-phase source offsets, value-array places and
region slots.  A failed check is counted and the access skipped, so a layout
bug shows as a nonzero count instead of a fault.  The cases run in a child
process (the library is chosen when the binding first loads it) over the
column-blocked, two-phase and tiled-CSR paths, FP32 and FP64, the adjoint and
top-k; every result must meet the oracle bar and no check may fail.  Last,
a column index >= n is given to the tiled-CSR path of this build only, and
its gathers must be counted, with the site and the index, and skipped.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases():
    """Runs in the child with CB_DEBUG=1; prints one JSON line."""
    import torch

    import oracle.adjoint as oa
    import oracle.communicability as oc
    from paper_1409_5000_gb300 import binding as B
    from paper_1409_5000_gb300 import synth
    from tests import parity

    out = {"debug_build": B.cb_debug_build(), "cases": {}}
    B.cb_debug_violations(reset=True)

    def scores(graphs, m, prec, **kw):
        with B.GraphSet(graphs, **kw) as gs:
            ls, S = B.ensemble_scores(gs, m, prec)
            idx, _ = B.topk(S, 10)
            torch.cuda.synchronize()
            return float(ls.item()), S.cpu().numpy(), idx.cpu().numpy()

    def check(name, graphs, m, prec, **kw):
        th_g, S_g, idx = scores(graphs, m, prec, **kw)
        th_o, S_o = oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in graphs], m)
        e = parity.errors(th_g, S_g, th_o, S_o)
        tol = parity.TOL_FP64 if prec == B.CB_FP64 else parity.TOL_FP32
        ok = e["head_rel"] <= tol and e["norm_rel"] <= tol
        ref, _ = oc.topk(S_o, 10)
        out["cases"][name] = dict(ok=bool(ok), topk=bool(set(idx.tolist()) == set(ref.tolist())),
                                  violations=B.cb_debug_violations()[0], **e)

    ens = synth.er_ensemble([30_000, 50_001, 7_000], 10.0, 10, 4, config=901)
    n = 70_000
    rng = np.random.default_rng(5)
    extra = [(7, int(v)) for v in rng.choice(np.arange(8, n), 20_000, replace=False)]
    extra += [(40_000, int(v)) for v in rng.choice(np.arange(1, 39_000), 3000, replace=False)]
    hub = synth.er(n, 6.0 / (n - 1), 99, np.asarray(extra, dtype=np.uint32))
    check("blocked_fp32", ens.graphs, 20, B.CB_FP32, path=1)
    check("twophase_fp32", ens.graphs, 20, B.CB_FP32, two_phase=True)
    check("twophase_hub_fp32", [hub], 20, B.CB_FP32, two_phase=True)
    check("blocked_hub_fp32", [hub], 20, B.CB_FP32, path=1)
    check("csr_fp32", [hub], 20, B.CB_FP32, csr_only=True)
    check("csr_fp64", ens.graphs, 20, B.CB_FP64)

    nodes = [int(x) for x in ens.target]
    th_o, g_o = oa.ensemble_edge_grad([(g.n, g.row_ptr, g.col) for g in ens.graphs], nodes, 20)
    for name, kw in [("adjoint_blocked", dict(path=1)), ("adjoint_twophase", dict(two_phase=True))]:
        with B.GraphSet(ens.graphs, **kw) as gs:
            ls, g = B.scores_backward(gs, 20, nodes)
            torch.cuda.synchronize()
            a = g.cpu().numpy().astype(np.float64) * math.exp(float(ls.item()) - th_o)
        big = np.abs(g_o) >= 1e-3 * np.abs(g_o).max()
        rel = float(np.max(np.abs(a - g_o)[big] / np.abs(g_o)[big]))
        out["cases"][name] = dict(ok=rel <= 1e-3, rel=rel, violations=B.cb_debug_violations()[0])
    out["violations"], out["first"] = B.cb_debug_violations(reset=True)

    # A column index >= n, uploaded without validation on the tiled-CSR path
    # (the only path whose format build does not look at the columns; the
    # two-phase build rejects it, the column-blocked build is not given it).
    # Only this build is given the input: each gather through the bad entry
    # is counted and skipped.
    assert B.cb_debug_build() == 1
    nb = 1000
    rp = np.arange(0, 2 * nb + 1, 2, dtype=np.uint32)
    col = np.empty(2 * nb, np.uint32)
    col[0::2] = (np.arange(nb) + 1) % nb
    col[1::2] = (np.arange(nb) - 1) % nb
    col[10] = nb + 5

    class G:
        pass

    bad = G()
    bad.n, bad.row_ptr, bad.col = nb, rp, col
    planted = {}
    for name, prec in [("fp32", B.CB_FP32), ("fp64", B.CB_FP64)]:
        with B.GraphSet([bad], csr_only=True) as gs:
            ls, S = B.ensemble_scores(gs, 10, prec)
            torch.cuda.synchronize()
            finite = bool(np.all(np.isfinite(S.cpu().numpy())))
        c, f = B.cb_debug_violations(reset=True)
        planted[name] = dict(count=c, site=f >> 48, index=f & 0xffffffffffff, finite=finite)
    with B.GraphSet([bad], csr_only=True) as gs:
        B.scores_backward(gs, 10, [0, 1, 2, 3, 4])
        torch.cuda.synchronize()
    c, f = B.cb_debug_violations(reset=True)
    planted["adjoint"] = dict(count=c, site=f >> 48, index=f & 0xffffffffffff, finite=True)
    out["planted"] = planted
    print(json.dumps(out))


def test_debug_build_every_path_clean():
    env = dict(os.environ, CB_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", "import tests.test_gpu_debug as t; t._cases()"],
                       cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["debug_build"] == 1
    bad = {k: v for k, v in res["cases"].items() if not v["ok"] or not v.get("topk", True)}
    assert not bad, bad
    assert res["violations"] == 0, (res["violations"], hex(res["first"]), res["cases"])
    # the planted bad column: counted at the CSR gather (site 3) with its
    # index, the access skipped (finite scores), on every path that reads it
    for name, p in res["planted"].items():
        assert p["count"] >= 1 and p["finite"], (name, p)
        assert p["site"] == 3 and p["index"] == 1005, (name, p)

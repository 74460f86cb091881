"""Identification-rate sweep: the GPU run equals the oracle's run on the same
graphs (needs a GB300).

The sweep's rate is |top-k of eq. 5 intersect target| / k.  For small
columns the oracle computes the same quantity from the same graphs (the
device generators' CPU statements) in FP64; the
GPU path in FP64 mode must pick the same top-k set.
"""
import numpy as np
import pytest

import oracle.communicability as oc
from paper_1409_5000_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    binding.lib()
    return binding


def _oracle_rate(kind, n, param, N, target, seed, m):
    from paper_1409_5000_gb300 import sweep

    nodes = synth.sample_nodes(n, sweep.K, synth.seed_for(seed, 0, salt=11))
    tedges = synth.target_edges(nodes, sweep.SPARSE_EXTRA if target == "sparse" else 0,
                                target == "clique", synth.seed_for(seed, 0, salt=12))
    s1 = synth.seed_for(seed, 1)
    if kind == "er":
        graphs = [synth.er_generated(n, synth.er_draw_count(n, param), s1, r, tedges) for r in range(N)]
    elif kind == "ws":
        graphs = [synth.ws_generated(n, int(param), sweep.WS_REWIRE, s1, r, tedges) for r in range(N)]
    else:
        graphs = [synth.ba_generated(n, int(param), s1, r, tedges) for r in range(N)]
    th, S = oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in graphs], m)
    idx, _ = oc.topk(S, sweep.K)
    return len(set(np.asarray(idx).tolist()) & set(nodes.tolist())) / sweep.K


@pytest.mark.parametrize("col", [("er", 600, 2.0, 4, "sparse"), ("er", 1024, 39.0, 1, "clique"),
                                 ("ws", 500, 20, 2, "clique"), ("ba", 600, 5, 1, "clique")])
def test_sweep_run_matches_oracle(B, col):
    from paper_1409_5000_gb300 import sweep

    kind, n, param, N, target = col
    for q in range(3):
        seed = 880 + q
        gpu = sweep.run_once(B, kind, n, param, N, target, seed, 30, prec=B.CB_FP64)
        ref = _oracle_rate(kind, n, param, N, target, seed, 30)
        assert gpu == ref, (col, q, gpu, ref)


def test_sweep_easy_column_finds_everything(B):
    """A 20-clique in sparse ER backgrounds stands far above every background node."""
    from paper_1409_5000_gb300 import sweep

    res = sweep.sweep(4, 30, columns=[(0, "easy", "er", 2000, 3.0, 4, "clique", 100.0)])
    assert res[0]["rate_pct"] == 100.0

"""CB_REORTH: full reorthogonalisation on the GPU (needs a GB300).

With the flag, every new Lanczos vector is orthogonalised against all
previous ones by two classical Gram-Schmidt passes, the oracle's own scheme.
In FP64 both sides then run the same algorithm and differ only in summation
order and in the tridiagonal exponential (contour rule vs eigendecomposition),
so the scores agree far more tightly than the 1e-10 bar of the plain path.
Checks: the single-background graphs and a small ensemble in FP64 at 1e-12;
FP32 with the flag at 1e-4 on an uneven ensemble; the flag is part of the
captured-graph key; the adjoint and the restarted path with the flag.
"""
import math

import numpy as np
import pytest

import oracle.adjoint as oa
import oracle.communicability as oc
from paper_1409_5000_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIGHT = 1e-12


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    binding.lib()
    return binding


@pytest.mark.parametrize("kind", ["er", "ba", "ws"])
def test_fp64_single_background_tight(B, kind):
    g = synth.single_clique_100k(kind).graphs[0]
    th_o, y_o, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, 30)
    with B.GraphSet([g]) as gs:
        ls, y = B.communicability(gs, 0, 30, B.CB_FP64 | B.CB_REORTH)
        e = parity.errors(float(ls.item()), y.cpu().numpy(), th_o, y_o)
    assert e["head_rel"] <= TIGHT and e["norm_rel"] <= TIGHT, e


def test_fp64_ensemble_tight_and_deep(B):
    """eq. 5 over the small ensemble, and m = 60 where the plain recurrence
    has lost orthogonality long before."""
    ens = synth.er_ensemble_small()
    gs_o = [(g.n, g.row_ptr, g.col) for g in ens.graphs]
    for m in (20, 60):
        th_o, S_o = oc.ensemble_scores(gs_o, m)
        with B.GraphSet(ens.graphs) as gs:
            ls, S = B.ensemble_scores(gs, m, B.CB_FP64 | B.CB_REORTH)
            e = parity.errors(float(ls.item()), S.cpu().numpy(), th_o, S_o)
        assert e["head_rel"] <= TIGHT and e["norm_rel"] <= TIGHT, (m, e)


def test_fp32_uneven_ensemble(B):
    ens = synth.er_ensemble_uneven(n_inst=6, n_lo=3_000, n_hi=40_000, config=321)
    m = ens.meta["m"]
    th_o, S_o = oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in ens.graphs], m)
    with B.GraphSet(ens.graphs) as gs:
        ls, S = B.ensemble_scores(gs, m, B.CB_FP32 | B.CB_REORTH)
        idx, val = B.topk(S, 30)
        parity.assert_scores(float(ls.item()), S.cpu().numpy(), th_o, S_o, "fp32")
        parity.assert_topk(idx.cpu().numpy(), val.cpu().numpy(), S_o, 30, parity.TOL_FP32)


def test_flag_is_part_of_the_graph_key(B, monkeypatch):
    """Alternating calls with and without the flag on the same outputs each
    replay their own captured pass, bit-identical to direct launches."""
    ens = synth.er_ensemble_uneven(n_inst=4, n_lo=3_000, n_hi=20_000, config=322)
    with B.GraphSet(ens.graphs) as gs:
        monkeypatch.setenv("CB_NO_GRAPH", "1")
        ref = {f: B.ensemble_scores(gs, 20, B.CB_FP32 | f)[1].cpu().numpy() for f in (0, B.CB_REORTH)}
        monkeypatch.delenv("CB_NO_GRAPH")
        assert not np.array_equal(ref[0], ref[B.CB_REORTH])
        S = torch.empty(gs.n_max, dtype=torch.float64, device="cuda")
        ls = torch.empty(1, dtype=torch.float64, device="cuda")
        for _ in range(3):
            for f in (0, B.CB_REORTH):
                B.ensemble_scores(gs, 20, B.CB_FP32 | f, out=(S, ls))
                assert np.array_equal(S.cpu().numpy(), ref[f]), f


def test_adjoint_with_flag(B):
    ens = synth.er_ensemble_small()
    nodes = [int(x) for x in ens.target]
    gs_o = [(g.n, g.row_ptr, g.col) for g in ens.graphs]
    th_o, g_o = oa.ensemble_edge_grad(gs_o, nodes, 20)
    with B.GraphSet(ens.graphs) as gs:
        ls, g = B.scores_backward(gs, 20, nodes, B.CB_FP64 | B.CB_REORTH)
        a = g.cpu().numpy().astype(np.float64) * math.exp(float(ls.item()) - th_o)
    big = np.abs(g_o) >= 1e-3 * np.abs(g_o).max()
    assert np.max(np.abs(a - g_o)[big] / np.abs(g_o)[big]) <= 1e-6
    assert np.linalg.norm(a - g_o) / np.linalg.norm(g_o) <= 1e-6


def test_restarted_with_flag(B):
    ens = synth.er_ensemble([2_500, 9_000], 8.0, 12, 6, config=323)
    parts = [oc.krylov_expv_restarted(g.n, g.row_ptr, g.col, 6, 4) for g in ens.graphs]
    ts = max(p[0] for p in parts)
    S_o = np.zeros(max(g.n for g in ens.graphs))
    for g, (th, y, _) in zip(ens.graphs, parts):
        S_o[: g.n] += math.exp(th - ts) * y
    with B.GraphSet(ens.graphs) as gs:
        ls, S = B.ensemble_scores_restarted(gs, 6, 4, B.CB_FP64 | B.CB_REORTH)
        e = parity.errors(float(ls.item()), S.cpu().numpy(), ts, S_o)
    assert e["head_rel"] <= 1e-11 and e["norm_rel"] <= 1e-11, e

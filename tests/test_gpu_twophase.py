"""Two-phase (propagation-blocked) FP32 SpMV against the FP64 oracle (GB300).

The two-phase format runs by default for realisations above the
column-blocked size limit (n > 32 * 16384) and for every realisation with
CB_TWO_PHASE.  The cases span several source tiles (32768 nodes) with a
ragged last tile, many bins, rows heavier than the bin limit (summed in
chunks from the CSR), long rows (the whole CTA), uneven ensembles, the
degenerate graphs of the method, the adjoint and the captured-graph replay.
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


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    binding.lib()
    return binding


def _ens_gpu(B, graphs, m, prec=0, **kw):
    with B.GraphSet(graphs, **kw) as gs:
        ls, S, rep = B.ensemble_scores(gs, m, prec, report=True)
        torch.cuda.synchronize()
        return float(ls.item()), S.cpu().numpy(), rep


def _ens_oracle(graphs, m):
    return oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in graphs], m)


def _hub_graph():
    """ER(70000, d = 6) with a hub of degree 20000 (> the bin limit 8192,
    five chunks), one of 3000 (a long row) and one of 700 (a medium row)."""
    n = 70_000
    rng = np.random.default_rng(5)
    extra = [(7, int(v)) for v in rng.choice(np.arange(8, n), 20_000, replace=False)]
    extra += [(40_000, int(v)) for v in rng.choice(np.arange(1, 39_000), 3000, replace=False)]
    extra += [(69_999, int(v)) for v in rng.choice(np.arange(1000, 60_000), 700, replace=False)]
    return synth.er(n, 6.0 / (n - 1), 99, np.asarray(extra, dtype=np.uint32))


def test_forced_two_phase_single_ragged(B):
    """ER(100003, d = 10): four source tiles, the last of 1699 nodes; ~40 bins."""
    g = synth.er(100_003, 10.0 / 100_002, 3)
    th_o, S_o = _ens_oracle([g], 20)
    th_g, S_g, rep = _ens_gpu(B, [g], 20, two_phase=True)
    parity.assert_scores(th_g, S_g, th_o, S_o, "fp32")
    assert rep[0].m_eff == 20 and rep[0].status == 0


def test_forced_two_phase_heavy_long_medium_rows(B):
    g = _hub_graph()
    deg = np.diff(g.row_ptr.astype(np.int64))
    assert deg.max() > 8192 and np.sum((deg > 1024) & (deg <= 8192)) >= 1
    th_o, S_o = _ens_oracle([g], 25)
    th_g, S_g, _ = _ens_gpu(B, [g], 25, two_phase=True)
    parity.assert_scores(th_g, S_g, th_o, S_o, "fp32")
    # the same graph on the tiled-CSR kernel: the same recurrence, other
    # FP32 summation trees only
    th_c, S_c, _ = _ens_gpu(B, [g], 25, csr_only=True)
    e = parity.errors(th_g, S_g, th_c, S_c)
    assert e["head_rel"] <= 1e-5 and e["norm_rel"] <= 1e-5, e


def test_forced_two_phase_uneven_ensemble_and_topk(B):
    """Uneven realisations (one of a single tile, one smaller than a tile,
    one with isolated nodes only) sharing a 20-node target, eq. 5 and top-20."""
    sizes = [70_001, 33_000, 5_000, 100_000]
    ens = synth.er_ensemble(sizes, 12.0, 20, 10, config=811)
    iso = synth.from_edges(3000, np.zeros((0, 2), np.uint32))
    graphs = list(ens.graphs) + [iso]
    th_o, S_o = _ens_oracle(graphs, 20)
    with B.GraphSet(graphs, two_phase=True) as gs:
        ls, S = B.ensemble_scores(gs, 20, B.CB_FP32)
        idx, val = B.topk(S, 20)
        torch.cuda.synchronize()
        th_g, S_g = float(ls.item()), S.cpu().numpy()
        idx_g, val_g = idx.cpu().numpy(), val.cpu().numpy()
    parity.assert_scores(th_g, S_g, th_o, S_o, "fp32")
    parity.assert_topk(idx_g, val_g, S_o, 20, parity.TOL_FP32)


def test_default_path_above_blocked_limit(B):
    """ER(600000, d = 8) exceeds the column-blocked limit, so the default
    upload takes the two-phase format; checked against the oracle and the
    tiled-CSR kernel."""
    g = synth.er(600_000, 8.0 / 599_999, 17)
    th_o, S_o = _ens_oracle([g], 20)
    th_g, S_g, _ = _ens_gpu(B, [g], 20)
    parity.assert_scores(th_g, S_g, th_o, S_o, "fp32")
    th_c, S_c, _ = _ens_gpu(B, [g], 20, csr_only=True)
    e = parity.errors(th_g, S_g, th_c, S_c)
    assert e["head_rel"] <= 1e-5 and e["norm_rel"] <= 1e-5, e


def test_fp64_on_two_phase_handle_is_the_csr_path(B):
    """FP64 calls on a two-phase handle run the tiled-CSR kernel: bit-identical
    to a CSR-only handle, and within the FP64 bar of the oracle."""
    g = synth.er(40_000, 9.0 / 39_999, 23)
    th_a, S_a, _ = _ens_gpu(B, [g], 20, 1, two_phase=True)
    th_b, S_b, _ = _ens_gpu(B, [g], 20, 1, csr_only=True)
    assert th_a == th_b and np.array_equal(S_a, S_b)
    th_o, S_o = _ens_oracle([g], 20)
    parity.assert_scores(th_a, S_a, th_o, S_o, "fp64")


def test_deterministic_across_uploads_and_replays(B):
    """Slots inside a chunk are assigned by atomics, so two uploads may lay
    the stream out differently; the scores may not differ in any bit, on
    direct launches or on the captured graph's replays."""
    g = _hub_graph()
    outs = []
    for _ in range(2):
        with B.GraphSet([g], two_phase=True) as gs:
            S = torch.empty(gs.n_max, dtype=torch.float64, device="cuda")
            ls = torch.empty(1, dtype=torch.float64, device="cuda")
            for _ in range(3):  # direct, capture, replay
                B.ensemble_scores(gs, 20, B.CB_FP32, out=(S, ls))
                torch.cuda.synchronize()
                outs.append((float(ls.item()), S.cpu().numpy().copy()))
    for th, S in outs[1:]:
        assert th == outs[0][0] and np.array_equal(S, outs[0][1])


def test_degenerate_graphs(B):
    """Empty graph (e^A 1 = 1, breakdown at step 1), K_40 (e^{39} 1) and a
    single node, each forced onto the two-phase format."""
    empty = synth.from_edges(5000, np.zeros((0, 2), np.uint32))
    th, S, rep = _ens_gpu(B, [empty], 10, two_phase=True)
    assert rep[0].m_eff == 1 and np.allclose(S * math.exp(th), 1.0, rtol=1e-7, atol=0)
    kn = synth.from_edges(40, [(i, j) for i in range(40) for j in range(i + 1, 40)])
    th, S, rep = _ens_gpu(B, [kn], 10, two_phase=True)
    assert np.max(np.abs(S * math.exp(th - 39.0) - 1.0)) <= 2e-6
    one = synth.from_edges(1, np.zeros((0, 2), np.uint32))
    th, S, rep = _ens_gpu(B, [one], 10, two_phase=True)
    assert abs(S[0] * math.exp(th) - 1.0) < 1e-12


def test_invalid_column_rejected(B):
    """A column index >= n fails the two-phase build with CB_ERR_ARG (the
    count pass skips it, nothing reads past the tile)."""
    n = 1000
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.uint32)
    col = np.empty(2 * n, np.uint32)
    col[0::2] = (np.arange(n) + 1) % n
    col[1::2] = (np.arange(n) - 1) % n
    col[10] = n + 5

    class G:
        pass

    g = G()
    g.n, g.row_ptr, g.col = n, rp, col
    with pytest.raises(B.CBError) as ei:
        B.GraphSet([g], two_phase=True)
    assert ei.value.code == B.CB_ERR_ARG


def test_adjoint_on_two_phase_handle(B):
    """The adjoint's two Lanczos bases run on the two-phase kernels; the edge
    gradient matches the oracle's Krylov form within the gradient bar."""
    sizes = [40_000, 70_000]
    ens = synth.er_ensemble(sizes, 8.0, 10, 4, config=812)
    nodes = [int(x) for x in ens.target]
    with B.GraphSet(ens.graphs, two_phase=True) as gs:
        ls, g = B.scores_backward(gs, 20, nodes)
        torch.cuda.synchronize()
        th_g, g_g = float(ls.item()), g.cpu().numpy().astype(np.float64)
    th_o, g_o = oa.ensemble_edge_grad([(x.n, x.row_ptr, x.col) for x in ens.graphs], nodes, 20)
    a = g_g * math.exp(th_g - th_o)
    big = np.abs(g_o) >= 1e-3 * np.abs(g_o).max()
    assert np.max(np.abs(a - g_o)[big] / np.abs(g_o)[big]) <= 1e-3
    assert np.linalg.norm(a - g_o) <= 1e-3 * np.linalg.norm(g_o)

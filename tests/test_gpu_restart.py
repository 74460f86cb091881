"""CUDA restarted Lanczos (cb_ensemble_scores_restarted) vs the FP64 oracle
(needs a GB300).

The oracle evaluates the restarted approximation from its definition (the
block bidiagonal H_k with a dense exponential, krylov_expv_restarted); the
CUDA path evaluates exp(H_k) e1 block by block with the contour rule and
running products per contour node.  Checks: one cycle equals
cb_ensemble_scores; per-cycle parity on uneven ensembles (several
finalize and column-block tiles, ragged tails) in both precisions;
convergence to dense e^A 1; realisations that break down beside others that
run all cycles; the shift-raising path (a later cycle's lambda_max above
the first's); the report; argument errors; the forward basis and the
captured ensemble graphs stay correct around a restarted call.
"""
import math

import numpy as np
import pytest

import oracle.communicability as oc
from paper_1409_5000_gb300 import synth
from tests import parity, pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {0: "fp32", 1: "fp64"}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    binding.lib()
    return binding


def _oracle(graphs, m, cycles):
    """eq. 5 over restarted per-realisation results: (theta*, S, runs)."""
    parts = [oc.krylov_expv_restarted(g.n, g.row_ptr, g.col, m, cycles) for g in graphs]
    ts = max(p[0] for p in parts)
    S = np.zeros(max(g.n for g in graphs))
    for g, (th, y, _) in zip(graphs, parts):
        S[: g.n] += math.exp(th - ts) * y
    return ts, S, [p[2] for p in parts]


def _gpu(B, graphs, m, cycles, prec, report=False):
    with B.GraphSet(graphs) as gs:
        out = B.ensemble_scores_restarted(gs, m, cycles, prec, report=report)
    ls, S = float(out[0].item()), out[1].cpu().numpy()
    return (ls, S, out[2]) if report else (ls, S)


def _union(g1, g2):
    """Disjoint union, g2's nodes after g1's."""
    edges = []
    for g, off in ((g1, 0), (g2, g1.n)):
        for i in range(g.n):
            for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]]:
                if i < j:
                    edges.append((i + off, int(j) + off))
    return synth.from_edges(g1.n + g2.n, edges)


@pytest.mark.parametrize("prec", [0, 1])
def test_one_cycle_is_plain_ensemble(B, prec):
    ens = synth.er_ensemble_uneven(n_inst=4, n_lo=3_000, n_hi=30_000, config=401)
    with B.GraphSet(ens.graphs) as gs:
        l0, S0 = B.ensemble_scores(gs, 12, prec)
        l1, S1 = B.ensemble_scores_restarted(gs, 12, 1, prec)
        a, b = S0.cpu().numpy(), S1.cpu().numpy()
    assert float(l0.item()) == float(l1.item())
    tol = 1e-6 if prec == 0 else 1e-13  # FP32 mode rounds y_r to float in the plain combine
    assert np.max(np.abs(a - b) / np.abs(a)) <= tol


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("m,cycles", [(6, 2), (6, 5), (10, 3), (4, 8)])
def test_parity_uneven_ensemble(B, prec, m, cycles):
    ens = synth.er_ensemble([2_500, 19_001, 40_000, 700], 8.0, 12, 6, config=402)
    ts, S, runs = _oracle(ens.graphs, m, cycles)
    assert all(r == cycles for r in runs)
    lg, Sg = _gpu(B, ens.graphs, m, cycles, prec)
    parity.assert_scores(lg, Sg, ts, S, PREC[prec])


@pytest.mark.parametrize("prec", [0, 1])
def test_parity_ba_hubs(B, prec):
    g = synth.ba(30_000, 4, 403)
    ts, S, _ = _oracle([g], 8, 4)
    lg, Sg = _gpu(B, [g], 8, 4, prec)
    parity.assert_scores(lg, Sg, ts, S, PREC[prec])


def test_converges_to_dense(B):
    """Short cycles, many of them: every score equals dense e^A 1."""
    for g in (synth.er(300, 0.03, 404), synth.ba(400, 3, 11)):
        ref = oc.total_communicability_dense(g.n, g.row_ptr, g.col)
        errs = []
        for cycles in (1, 3, 8):
            lg, Sg = _gpu(B, [g], 5, cycles, 1)
            errs.append(parity.errors(lg, Sg, 0.0, ref)["max_rel"])
        assert errs[0] > 1e-4 and errs[1] < errs[0] and errs[2] <= 1e-11, errs


def test_breakdown_beside_running_realisations(B):
    """K_7 breaks down after one step (1 is an eigenvector) and K_{4,5} after
    two (its Krylov space from 1 has dimension 2), both in the first cycle,
    while an ER graph runs all cycles: the finished realisations keep their
    exact result through the later cycles."""
    graphs = [synth.from_edges(7, pins.complete(7)),
              synth.from_edges(9, pins.bipartite(4, 5)),
              synth.er(500, 0.02, 405)]
    lg, Sg, rep = _gpu(B, graphs, 4, 6, 1, report=True)
    ts, S, runs = _oracle(graphs, 4, 6)
    parity.assert_scores(lg, Sg, ts, S, "fp64")
    assert runs == [1, 1, 6]
    assert [r.m_eff for r in rep] == [1, 2, 24]
    # complete bipartite alone: exact closed form
    lg, Sg = _gpu(B, graphs[1:2], 4, 6, 1)
    parity.assert_scores_all(lg, Sg, 0.0, pins.bipartite_closed_form(4, 5), 1e-12)


@pytest.mark.parametrize("prec", [0, 1])
def test_shift_raised_by_later_cycle(B, prec):
    """A star K_{1,60} beside a sparse ER graph: the first cycle's top Ritz
    value misses the star's sqrt(60), a later cycle finds it, and the shift
    rises with the accumulated result rescaled."""
    g = _union(synth.er(3_000, 4 / 3_000, 9), synth.from_edges(61, pins.bipartite(1, 60)))
    ts, S, _ = _oracle([g], 4, 6)
    lg, Sg, rep = _gpu(B, [g], 4, 6, prec, report=True)
    # the oracle's theta is lambda_max(T_1) = 5.89; a later cycle's top Ritz
    # value is 7.69, below lambda_max(A) = sqrt(60) = 7.746
    assert ts + 1.5 < lg <= math.sqrt(60.0) + 1e-6 and rep[0].theta == lg
    parity.assert_scores(lg, Sg, ts, S, PREC[prec])


def test_report(B):
    ens = synth.er_ensemble([1_000, 3_000], 6.0, 8, 4, config=406)
    _, _, rep = _gpu(B, ens.graphs, 7, 3, 1, report=True)
    for g, r in zip(ens.graphs, rep):
        assert r.m_eff == 21 and r.status == 0 and r.beta_last > 0
        assert r.beta0 == math.sqrt(g.n)


def test_argument_errors(B):
    g = synth.er(100, 0.05, 407)
    with B.GraphSet([g]) as gs:
        for m, cycles in [(0, 2), (B.CB_MAX_M + 1, 2), (4, 0), (4, B.CB_MAX_CYCLES + 1)]:
            with pytest.raises(B.CBError):
                B.ensemble_scores_restarted(gs, m, cycles, 1)
        with pytest.raises(B.CBError):
            B.ensemble_scores_restarted(gs, 4, 2, 1, n_out=50)
        with pytest.raises(B.CBError):
            B.ensemble_scores_restarted(gs, 4, 2, 7)


def test_forward_basis_and_graphs_survive(B):
    """A restarted call overwrites the workspace: a later adjoint must
    recompute its forward basis, and replayed ensemble graphs must
    reinitialise it."""
    ens = synth.er_ensemble_uneven(n_inst=3, n_lo=4_000, n_hi=20_000, config=408)
    with B.GraphSet(ens.graphs) as gs:
        out = (torch.empty(gs.n_max, dtype=torch.float64, device="cuda"),
               torch.empty(1, dtype=torch.float64, device="cuda"))
        for _ in range(3):  # direct, captured, replayed
            B.ensemble_scores(gs, 10, 0, out=out)
        idx, _ = B.topk(out[0], 20)
        ref = (float(out[1].item()), out[0].cpu().numpy())
        g_ref = B.scores_backward(gs, 10, idx)[1].cpu().numpy()
        B.ensemble_scores(gs, 10, 0, out=out)
        B.ensemble_scores_restarted(gs, 10, 3, 0)
        g_after = B.scores_backward(gs, 10, idx)[1].cpu().numpy()
        B.ensemble_scores_restarted(gs, 10, 3, 0)
        B.ensemble_scores(gs, 10, 0, out=out)  # replay
        again = (float(out[1].item()), out[0].cpu().numpy())
    assert np.array_equal(g_ref, g_after)
    assert again[0] == ref[0] and np.array_equal(again[1], ref[1])

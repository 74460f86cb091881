"""Parity at the benchmark's full sizes, in the launch configuration
bench.py times (needs a GB300; a few minutes of host time for the oracle).

* 256 uneven ER realisations (n ~ U[2e4, 4e5], mean degree 20, 30-node
  target, m = 25, FP32 vectors): the third call with the same outputs
  replays the captured CUDA graph, as the timed steps do.  The FP64 oracle
  evaluates all 256 realisations in a spawn pool, so every score is checked
  (head and 2-norm within 1e-4) and the recovered top-30 must match.
* BA(n = 1e7, m = 8) + 20-clique, m = 40, FP32 (tiled-CSR kernel, hubs
  split across CTAs): every score against the oracle, and the top-20.
* The adjoint on 64 x ER(1e5, mean degree 16), m = 30, FP32, S = the
  recovered top-25: the gradients of sampled realisations (one at each end
  and one in the middle) against the oracle's Krylov form, within 1e-3.
"""
import math

import numpy as np
import pytest

import oracle.communicability as oc
from paper_1409_5000_gb300 import synth
from tests import fullsize_oracle as fo
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


def test_ensemble_256_every_score(B):
    sizes = synth.er_ensemble_uneven_sizes()
    ens = synth.er_ensemble_uneven()
    m, k = ens.meta["m"], ens.meta["k"]
    assert [g.n for g in ens.graphs] == sizes
    with B.GraphSet(ens.graphs) as gs:
        S = torch.empty(gs.n_max, dtype=torch.float64, device="cuda")
        ls = torch.empty(1, dtype=torch.float64, device="cuda")
        for _ in range(3):  # direct, captured, replayed
            S.fill_(float("nan"))
            B.ensemble_scores(gs, m, B.CB_FP32, out=(S, ls))
        idx, val = B.topk(S, k)
        torch.cuda.synchronize()
        S_g, th_g = S.cpu().numpy(), float(ls.item())
        idx_g, val_g = idx.cpu().numpy(), val.cpu().numpy()
    del ens
    parts = fo.pool_map(fo.ensemble_member_scores,
                        [(sizes, 20.0, k, 15, 3, r, m) for r in range(len(sizes))])
    th_o = max(p[1] for p in parts)
    S_o = np.zeros(max(sizes))
    for r, th, y in sorted(parts, key=lambda p: p[0]):
        S_o[: sizes[r]] += math.exp(th - th_o) * y
    parity.assert_scores(th_g, S_g, th_o, S_o, "fp32")
    parity.assert_topk(idx_g, val_g, S_o, k, parity.TOL_FP32)


def test_ba_1e7_every_score(B):
    ens = synth.ba_clique_large()
    g = ens.graphs[0]
    m, k = ens.meta["m"], ens.meta["k"]
    with B.GraphSet([g]) as gs:
        ls, y = B.communicability(gs, 0, m, B.CB_FP32)
        idx, val = B.topk(y, k)
        torch.cuda.synchronize()
        y_g, th_g = y.cpu().numpy(), float(ls.item())
        idx_g, val_g = idx.cpu().numpy(), val.cpu().numpy()
    th_o, y_o, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, m)
    parity.assert_scores(th_g, y_g, th_o, y_o, "fp32")
    parity.assert_topk(idx_g, val_g, y_o, k, parity.TOL_FP32)


def test_adjoint_64_sampled_realisations(B):
    ens = synth.er_ensemble_grad()
    m, k = ens.meta["m"], ens.meta["k"]
    n = ens.graphs[0].n
    sizes = [g.n for g in ens.graphs]
    with B.GraphSet(ens.graphs) as gs:
        _, S = B.ensemble_scores(gs, m, B.CB_FP32)
        idx, _ = B.topk(S, k)
        ls, grad = B.scores_backward(gs, m, idx, B.CB_FP32)
        torch.cuda.synchronize()
        g_all, th_g = grad.cpu().numpy().astype(np.float64), float(ls.item())
        nodes = [int(i) for i in idx.cpu().numpy()]
    base = np.concatenate([[0], np.cumsum([g.nnz for g in ens.graphs])])
    sample = [0, len(sizes) // 2, len(sizes) - 1]
    parts = fo.pool_map(fo.ensemble_member_grad,
                        [(sizes, 16.0, k, 10, 5, r, m, nodes) for r in sample])
    for r, th_o, g_o in parts:
        a = g_all[base[r]:base[r + 1]] * math.exp(th_g - th_o)
        big = np.abs(g_o) >= 1e-3 * np.abs(g_o).max()
        head = float(np.max(np.abs(a - g_o)[big] / np.abs(g_o)[big]))
        norm = float(np.linalg.norm(a - g_o) / np.linalg.norm(g_o))
        assert head <= 1e-3 and norm <= 1e-3, dict(r=r, head=head, norm=norm)
    assert n == 100_000


def test_adjoint_64_budgeted_groups_full_size(B):
    """The C5 shape under a device-memory budget of a quarter of its adjoint
    working set: cb_scores_backward_budget runs the 64 realisations in groups
    (about four) in temporary handles, recomputing each group's bases.  A
    group handle holds fewer blocked tiles than one per SM, so its automatic
    FP32 SpMV path is the tiled-CSR kernel where the whole handle's is the
    column-blocked one: the bases differ by FP32 rounding, so the gradient,
    brought to the same log scale, is compared at 1e-4 (relative to its
    largest entry and in the 2-norm), with the same zero pattern."""
    ens = synth.er_ensemble_grad()
    m, k = ens.meta["m"], ens.meta["k"]
    r4 = (m + 3) // 4 * 4
    ws = sum(4 * g.n * (2 * (m + 1) + 2 * r4) + 12 * g.nnz for g in ens.graphs)
    with B.GraphSet(ens.graphs) as gs:
        _, S = B.ensemble_scores(gs, m, B.CB_FP32)
        idx, _ = B.topk(S, k)
        ls0, g0 = B.scores_backward(gs, m, idx, B.CB_FP32)
        g = torch.empty_like(g0)
        ls = torch.empty(1, dtype=torch.float64, device="cuda")
        B.cb_scores_backward_budget(gs.h, m, B.CB_FP32, idx.data_ptr(), k, g.data_ptr(),
                                    ls.data_ptr(), ws // 4, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        shift = float(ls.item()) - float(ls0.item())
        assert abs(shift) <= 1e-6
        a = g.cpu().numpy().astype(np.float64) * math.exp(shift)
        b = g0.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(b))
    assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b)
    assert np.array_equal(a == 0, b == 0)


"""CUDA adjoint (cb_scores_backward) vs the FP64 adjoint oracle (needs a GB300).

The loss is the summed score of a fixed node set S over the realisations
(eq. 5 restricted to S); the gradient is taken with respect to the
undirected weight of every existing edge.  Checks: the Krylov-form oracle at
the same m; the dense Frechet derivative where m spans the Krylov spaces;
central finite differences of the oracle's m-step loss on random edges; the
scalar identity sum_e g_e = 2 w^T A e^A 1; degenerate cases; the autograd
wrapper.
"""
import math

import numpy as np
import pytest

import oracle.adjoint as oa
import oracle.communicability as oc
from paper_1409_5000_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3  # FP32 mode, relative (head + normwise)
# FP64 mode: the contour rule's error for divided differences of exp (the
# derivative of its ~2e-14 error for exp itself) leaves ~6e-8 relative.
TOL_GRAD64 = 1e-6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    binding.lib()
    return binding


def _gpu_grad(B, graphs, nodes, m, prec):
    with B.GraphSet(graphs) as gs:
        ls, g = B.scores_backward(gs, m, nodes, prec)
        torch.cuda.synchronize()
        return float(ls.item()), g.cpu().numpy().astype(np.float64)


def _compare(th_g, g, th_o, g_o, tol):
    a = g * math.exp(th_g - th_o)
    b = g_o
    big = np.abs(b) >= 1e-3 * np.abs(b).max()
    head = float(np.max(np.abs(a - b)[big] / np.abs(b)[big]))
    norm = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert head <= tol and norm <= tol, dict(head=head, norm=norm)
    return head, norm


@pytest.mark.parametrize("prec", [0, 1])
def test_small_ensemble_vs_krylov_oracle(B, prec):
    """10 x ER(500) + 15-node target, m = 20, S = the target nodes."""
    ens = synth.er_ensemble_small()
    nodes = [int(x) for x in ens.target]
    th_o, g_o = oa.ensemble_edge_grad([(g.n, g.row_ptr, g.col) for g in ens.graphs], nodes, 20)
    th_g, g = _gpu_grad(B, ens.graphs, nodes, 20, prec)
    _compare(th_g, g, th_o, g_o, TOL_GRAD if prec == 0 else TOL_GRAD64)


@pytest.mark.parametrize("prec", [0, 1])
def test_dense_frechet(B, prec):
    """n = 60, m = 60 spans the Krylov spaces: the Krylov gradient is the
    dense Frechet derivative (block-exponential oracle)."""
    g = synth.er(60, 0.1, 77)
    nodes = [3, 10, 11, 42, 59]
    w = np.zeros(60)
    w[nodes] = 1.0
    ref = oa.dense_edge_grad(g.n, g.row_ptr, g.col, w, how="block")
    th_g, gg = _gpu_grad(B, [g], nodes, 60, prec)
    _compare(th_g, gg, 0.0, ref, TOL_GRAD if prec == 0 else TOL_GRAD64)


def test_finite_differences(B):
    """4 x ER(2e4, dbar 16) + 25-node target (tree + 10), m = 30: central
    differences (h = 1e-3) of the oracle's m-step loss on 200 random edges."""
    ens = synth.er_ensemble([20_000] * 4, 16.0, 25, 10, config=505)
    nodes = [int(x) for x in ens.target]
    th_g, g = _gpu_grad(B, ens.graphs, nodes, 30, 0)
    rng = np.random.default_rng(7)
    offs = np.cumsum([0] + [x.nnz for x in ens.graphs])
    errs = []
    gmax = 0.0
    picks = []
    for _ in range(200):
        r = int(rng.integers(0, 4))
        e = int(rng.integers(0, ens.graphs[r].nnz))
        picks.append((r, e))
    # bias half of the sample towards edges at the target, where gradients are large
    for q in range(0, 100):
        r = q % 4
        gr = ens.graphs[r]
        t = nodes[q % len(nodes)]
        lo, hi = int(gr.row_ptr[t]), int(gr.row_ptr[t + 1])
        if hi > lo:
            picks[q] = (r, lo + int(rng.integers(0, hi - lo)))
    for r, e in picks:
        gr = ens.graphs[r]
        (th_fd, fd), = oa.fd_edge_grad(gr.n, gr.row_ptr, gr.col, nodes, 30, [e], h=1e-3)
        gpu = g[offs[r] + e] * math.exp(th_g - th_fd)
        errs.append((abs(gpu - fd), abs(fd)))
        gmax = max(gmax, abs(fd))
    for d, ref in errs:
        assert d <= TOL_GRAD * max(ref, 1e-3 * gmax), (d, ref)


def test_scalar_identity(B):
    """sum_e g_e = 2 w^T A e^A 1 (each undirected edge appears twice)."""
    g = synth.er(3000, 8.0 / 3000, 12)
    nodes = [5, 17, 900, 2999]
    w = np.zeros(g.n)
    w[nodes] = 1.0
    th_g, gg = _gpu_grad(B, [g], nodes, 60, 1)
    A = oc.csr_matrix(g.n, g.row_ptr, g.col)
    th, y, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, 60)
    lhs = np.sum(gg) * math.exp(th_g - th)
    rhs = 2.0 * w @ (A @ y)
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs), (lhs, rhs)


def test_realisation_without_target_nodes(B):
    """Uneven n: nodes beyond a realisation's range contribute nothing."""
    g1 = synth.er(500, 0.02, 1)
    g2 = synth.er(3000, 0.004, 2)
    nodes = [1000, 2500]  # only inside g2
    th_g, g = _gpu_grad(B, [g1, g2], nodes, 20, 0)
    assert np.all(g[: g1.nnz] == 0.0)
    assert np.any(g[g1.nnz:] != 0.0)
    w = np.zeros(g2.n)
    w[nodes] = 1.0
    th_o, g_o = oa.krylov_edge_grad(g2.n, g2.row_ptr, g2.col, w, 20)
    _compare(th_g, g[g1.nnz:], th_o, g_o, TOL_GRAD)


def test_autograd_function(B):
    ens = synth.er_ensemble_small()
    nodes = [int(x) for x in ens.target]
    with B.GraphSet(ens.graphs) as gs:
        wgt = torch.ones(sum(gs.nnz), dtype=torch.float32, device="cuda", requires_grad=True)
        loss = B.summed_topk_score(wgt, gs, 20, nodes)
        loss.backward()
        ls_f, S = B.ensemble_scores(gs, 20, B.CB_FP32)
        ls_b, g = B.scores_backward(gs, 20, nodes)
        expect = g * torch.exp(ls_b - ls_f).float()
        assert torch.allclose(wgt.grad, expect, rtol=1e-6, atol=0)
        assert abs(loss.item() - S[torch.as_tensor(nodes, device="cuda")].sum().item()) <= 1e-12 * abs(loss.item())
        # an upstream factor scales the gradient (vector-Jacobian product)
        wgt.grad = None
        loss = B.summed_topk_score(wgt, gs, 20, nodes)
        (3.0 * loss).backward()
        assert torch.allclose(wgt.grad, 3.0 * expect, rtol=1e-6, atol=0)


def test_autograd_rejects_non_unit_weights(B):
    """The store is pattern-only: weights other than one would silently give
    unit-weight results, so they are refused."""
    ens = synth.er_ensemble_small()
    nodes = [int(x) for x in ens.target]
    with B.GraphSet(ens.graphs) as gs:
        wgt = torch.ones(sum(gs.nnz), dtype=torch.float32, device="cuda", requires_grad=True)
        with torch.no_grad():
            wgt[7] = 1.5
        with pytest.raises(ValueError, match="all ones"):
            B.summed_topk_score(wgt, gs, 20, nodes)
        with pytest.raises(ValueError, match="one entry per CSR entry"):
            B.summed_topk_score(wgt[:-1], gs, 20, nodes)


def test_score_sum_and_grad_rescale(B):
    """cb_score_sum against a host sum over the node set (entries >= n
    skipped); cb_grad_rescale against exp(ls_g - ls_r) * grad_out."""
    S = torch.rand(1000, dtype=torch.float64, device="cuda")
    nodes = torch.tensor([5, 999, 1000, 3, 5, 4000], dtype=torch.int32, device="cuda")
    out = torch.empty((), dtype=torch.float64, device="cuda")
    B.cb_score_sum(S.data_ptr(), 1000, nodes.data_ptr(), 6, out.data_ptr(),
                   torch.cuda.current_stream().cuda_stream)
    Sh = S.cpu().numpy()
    ref = Sh[5] + Sh[999] + Sh[3] + Sh[5]
    assert abs(out.item() - ref) <= 1e-15 * ref
    g = torch.randn(100_003, dtype=torch.float32, device="cuda")
    g0 = g.clone()
    lg = torch.tensor([3.25], dtype=torch.float64, device="cuda")
    lr = torch.tensor([2.0], dtype=torch.float64, device="cuda")
    go = torch.tensor([-0.5], dtype=torch.float64, device="cuda")
    B.cb_grad_rescale(g.data_ptr(), g.numel(), lg.data_ptr(), lr.data_ptr(), go.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    f = math.exp(1.25) * -0.5
    g1 = g.cpu().numpy()
    assert np.allclose(g1, g0.cpu().numpy().astype(np.float64) * f, rtol=3e-7, atol=0)
    B.cb_grad_rescale(g.data_ptr(), g.numel(), lg.data_ptr(), lg.data_ptr(), 0,
                      torch.cuda.current_stream().cuda_stream)  # factor exactly 1
    assert np.array_equal(g.cpu().numpy(), g1)


def test_forward_basis_reuse(B):
    """After an ensemble pass at the same m and precision the adjoint reuses
    its basis from 1; the gradient must be bit-identical to a recomputation
    (the first backward on a fresh handle computes the basis itself), also
    when a per-realisation call or another depth came in between."""
    ens = synth.er_ensemble_small()
    nodes = [int(x) for x in ens.target]
    with B.GraphSet(ens.graphs) as gs:
        ls0, g0 = B.scores_backward(gs, 20, nodes)
        g0 = g0.cpu().numpy()
        for between in (None, "single", "depth"):
            B.ensemble_scores(gs, 20, 0)
            if between == "single":
                B.communicability(gs, 3, 20)
            elif between == "depth":
                B.ensemble_scores(gs, 12, 0)
            ls, g = B.scores_backward(gs, 20, nodes)
            assert float(ls.item()) == float(ls0.item()), between
            assert np.array_equal(g.cpu().numpy(), g0), between


@pytest.mark.parametrize("budget", [1, 40 << 20])
def test_memory_budget_groups(B, budget):
    """A budget below the working set runs the adjoint over groups of
    realisations (one per group at budget 1) in temporary handles; the result
    is the unbudgeted gradient up to the FP32 rounding of the rescaling."""
    ens = synth.er_ensemble([20_000, 60_000, 5_000, 40_000, 30_000], 12.0, 20, 8, config=506)
    nodes = torch.as_tensor(np.asarray(ens.target, dtype=np.int32), device="cuda")
    with B.GraphSet(ens.graphs) as gs:
        ls0, g0 = B.scores_backward(gs, 25, [int(x) for x in ens.target])
        g = torch.empty_like(g0)
        ls = torch.empty(1, dtype=torch.float64, device="cuda")
        B.cb_scores_backward_budget(gs.h, 25, 0, nodes.data_ptr(), nodes.numel(), g.data_ptr(),
                                    ls.data_ptr(), budget, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert float(ls.item()) == float(ls0.item())
        a, b = g.cpu().numpy().astype(np.float64), g0.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))
        assert np.array_equal(a == 0, b == 0)


def test_backward_argument_errors(B):
    g = synth.er(100, 0.05, 1)
    with B.GraphSet([g]) as gs:
        with pytest.raises(B.CBError):
            B.scores_backward(gs, 65, [1, 2])  # beyond the adjoint depth limit
        with pytest.raises(B.CBError):
            B.scores_backward(gs, 0, [1])

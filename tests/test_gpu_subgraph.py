"""CUDA sub-graph centrality (cb_subgraph_centrality, eq. 3) vs the FP64 oracle
(needs a GB300).

Checks: closed forms (K_n, star, cycle, isolated node); the dense diagonal of
e^A where m spans the Krylov space from e_i; the oracle's Gauss rule at the
same m on larger graphs, nodes given on the host or on the device; the
lower-bound property across m; argument errors.
"""
import math

import numpy as np
import pytest

import oracle.communicability as oc
from paper_1409_5000_gb300 import synth
from tests import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    binding.lib()
    return binding


def _sc(B, graphs, inst, m, nodes, prec):
    with B.GraphSet(graphs) as gs:
        ls, sc = B.subgraph_centrality(gs, inst, m, nodes, prec)
        return np.exp(float(ls.item())) * sc.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("prec", [0, 1])
def test_closed_forms(B, prec):
    s6 = math.sqrt(6.0)
    cases = [
        (synth.from_edges(7, pins.complete(7)), np.full(7, (math.exp(6) + 6 * math.exp(-1)) / 7)),
        (synth.from_edges(7, pins.bipartite(1, 6)),
         np.concatenate([[math.cosh(s6)], np.full(6, 1 + (math.cosh(s6) - 1) / 6)])),
        (synth.from_edges(9, pins.cycle(9)),
         np.full(9, sum(math.exp(2 * math.cos(2 * math.pi * j / 9)) for j in range(9)) / 9)),
    ]
    for g, ref in cases:
        got = _sc(B, [g], 0, g.n, list(range(g.n)), prec)
        assert _rel(got, ref) <= TOL[prec]


def test_isolated_node(B):
    g = synth.from_edges(5, [(0, 1), (1, 2)])  # nodes 3, 4 isolated
    got = _sc(B, [g], 0, 10, [3, 4, 1], 1)
    assert abs(got[0] - 1.0) <= 1e-14 and abs(got[1] - 1.0) <= 1e-14  # e^0
    ref = oc.subgraph_centrality_dense(g.n, g.row_ptr, g.col)[1]
    assert abs(got[2] - ref) <= 1e-12 * ref


@pytest.mark.parametrize("prec", [0, 1])
def test_dense_diagonal(B, prec):
    """n = 70, m = 70: the Gauss rule is exact; all nodes, second realisation."""
    g0 = synth.er(40, 0.1, 3)
    g = synth.er(70, 0.08, 4)
    ref = oc.subgraph_centrality_dense(g.n, g.row_ptr, g.col)
    got = _sc(B, [g0, g], 1, 70, list(range(70)), prec)
    assert _rel(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("where", ["host", "device"])
def test_gauss_rule_vs_oracle(B, prec, where):
    """ER(2e4, d 12), m = 15, 48 nodes: same Gauss rule as the oracle."""
    g = synth.er(20_000, 12.0 / 20_000, 8)
    nodes = synth.sample_nodes(g.n, 48, 9).astype(np.int64)
    th, c0 = oc.subgraph_centrality_krylov(g.n, g.row_ptr, g.col, nodes, 15)
    ref = np.exp(th) * c0
    with B.GraphSet([g]) as gs:
        if where == "host":
            ls, sc = B.subgraph_centrality(gs, 0, 15, nodes, prec)
        else:
            d = torch.as_tensor(nodes.astype(np.int32), device="cuda")
            sc = torch.empty(48, dtype=torch.float64, device="cuda")
            ls = torch.empty(1, dtype=torch.float64, device="cuda")
            B.cb_subgraph_centrality(gs.h, 0, 15, prec, 48, d.data_ptr(), sc.data_ptr(),
                                     ls.data_ptr(), torch.cuda.current_stream().cuda_stream)
        theta = float(ls.item())
        got = np.exp(theta) * sc.cpu().numpy()
    if prec == 0:
        assert _rel(got, ref) <= TOL[0]
    else:
        # FP64: the quadrature is exp(theta) * c0 with c0 = [exp(T - theta) e1]_0 <= 1;
        # the contour rule and the recurrence are accurate relative to
        # ||exp(T - theta)|| = 1, so nodes with SC << exp(theta) carry errors
        # measured in units of exp(theta), not of SC itself
        assert float(np.max(np.abs(got - ref))) <= 1e-12 * math.exp(theta)
        assert _rel(got, ref) <= 1e-9


def test_lower_bound_increasing_in_m(B):
    g = synth.er(300, 0.04, 12)
    nodes = [0, 5, 77, 299]
    dense = oc.subgraph_centrality_dense(g.n, g.row_ptr, g.col)[nodes]
    prev = np.zeros(4)
    for m in (1, 2, 4, 8, 16):
        est = _sc(B, [g], 0, m, nodes, 1)
        assert np.all(est >= prev * (1 - 1e-12)) and np.all(est <= dense * (1 + 1e-10)), m
        prev = est


def test_argument_errors(B):
    g = synth.er(100, 0.05, 1)
    with B.GraphSet([g]) as gs:
        with pytest.raises(B.CBError):
            B.subgraph_centrality(gs, 0, 10, [100])  # node out of range
        with pytest.raises(B.CBError):
            B.subgraph_centrality(gs, 1, 10, [1])  # realisation out of range
        with pytest.raises(B.CBError):
            B.subgraph_centrality(gs, 0, 0, [1])  # m = 0

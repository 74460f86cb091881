"""On-device ER generation (cb_graph_generate_er) vs its CPU statement (needs a GB300).

The device generator and synth.er_generated implement the same counter-based
definition independently (CUDA vs numpy); the CSR patterns must agree bit for
bit, and the scores of a generated handle must equal those of the same graphs
uploaded from the host.
"""
import numpy as np
import pytest

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


def _cpu(n, dbar, seed, tedges):
    return [synth.er_generated(x, synth.er_draw_count(x, dbar), seed, r, tedges)
            for r, x in enumerate(n)]


@pytest.mark.parametrize("case", ["small", "uneven", "no_target", "dense", "very_dense", "huge_rows",
                                  "tiny"])
def test_generated_csr_matches_cpu_definition(B, case):
    if case == "small":
        n, dbar, tedges = [500] * 10, 3.2, synth.target_edges(np.arange(15, dtype=np.uint32) * 7, 8, False, 3)
    elif case == "uneven":
        n, dbar, tedges = [20_000, 3_000, 150_000, 777], 20.0, [(0, 1), (1, 2), (2, 0), (5, 900), (10, 2999)]
    elif case == "no_target":
        n, dbar, tedges = [100_000, 100_000], 16.0, None
    elif case == "dense":  # many repeated pairs collapse; rows of 33-64 raw entries
        n, dbar, tedges = [64, 64, 64], 40.0, [(1, 2)]
    elif case == "very_dense":  # rows of > 64 raw entries: sorted by a CTA in shared memory
        n, dbar, tedges = [64, 96], 200.0, [(1, 2)]
    elif case == "huge_rows":  # rows of > 32768 raw entries keep the serial sort (one repeated pair)
        n, dbar, tedges = [2], 33_500.0, None
    else:  # one-node realisations (every draw a self-loop, the target edge out of range),
        # realisations shorter than a warp's 32 rows, several per chunk of draws
        n, dbar, tedges = [1, 37, 2, 1000, 1, 64], 3.0, [(0, 1), (3, 36)]
    seed = synth.seed_for(901, 0)
    ref = _cpu(n, dbar, seed, tedges)
    gs = B.GraphSet.generate_er(n, dbar, seed, tedges)
    try:
        assert gs.nnz == [g.nnz for g in ref]
        for r, g in enumerate(ref):
            rp, col = B.read_graph(gs, r)
            assert np.array_equal(rp, g.row_ptr), r
            assert np.array_equal(col, g.col), r
    finally:
        gs.close()


def test_generated_scores_equal_uploaded(B):
    """Same graphs through both entry points give bit-identical scores."""
    n = [30_000, 60_000, 45_000, 30_000]
    nodes = synth.sample_nodes(30_000, 20, 5)
    tedges = synth.target_edges(nodes, 10, False, 6)
    seed = synth.seed_for(902, 0)
    ref = _cpu(n, 12.0, seed, tedges)
    with B.GraphSet(ref) as up, B.GraphSet.generate_er(n, 12.0, seed, tedges) as gen:
        for prec in (0, 1):
            a = B.ensemble_scores(up, 20, prec)
            b = B.ensemble_scores(gen, 20, prec)
            assert float(a[0].item()) == float(b[0].item())
            assert torch.equal(a[1], b[1])


def test_generate_argument_errors(B):
    with pytest.raises(B.CBError):
        B.cb_graph_generate_er([100, 0], [10, 10], 1, None, 0)  # n = 0
    with pytest.raises(B.CBError):
        B.cb_graph_generate_er([100], [2**31], 1, None, 0)  # too many draws
    with pytest.raises(B.CBError):
        B.cb_graph_generate_er([100], [10], 1, [(1, 2**31)], 0)  # endpoint range


def test_read_argument_errors(B):
    gs = B.GraphSet.generate_er([50], 4.0, 1)
    try:
        rp = np.empty(51, np.uint32)
        with pytest.raises(B.CBError):
            B.cb_graph_read(gs.h, 1, rp.ctypes.data, rp.ctypes.data, 0)
    finally:
        gs.close()


def _check_same(B, gs, ref):
    assert gs.nnz == [g.nnz for g in ref]
    for r, g in enumerate(ref):
        rp, col = B.read_graph(gs, r)
        assert np.array_equal(rp, g.row_ptr), r
        assert np.array_equal(col, g.col), r


@pytest.mark.parametrize("n,k,p,tedges", [
    ([500] * 6, 10, 0.1, [(0, 250), (3, 4), (100, 400)]),
    ([20_000, 3_000, 100_000], 40, 0.1, None),       # Table 2 shape, uneven n
    ([1_000, 1_000], 6, 0.0, [(1, 500)]),            # the plain ring lattice
    ([2_000], 8, 1.0, None),                         # every edge rewired
])
def test_ws_matches_cpu_definition(B, n, k, p, tedges):
    seed = synth.seed_for(903, 0)
    ref = [synth.ws_generated(x, k, p, seed, r, tedges) for r, x in enumerate(n)]
    gs = B.GraphSet.generate_ws(n, k, p, seed, tedges)
    try:
        _check_same(B, gs, ref)
    finally:
        gs.close()


@pytest.mark.parametrize("n,m,tedges", [
    ([500] * 6, 3, [(0, 250), (3, 4)]),
    ([50_000, 7_000, 120_000], 10, None),            # Table 3 shape (hubs: long rows)
    ([3_000], 1, [(5, 6)]),                          # a tree plus the target edge
    ([64, 200], 20, None),                           # dense: many repeated picks
    ([300_000], 10, None),                           # hub rows of > 1024 raw entries
])
def test_ba_matches_cpu_definition(B, n, m, tedges):
    seed = synth.seed_for(904, 0)
    ref = [synth.ba_generated(x, m, seed, r, tedges) for r, x in enumerate(n)]
    gs = B.GraphSet.generate_ba(n, m, seed, tedges)
    try:
        _check_same(B, gs, ref)
    finally:
        gs.close()


def test_ws_ba_scores_equal_uploaded(B):
    seed = synth.seed_for(905, 0)
    for make, cpu in ((lambda: B.GraphSet.generate_ws([30_000, 20_000], 10, 0.2, seed),
                       [synth.ws_generated(x, 10, 0.2, seed, r) for r, x in enumerate([30_000, 20_000])]),
                      (lambda: B.GraphSet.generate_ba([30_000, 20_000], 5, seed),
                       [synth.ba_generated(x, 5, seed, r) for r, x in enumerate([30_000, 20_000])])):
        with B.GraphSet(cpu) as up, make() as gen:
            a = B.ensemble_scores(up, 20, 0)
            b = B.ensemble_scores(gen, 20, 0)
            assert float(a[0].item()) == float(b[0].item()) and torch.equal(a[1], b[1])


def test_ws_ba_argument_errors(B):
    for args in ([100], 3, 0.1), ([100], 0, 0.1), ([100], 100, 0.1), ([100], 4, 1.5), ([100], 4, -0.1):
        with pytest.raises(B.CBError):
            B.cb_graph_generate_ws(*args, 1, None, 0)
    for args in ([100], 0), ([10], 10), ([100, 0], 2):
        with pytest.raises(B.CBError):
            B.cb_graph_generate_ba(*args, 1, None, 0)

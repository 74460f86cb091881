"""Tiled-CSR group widths: parity at every width, the tuner, the cache (needs a GB300)."""
import numpy as np
import pytest

import oracle.communicability as oc
from paper_1409_5000_gb300 import synth, tune
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


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_every_width_matches_oracle(B, lanes):
    """FP64 (always the tiled-CSR kernel) on a heavy-tailed graph and an ER graph."""
    graphs = [synth.ba(30_000, 6, 31), synth.er(20_000, 10.0 / 20_000, 32)]
    th_o, S_o = oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in graphs], 20)
    with B.GraphSet(graphs) as gs:
        B.cb_graph_set_lanes(gs.h, lanes)
        assert B.cb_graph_lanes(gs.h) == lanes
        ls, S = B.ensemble_scores(gs, 20, B.CB_FP64)
        parity.assert_scores(float(ls.item()), S.cpu().numpy(), th_o, S_o, "fp64")


def test_tuner_keeps_fastest(B):
    graphs = [synth.ba(200_000, 8, 41)]
    with B.GraphSet(graphs) as gs:
        lanes, ms = B.cb_graph_tune(gs.h, B.CB_FP64, 0)
        assert lanes in (1, 2, 4, 8, 16, 32) and B.cb_graph_lanes(gs.h) == lanes
        timed = [x for x in ms if x >= 0]
        assert len(timed) == 6 and ms[6] == -1.0 and ms[7] == -1.0  # FP64: the width only
        assert ms[[1, 2, 4, 8, 16, 32].index(lanes)] == min(timed)


def test_tuner_fp32_picks_width_and_path(B):
    """FP32 on a handle with the column-blocked format: the six widths on the
    tiled-CSR path and the format path are all timed, and the fastest is kept."""
    with B.GraphSet([synth.er(60_000, 10.0 / 60_000, 5)]) as gs:
        lanes, ms = B.cb_graph_tune(gs.h, B.CB_FP32, 0)
        assert len(ms) == 8 and all(x >= 0 for x in ms[:7]) and ms[7] == -1.0
        path = B.cb_graph_path(gs.h)
        kept = 6 if path == B.CB_PATH_FORMATS else [1, 2, 4, 8, 16, 32].index(lanes)
        assert path in (B.CB_PATH_FORMATS, B.CB_PATH_CSR)
        assert ms[kept] == min(ms[:7])


@pytest.mark.parametrize("prec", [0, 1])
def test_tuner_times_the_single_launch_of_small_handles(B, prec):
    """A handle whose realisations all fit the single-launch path: the tuner
    also times it (slot 7) and keeps it when fastest; scores then meet the
    oracle bar whatever was kept."""
    graphs = [synth.er(n, 8.0 / n, 70 + q) for q, n in enumerate([500, 2000, 800] * 20)]
    with B.GraphSet(graphs) as gs:
        lanes, ms = B.cb_graph_tune(gs.h, prec, 0)
        assert ms[7] >= 0
        path = B.cb_graph_path(gs.h)
        if path == B.CB_PATH_AUTO:
            assert ms[7] == min(x for x in ms if x >= 0)
        ls, S = B.ensemble_scores(gs, 20, prec)
        torch.cuda.synchronize()
        th_o, S_o = oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in graphs], 20)
        parity.assert_scores(float(ls.item()), S.cpu().numpy(), th_o, S_o, "fp64" if prec else "fp32")


@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("two_phase", [False, True])
def test_every_path_matches_oracle(B, path, two_phase):
    """Every FP32 path (automatic, formats, tiled CSR) on the column-blocked
    and on the two-phase format, against the oracle."""
    graphs = [synth.ba(40_000, 6, 61), synth.er(25_000, 12.0 / 25_000, 62)]
    th_o, S_o = oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in graphs], 20)
    with B.GraphSet(graphs, two_phase=two_phase) as gs:
        B.cb_graph_set_path(gs.h, path)
        assert B.cb_graph_path(gs.h) == path
        ls, S = B.ensemble_scores(gs, 20, B.CB_FP32)
        parity.assert_scores(float(ls.item()), S.cpu().numpy(), th_o, S_o, "fp32")


def test_path_errors(B):
    with B.GraphSet([synth.er(100, 0.05, 1)]) as gs:
        with pytest.raises(B.CBError):
            B.cb_graph_set_path(gs.h, 3)


def test_autotune_cache(B, tmp_path):
    path = str(tmp_path / "tune.json")
    graphs = [synth.er(50_000, 12.0 / 50_000, 51)]
    with B.GraphSet(graphs) as gs:
        lanes, cached = tune.autotune(gs, B.CB_FP64, graphs, path)
        assert not cached and lanes == B.cb_graph_lanes(gs.h)
    with B.GraphSet(graphs) as gs:
        B.cb_graph_set_lanes(gs.h, 1 if lanes != 1 else 2)
        lanes2, cached = tune.autotune(gs, B.CB_FP64, graphs, path)
        assert cached and lanes2 == lanes == B.cb_graph_lanes(gs.h)


def test_set_lanes_errors(B):
    with B.GraphSet([synth.er(100, 0.05, 1)]) as gs:
        with pytest.raises(B.CBError):
            B.cb_graph_set_lanes(gs.h, 3)

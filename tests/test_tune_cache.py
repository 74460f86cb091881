"""Shape keys and the JSON cache of tiled-CSR group widths (host logic, CPU)."""
import json

import numpy as np

from paper_1409_5000_gb300 import synth, tune


def test_degree_cv_matches_numpy():
    gs = [synth.er(500, 0.02, 1), synth.ba(800, 3, 2)]
    d = np.concatenate([g.degrees() for g in gs]).astype(np.float64)
    assert abs(tune.degree_cv(gs) - d.std() / d.mean()) < 1e-12
    assert tune.degree_cv([synth.from_edges(4, [])]) == 0.0


def test_shape_key_buckets():
    k1 = tune.shape_key([100_000] * 64, [1_600_000] * 64, 0, 0.25)
    k2 = tune.shape_key([101_000] * 64, [1_610_000] * 64, 0, 0.25)
    assert k1 == k2  # same bucket
    assert k1 != tune.shape_key([100_000] * 64, [1_600_000] * 64, 1, 0.25)  # precision
    assert k1 != tune.shape_key([100_000] * 64, [6_400_000] * 64, 0, 0.25)  # mean degree
    assert k1 != tune.shape_key([100_000] * 64, [1_600_000] * 64, 0, 2.5)  # degree spread
    assert tune.shape_key([10], [0], 0).endswith("cvna")


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert tune.load_cache(path) == {}
    tune.store("a", 4, [1.0, 0.5, 0.25, 0.3, 0.4, 0.6], path)
    tune.store("b", 8, [-1.0] * 6, path)
    data = tune.load_cache(path)
    assert data["a"]["lanes"] == 4 and data["b"]["lanes"] == 8
    with open(path, "w") as f:
        f.write("not json")
    assert tune.load_cache(path) == {}
    with open(path, "w") as f:
        json.dump([1, 2], f)
    assert tune.load_cache(path) == {}

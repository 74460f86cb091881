"""SpMV configuration of a handle: measured once per graph shape, then cached.

``cb_graph_tune`` times every group width (1, 2, 4, 8, 16, 32 lanes per short
row) of the tiled-CSR SpMV and, in FP32, the path through the formats built
at upload (column-blocked or two-phase kernels) on a short Lanczos run over
the handle, and keeps the fastest width and path.  This module keys the result by the shape of the input -- the
precision, the number of realisations, the largest n, the mean degree and
the coefficient of variation of the degrees, each bucketed -- and keeps a
JSON cache so that later handles of the same shape take the width without
timing.

The cache file is ``$CB_TUNE_CACHE`` if set, else
``~/.cache/paper_1409_5000_gb300/tune.json``.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np


def degree_cv(graphs) -> float:
    """Coefficient of variation of the degrees over all realisations (host CSR)."""
    s1 = s2 = cnt = 0.0
    for g in graphs:
        rp = g.row_ptr.numpy() if hasattr(g.row_ptr, "numpy") else np.asarray(g.row_ptr)
        d = np.diff(rp.astype(np.int64))
        s1 += float(d.sum())
        s2 += float((d.astype(np.float64) ** 2).sum())
        cnt += len(d)
    if cnt == 0 or s1 == 0:
        return 0.0
    mean = s1 / cnt
    return float(math.sqrt(max(s2 / cnt - mean * mean, 0.0)) / mean)


def shape_key(n, nnz, prec: int, cv=None) -> str:
    """Bucketed shape: precision, log2 of N and of the largest n, mean degree
    (rounded to 2^(1/2) steps) and the degree CV (tenths; 'na' if unknown)."""
    N = len(n)
    mean_deg = sum(nnz) / max(sum(n), 1)
    parts = [f"p{prec}", f"N{round(math.log2(N))}", f"n{round(math.log2(max(n)))}",
             f"d{round(2 * math.log2(mean_deg)) if mean_deg > 0 else 'z'}",
             f"cv{round(cv, 1) if cv is not None else 'na'}"]
    return "-".join(parts)


def cache_path() -> str:
    return os.environ.get("CB_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1409_5000_gb300", "tune.json")


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, lanes: int, ms, path=None, spmv_path: int = 0) -> None:
    path = path or cache_path()
    data = load_cache(path)
    data[key] = {"lanes": int(lanes), "path": int(spmv_path), "ms": [float(x) for x in ms]}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(gs, prec: int = 0, graphs=None, path=None, stream=None):
    """Set the handle's group width and SpMV path from the cache, or measure
    and cache them.

    Returns (lanes, from_cache); the path is cb_graph_path(gs.h).  `graphs`
    (the host realisations) adds the degree CV to the key."""
    from . import binding as B

    cv = degree_cv(graphs) if graphs is not None else None
    key = shape_key(gs.n, gs.nnz, prec, cv)
    hit = load_cache(path).get(key)
    if hit is not None and int(hit.get("lanes", 0)) in (1, 2, 4, 8, 16, 32):
        B.cb_graph_set_lanes(gs.h, int(hit["lanes"]))
        B.cb_graph_set_path(gs.h, int(hit.get("path", B.CB_PATH_AUTO)))
        return int(hit["lanes"]), True
    lanes, ms = B.cb_graph_tune(gs.h, prec, B._stream_handle(stream))
    if any(x >= 0 for x in ms):  # only measured shapes are worth remembering
        store(key, lanes, ms, path, B.cb_graph_path(gs.h))
    return lanes, False

"""Tolerances and comparison helpers for CUDA-vs-oracle parity.

Scores are compared as exp(theta) * y without forming the exponential:
the CUDA result is rescaled by exp(theta_gpu - theta_oracle).

Bars (stated as numbers, see the design notes for their derivation):
* FP32 mode: every score in the ranking head (score >= 1e-3 of the
  largest) within 1e-4 relative, and the whole vector within 1e-4 in the
  2-norm; the largest relative error over all nodes is reported too.
* FP64 mode: the same structure at 1e-10.  Scores far below the maximum
  carry only the absolute accuracy of the m-step approximation (about
  eps * max score), so no per-score bound holds there; where the
  approximation has converged (``assert_scores_all``) every score is
  checked.
* top-k indices: bit-exact wherever the gap between the k-th and the
  (k+1)-th oracle score exceeds 10x the score tolerance; otherwise the
  selected sets may differ only inside the tied block.
"""
from __future__ import annotations

import math

import numpy as np

TOL_FP64 = 1e-10
TOL_FP32 = 1e-4
HEAD_FRAC = 1e-3


def rescale(theta_g, y_g, theta_o):
    return np.asarray(y_g, dtype=np.float64) * math.exp(float(theta_g) - float(theta_o))


def errors(theta_g, y_g, theta_o, y_o):
    a = rescale(theta_g, y_g, theta_o)
    b = np.asarray(y_o, dtype=np.float64)
    rel = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    head = b >= HEAD_FRAC * b.max()
    return dict(max_rel=float(rel.max()), head_rel=float(rel[head].max()),
                norm_rel=float(np.linalg.norm(a - b) / np.linalg.norm(b)))


def assert_scores(theta_g, y_g, theta_o, y_o, prec):
    e = errors(theta_g, y_g, theta_o, y_o)
    tol = TOL_FP64 if prec == "fp64" else TOL_FP32
    assert e["head_rel"] <= tol, e
    assert e["norm_rel"] <= tol, e
    return e


def assert_scores_all(theta_g, y_g, theta_o, y_o, tol):
    e = errors(theta_g, y_g, theta_o, y_o)
    assert e["max_rel"] <= tol, e
    return e


def assert_topk(idx_g, val_g, S_o, k, tol):
    """idx_g from the CUDA path (computed on its own scores); S_o oracle scores."""
    order = np.lexsort((np.arange(len(S_o)), -S_o))
    ref = order[:k]
    idx_g = np.asarray(idx_g, dtype=np.int64)
    gap = (S_o[ref[-1]] - S_o[order[k]]) / S_o[ref[-1]] if k < len(S_o) else math.inf
    if gap > 10 * tol:
        assert set(idx_g.tolist()) == set(ref.tolist()), (gap, sorted(idx_g), sorted(ref))
    else:
        # only members of the near-tied block around rank k may differ
        thr = S_o[ref[-1]] * (1 - 10 * tol)
        sure = set(order[: int(np.sum(S_o > S_o[ref[-1]] * (1 + 10 * tol)))].tolist())
        assert sure <= set(idx_g.tolist())
        assert all(S_o[i] >= thr for i in idx_g)
    return gap

"""Seeded synthetic inputs: backgrounds plus an embedded target.

This module is shared by the CUDA path's tests and benchmarks and by the
FP64 oracle's tests.  It holds none of the method's arithmetic, only the
graph generators (compiled from ``csrc/synth.c``) and the recipes that
shape the workloads like the paper's experiments:

* Erdos-Renyi backgrounds with a sparse target OR-ed into each of N
  realisations (paper, "Multiple backgrounds scenario", eq. 5, Table 1);
* ER / Watts-Strogatz / Barabasi-Albert single backgrounds with a planted
  clique (paper, "Single background scenario", Table 3).

Every graph is a simple undirected graph given as a symmetric CSR pattern
(``row_ptr`` uint32[n+1], ``col`` uint32[nnz], rows sorted, no self-loops,
no duplicates), i.e. the 0/1 adjacency matrix A of the paper's "Signal
processing on graphs" section.
"""
from __future__ import annotations

import ctypes
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import math

import numpy as np

SEED_BASE = 14095000

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        from ._build import synth_lib_path, build_synth

        path = synth_lib_path()
        if not os.path.exists(path):
            build_synth()
        lib = ctypes.CDLL(path)
        vp, u32, u64, i64, dbl = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_int64, ctypes.c_double)
        lib.cbs_mix.restype = u64
        lib.cbs_mix.argtypes = [u64, u64, u64]
        lib.cbs_er_begin.restype = vp
        lib.cbs_er_begin.argtypes = [u32, dbl, u64]
        lib.cbs_ba_begin.restype = vp
        lib.cbs_ba_begin.argtypes = [u32, u32, u64]
        lib.cbs_ws_begin.restype = vp
        lib.cbs_ws_begin.argtypes = [u32, u32, dbl, u64]
        lib.cbs_empty_begin.restype = vp
        lib.cbs_empty_begin.argtypes = [u32]
        lib.cbs_add_edges.restype = ctypes.c_int
        lib.cbs_add_edges.argtypes = [vp, vp, vp, u64]
        lib.cbs_finish_count.restype = i64
        lib.cbs_finish_count.argtypes = [vp]
        lib.cbs_finish_fill.restype = ctypes.c_int
        lib.cbs_finish_fill.argtypes = [vp, vp, vp]
        lib.cbs_n.restype = u32
        lib.cbs_n.argtypes = [vp]
        lib.cbs_free.restype = None
        lib.cbs_free.argtypes = [vp]
        lib.cbs_target_edges.restype = i64
        lib.cbs_target_edges.argtypes = [vp, u32, u32, ctypes.c_int, u64, vp, vp, u64]
        lib.cbs_sm64_stream.restype = ctypes.c_int
        lib.cbs_sm64_stream.argtypes = [u64, u64, vp]
        lib.cbs_sample_nodes.restype = ctypes.c_int
        lib.cbs_sample_nodes.argtypes = [u32, u32, u64, vp]
        _LIB = lib
    return _LIB


def seed_for(config: int, realisation: int, salt: int = 0) -> int:
    """Deterministic 64-bit seed for (config, realisation, salt)."""
    return int(_lib().cbs_mix(SEED_BASE + salt, config, realisation))


@dataclass
class Graph:
    """Symmetric CSR pattern of a simple undirected graph."""

    n: int
    row_ptr: np.ndarray  # uint32[n+1]
    col: np.ndarray  # uint32[nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


@dataclass
class Ensemble:
    """N realisations sharing one embedded target (paper eq. 5)."""

    graphs: list
    target: np.ndarray  # uint32[k], sorted node indices of the target
    target_edges: np.ndarray  # uint32[e, 2]
    meta: dict = field(default_factory=dict)

    @property
    def n_max(self) -> int:
        return max(g.n for g in self.graphs)


def _finish(h, extra_edges=None) -> Graph:
    lib = _lib()
    if not h:
        raise ValueError("graph generator rejected its arguments or ran out of memory")
    if extra_edges is not None and len(extra_edges):
        e = np.ascontiguousarray(extra_edges, dtype=np.uint32)
        u = np.ascontiguousarray(e[:, 0])
        v = np.ascontiguousarray(e[:, 1])
        rc = lib.cbs_add_edges(h, u.ctypes.data, v.ctypes.data, len(u))
        if rc != 0:
            lib.cbs_free(h)
            raise ValueError(f"cbs_add_edges failed ({rc})")
    nnz = lib.cbs_finish_count(h)
    if nnz < 0:
        lib.cbs_free(h)
        raise MemoryError("cbs_finish_count failed")
    n = int(lib.cbs_n(h))
    row_ptr = np.empty(n + 1, dtype=np.uint32)
    col = np.empty(max(nnz, 1), dtype=np.uint32)[:nnz]
    rc = lib.cbs_finish_fill(h, row_ptr.ctypes.data, col.ctypes.data if nnz else
                             np.empty(1, np.uint32).ctypes.data)
    if rc != 0:
        raise ValueError("graph too large for uint32 row offsets")
    return Graph(int(n), row_ptr, col)


# ---------------------------------------------------------------------------
# Counter-based ER backgrounds (the definition the device generator
# cb_graph_generate_er follows; this is its CPU statement).
#
# SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014) in counter form: output(c) = mix(seed + (c+1) G),
# G = 0x9E3779B97F4A7C15, mix = the generator's output function.  Realisation
# r takes draws t = 0 .. M_r - 1 with counter c = r * 2^32 + t; draw t gives
# the pair u = (hi32(z) * n) >> 32, v = (lo32(z) * n) >> 32.  Draws with
# u == v are dropped and repeated pairs collapse (a fixed-draw G(n, M)
# reading of the paper's Erdos-Renyi backgrounds); the target's edges are
# OR-ed in; rows come out sorted.
# ---------------------------------------------------------------------------
SM64_GOLDEN = 0x9E3779B97F4A7C15


def sm64_stream(seed: int, count: int) -> np.ndarray:
    """`count` consecutive SplitMix64 outputs from state `seed` (C reference)."""
    out = np.empty(max(count, 1), dtype=np.uint64)
    _lib().cbs_sm64_stream(seed & (2**64 - 1), count, out.ctypes.data)
    return out[:count]


def sm64_counter(seed: int, counters) -> np.ndarray:
    """Counter form of SplitMix64: mix(seed + (c + 1) * G) for each counter c."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & (2**64 - 1)) + (c + np.uint64(1)) * np.uint64(SM64_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def er_draw_count(n: int, dbar: float) -> int:
    """M = floor(dbar * n / 2 + 1/2) draws give mean degree ~dbar."""
    return int(np.floor(float(dbar) * float(n) * 0.5 + 0.5))


def er_draws(n: int, m_draws: int, seed: int, r: int):
    """(u, v) of the M draws of realisation r (u == v not yet dropped)."""
    t = np.arange(m_draws, dtype=np.uint64)
    z = sm64_counter(seed, (np.uint64(r) << np.uint64(32)) + t)
    with np.errstate(over="ignore"):
        u = ((z >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
        v = ((z & np.uint64(0xFFFFFFFF)) * np.uint64(n)) >> np.uint64(32)
    return u.astype(np.int64), v.astype(np.int64)


def er_generated(n: int, m_draws: int, seed: int, r: int, target_edges=None) -> Graph:
    """Realisation r of the counter-based ER recipe, target edges OR-ed in."""
    u, v = er_draws(n, m_draws, seed, r)
    if target_edges is not None and len(target_edges):
        te = np.asarray(target_edges, dtype=np.int64).reshape(-1, 2)
        te = te[(te[:, 0] < n) & (te[:, 1] < n)]
        u = np.concatenate([u, te[:, 0]])
        v = np.concatenate([v, te[:, 1]])
    keep = u != v
    u, v = u[keep], v[keep]
    key = np.unique(np.concatenate([u * n + v, v * n + u]))
    rows = key // n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return Graph(int(n), np.cumsum(row_ptr).astype(np.uint32), (key % n).astype(np.uint32))


def _pairs_to_graph(n: int, u, v, target_edges=None) -> Graph:
    """Symmetric sorted CSR of the pairs (u, v) plus target edges with both
    ends < n; self-loops dropped, repeats collapsed."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if target_edges is not None and len(target_edges):
        te = np.asarray(target_edges, dtype=np.int64).reshape(-1, 2)
        te = te[(te[:, 0] < n) & (te[:, 1] < n)]
        u = np.concatenate([u, te[:, 0]])
        v = np.concatenate([v, te[:, 1]])
    keep = u != v
    u, v = u[keep], v[keep]
    key = np.unique(np.concatenate([u * n + v, v * n + u]))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, key // n + 1, 1)
    return Graph(int(n), np.cumsum(row_ptr).astype(np.uint32), (key % n).astype(np.uint32))


def ws_threshold(p: float) -> int:
    """Rewiring threshold floor(p 2^32) (2^32 at p = 1: every edge rewired)."""
    return int(math.floor(float(p) * 4294967296.0))


def ws_generated(n: int, k: int, p: float, seed: int, r: int, target_edges=None) -> Graph:
    """Realisation r of the counter-based Watts-Strogatz recipe: ring edge
    (i, (i + d) mod n), d = 1..k/2, as draw t = i k/2 + d - 1, rewired to
    (lo32(z) n) >> 32 when hi32(z) < floor(p 2^32)."""
    kh = k // 2
    t = np.arange(n * kh, dtype=np.uint64)
    z = sm64_counter(seed, (np.uint64(r) << np.uint64(32)) + t)
    i = (t // np.uint64(kh)).astype(np.int64)
    d = (t % np.uint64(kh)).astype(np.int64) + 1
    v = (i + d) % n
    with np.errstate(over="ignore"):
        rew = (z >> np.uint64(32)).astype(np.int64) < ws_threshold(p)
        nv = (((z & np.uint64(0xFFFFFFFF)) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
    v = np.where(rew, nv, v)
    return _pairs_to_graph(n, i, v, target_edges)


def ba_targets(n: int, m: int, seed: int, r: int) -> np.ndarray:
    """Targets of the m (n - m) edges of the counter-based Batagelj-Brandes
    recipe: edge t of new node m + t/m picks position
    (lo32(z_t) 2 m T) >> 32, T = t/m, of the earlier endpoint list (even
    2e: node m + e/m; odd 2e + 1: the target of edge e); the first new node
    links to the seeds.  Resolved for all edges at once, step by step."""
    E = m * (n - m)
    t0 = np.arange(E, dtype=np.int64)
    out = np.full(E, -1, dtype=np.int64)
    cur = t0.copy()  # the edge whose target is still needed
    live = np.ones(E, dtype=bool)
    while live.any():
        idx = np.nonzero(live)[0]
        e = cur[idx]
        T = e // m
        seed_hit = T == 0
        out[idx[seed_hit]] = e[seed_hit]
        rest = ~seed_hit
        idx, e, T = idx[rest], e[rest], T[rest]
        z = sm64_counter(seed, (np.uint64(r) << np.uint64(32)) + e.astype(np.uint64))
        with np.errstate(over="ignore"):
            pos = (((z & np.uint64(0xFFFFFFFF)) * (np.uint64(2 * m) * T.astype(np.uint64)))
                   >> np.uint64(32)).astype(np.int64)
        even = (pos & 1) == 0
        out[idx[even]] = m + (pos[even] >> 1) // m
        cur[idx[~even]] = pos[~even] >> 1
        live[:] = False
        live[idx[~even]] = True
    return out


def ba_generated(n: int, m: int, seed: int, r: int, target_edges=None) -> Graph:
    """Realisation r of the counter-based Barabasi-Albert recipe."""
    t = np.arange(m * (n - m), dtype=np.int64)
    return _pairs_to_graph(n, m + t // m, ba_targets(n, m, seed, r), target_edges)


def er(n: int, p: float, seed: int, extra_edges=None) -> Graph:
    """Erdos-Renyi G(n, p) (paper: ER backgrounds, Table 1)."""
    return _finish(_lib().cbs_er_begin(n, float(p), seed), extra_edges)


def ba(n: int, m: int, seed: int, extra_edges=None) -> Graph:
    """Barabasi-Albert, m0 = m seed nodes (paper: BA background, Table 3)."""
    return _finish(_lib().cbs_ba_begin(n, m, seed), extra_edges)


def ws(n: int, k: int, p: float, seed: int, extra_edges=None) -> Graph:
    """Watts-Strogatz small world (paper: SW backgrounds, Tables 2-3)."""
    return _finish(_lib().cbs_ws_begin(n, k, float(p), seed), extra_edges)


def from_edges(n: int, edges) -> Graph:
    """Simple graph from an undirected edge list (duplicates collapse)."""
    return _finish(_lib().cbs_empty_begin(n), np.asarray(edges, dtype=np.uint32).reshape(-1, 2))


def sample_nodes(range_: int, k: int, seed: int) -> np.ndarray:
    out = np.empty(k, dtype=np.uint32)
    if _lib().cbs_sample_nodes(range_, k, seed, out.ctypes.data) != 0:
        raise ValueError("k > range")
    return out


def target_edges(nodes: np.ndarray, extra: int, clique: bool, seed: int) -> np.ndarray:
    """Target sub-graph on `nodes`: random tree + `extra` edges, or a clique."""
    nodes = np.ascontiguousarray(nodes, dtype=np.uint32)
    k = len(nodes)
    cap = max(1, k * (k - 1) // 2)
    eu = np.empty(cap, dtype=np.uint32)
    ev = np.empty(cap, dtype=np.uint32)
    cnt = _lib().cbs_target_edges(nodes.ctypes.data, k, extra, int(clique), seed,
                                  eu.ctypes.data, ev.ctypes.data, cap)
    if cnt < 0:
        raise ValueError("target edge generation failed")
    return np.stack([eu[:cnt], ev[:cnt]], axis=1)


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def er_ensemble(sizes, dbar: float, k: int, extra: int, config: int,
                clique: bool = False, threads: int | None = None) -> Ensemble:
    """N ER realisations (one per entry of `sizes`) sharing one target.

    The target node set is drawn once, uniformly from [0, min(sizes)); its
    edges (random tree + `extra` edges, or a clique) are OR-ed into every
    realisation (paper, "Multiple backgrounds scenario").  p = dbar/(n-1).
    """
    sizes = [int(s) for s in sizes]
    nodes, tedges = _ensemble_target(sizes, k, extra, clique, config)

    def one(r):
        n = sizes[r]
        return er(n, dbar / (n - 1), seed_for(config, r + 1), tedges)

    with ThreadPoolExecutor(threads or _threads()) as ex:
        graphs = list(ex.map(one, range(len(sizes))))
    return Ensemble(graphs, nodes, tedges, dict(kind="er", dbar=dbar, config=config))


def _ensemble_target(sizes, k, extra, clique, config):
    nodes = sample_nodes(min(sizes), k, seed_for(config, 0, salt=1))
    return nodes, target_edges(nodes, extra, clique, seed_for(config, 0, salt=2))


def er_ensemble_member(sizes, dbar: float, k: int, extra: int, config: int, r: int,
                       clique: bool = False) -> Graph:
    """Realisation r of er_ensemble(sizes, dbar, k, extra, config, clique) alone."""
    sizes = [int(s) for s in sizes]
    _, tedges = _ensemble_target(sizes, k, extra, clique, config)
    n = sizes[r]
    return er(n, dbar / (n - 1), seed_for(config, r + 1), tedges)


def er_ensemble_uneven_sizes(n_inst: int = 256, n_lo: int = 20_000, n_hi: int = 400_000,
                             config: int = 3):
    """The realisation sizes er_ensemble_uneven draws."""
    rng = np.random.Generator(np.random.PCG64(seed_for(config, 0, salt=3)))
    return [int(x) for x in rng.integers(n_lo, n_hi + 1, size=n_inst)]


def single_background(kind: str, n: int, k: int, config: int, clique: bool = True,
                      extra: int = 0, dbar: float = 10.0, ba_m: int = 5, ws_k: int = 10,
                      ws_p: float = 0.1) -> Ensemble:
    """One ER / WS / BA background with a planted target (paper Table 3)."""
    nodes = sample_nodes(n, k, seed_for(config, 0, salt=1))
    tedges = target_edges(nodes, extra, clique, seed_for(config, 0, salt=2))
    s = seed_for(config, 1)
    if kind == "er":
        g = er(n, dbar / (n - 1), s, tedges)
    elif kind == "ba":
        g = ba(n, ba_m, s, tedges)
    elif kind == "ws":
        g = ws(n, ws_k, ws_p, s, tedges)
    else:
        raise ValueError(kind)
    return Ensemble([g], nodes, tedges, dict(kind=kind, config=config))


# ---------------------------------------------------------------------------
# Workload recipes.  Shapes follow the paper's experiments, scaled up; the
# exact parameters are those of the project's five benchmark configurations.
# ---------------------------------------------------------------------------

def er_ensemble_small():
    """10 x ER(500, p=0.016) + 15-node tree(+8) target; m=20, k=15."""
    ens = er_ensemble([500] * 10, 0.016 * 499, 15, 8, config=1)
    ens.meta.update(m=20, k=15)
    return ens


def single_clique_100k(kind: str):
    """ER(d=10) / BA(m=5) / WS(k=10,p=0.1) at n=1e5 + 12-clique; m=30, k=12."""
    ens = single_background(kind, 100_000, 12, config=2 + {"er": 0, "ba": 10, "ws": 20}[kind],
                            clique=True, dbar=10.0, ba_m=5, ws_k=10, ws_p=0.1)
    ens.meta.update(m=30, k=12)
    return ens


def er_ensemble_uneven(n_inst: int = 256, n_lo: int = 20_000, n_hi: int = 400_000,
                       dbar: float = 20.0, k: int = 30, extra: int = 15, config: int = 3):
    """N ER realisations, n ~ U[n_lo, n_hi] per instance, dbar=20, 30-node
    tree(+15) target on [0, n_lo); m=25, k=30."""
    sizes = er_ensemble_uneven_sizes(n_inst, n_lo, n_hi, config)
    ens = er_ensemble(sizes, dbar, k, extra, config=config)
    ens.meta.update(m=25, k=k)
    return ens


def ba_clique_large(n: int = 10_000_000, m_ba: int = 8, k: int = 20, config: int = 4):
    """BA(n, m=8) + 20-clique; m=40, k=20."""
    ens = single_background("ba", n, k, config=config, clique=True, ba_m=m_ba)
    ens.meta.update(m=40, k=k)
    return ens


def er_ensemble_grad(n_inst: int = 64, n: int = 100_000, dbar: float = 16.0, k: int = 25,
                     extra: int = 10, config: int = 5):
    """N ER(1e5, dbar=16) + 25-node tree(+10) target; m=30, k=25."""
    ens = er_ensemble([n] * n_inst, dbar, k, extra, config=config)
    ens.meta.update(m=30, k=k)
    return ens

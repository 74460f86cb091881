"""Seeded generators: structure, determinism, and the paper's target shape."""
import os

import numpy as np
import pytest

from paper_1409_5000_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _check_simple(g):
    rp = g.row_ptr.astype(np.int64)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(g.col)
    assert np.all(g.col < g.n)
    for i in range(g.n):
        r = g.col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(r.astype(np.int64)) > 0)  # sorted, no duplicates
        assert not np.any(r == i)  # no self-loops
    # symmetry
    src = np.repeat(np.arange(g.n), np.diff(rp))
    a = set(zip(src.tolist(), g.col.tolist()))
    assert all((v, u) in a for (u, v) in a)


@pytest.mark.parametrize("kind", ["er", "ba", "ws"])
def test_generators_simple_and_deterministic(kind):
    mk = {"er": lambda s: synth.er(300, 0.03, s), "ba": lambda s: synth.ba(300, 3, s),
          "ws": lambda s: synth.ws(300, 6, 0.2, s)}[kind]
    g1, g2, g3 = mk(11), mk(11), mk(12)
    _check_simple(g1)
    assert np.array_equal(g1.row_ptr, g2.row_ptr) and np.array_equal(g1.col, g2.col)
    assert not (np.array_equal(g1.row_ptr, g3.row_ptr) and np.array_equal(g1.col, g3.col))


def test_degree_conventions():
    g = synth.ba(2000, 4, 1)
    assert g.nnz == 2 * 4 * (2000 - 4)  # m edges per new node
    g = synth.ws(1000, 10, 0.1, 1)
    assert g.nnz == 1000 * 10  # rewiring keeps the edge count
    g = synth.er(4000, 10 / 3999, 1)
    assert abs(g.nnz / 4000 - 10) < 0.3  # mean degree dbar = p (n-1)


def test_target_planted_in_every_realisation():
    ens = synth.er_ensemble([200, 300, 250], 4.0, 10, 3, config=77)
    assert len(ens.target_edges) == 9 + 3
    assert np.all(ens.target < 200)
    for g in ens.graphs:
        rp = g.row_ptr
        for u, v in ens.target_edges:
            assert v in g.col[rp[u]:rp[u + 1]]


def test_clique_target():
    nodes = synth.sample_nodes(100, 12, 5)
    e = synth.target_edges(nodes, 0, True, 1)
    assert len(e) == 12 * 11 // 2


def test_paper_sparse_target_shape():
    """A random tree on 20 nodes plus 2 extra edges has the paper's stated
    average degree 2.1 and density 0.11."""
    vals = {}
    with open(os.path.join(GOLDEN, "paper_sparse_target.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    k = int(vals["nodes"])
    e = synth.target_edges(np.arange(k, dtype=np.uint32), 2, False, 3)
    n_e = len(e)
    assert round(2 * n_e / k, 2) == vals["avg_degree"]
    assert round(n_e / (k * (k - 1) / 2), 2) == vals["density"]
    # connected (a spanning tree is inside)
    g = synth.from_edges(k, e)
    seen, stack = {0}, [0]
    while stack:
        u = stack.pop()
        for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
            if int(v) not in seen:
                seen.add(int(v))
                stack.append(int(v))
    assert len(seen) == k


# --- counter-based ER recipe (the definition the device generator follows) ---

def _mix_py(x):
    """SplitMix64 output function on a Python int (mod 2^64), written out."""
    M = (1 << 64) - 1
    z = x & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 17, 2**64 - 1])
def test_sm64_counter_matches_sequential_c(seed):
    """Counter form c -> mix(seed + (c+1) G) equals the C generator's stream."""
    ref = synth.sm64_stream(seed, 64)
    got = synth.sm64_counter(seed, np.arange(64))
    assert np.array_equal(ref, got)
    assert int(got[5]) == _mix_py(seed + 6 * synth.SM64_GOLDEN)


def test_er_generated_matches_loop_statement():
    """The vectorised recipe equals a plain loop over the draws (tiny n)."""
    n, M, seed, r = 37, 60, 2024, 5
    tedges = [(0, 1), (1, 2), (2, 3), (3, 0), (1, 36)]
    adj = set()
    for t in range(M):
        z = _mix_py(seed + ((r << 32) + t + 1) * synth.SM64_GOLDEN)
        u, v = ((z >> 32) * n) >> 32, ((z & 0xFFFFFFFF) * n) >> 32
        if u != v:
            adj |= {(u, v), (v, u)}
    for u, v in tedges:
        adj |= {(u, v), (v, u)}
    g = synth.er_generated(n, M, seed, r, tedges)
    _check_simple(g)
    src = np.repeat(np.arange(n), g.degrees())
    assert set(zip(src.tolist(), g.col.tolist())) == adj


def test_er_generated_degree_and_independence():
    n = 20_000
    M = synth.er_draw_count(n, 8.0)
    g0 = synth.er_generated(n, M, 7, 0)
    g1 = synth.er_generated(n, M, 7, 1)
    # each draw is a uniform pair; collisions and u == v are O(1/n) rare
    assert abs(g0.nnz - 2 * M) <= 2 * M * 5e-3
    assert abs(g0.degrees().mean() - 8.0) < 0.05
    # realisations differ, and their degree variance is Poisson-like
    assert not np.array_equal(g0.col[:1000], g1.col[:1000])
    assert 6.5 < g0.degrees().var() < 9.5


def test_ensemble_member_reproduces_the_ensemble():
    """er_ensemble_member(r) is realisation r of er_ensemble, bit for bit (the
    full-size parity tests rebuild realisations one by one in oracle workers)."""
    sizes = synth.er_ensemble_uneven_sizes(5, 1_000, 4_000, 91)
    ens = synth.er_ensemble_uneven(n_inst=5, n_lo=1_000, n_hi=4_000, config=91)
    assert [g.n for g in ens.graphs] == sizes
    for r in range(5):
        g = synth.er_ensemble_member(sizes, 20.0, 30, 15, 91, r)
        assert np.array_equal(g.row_ptr, ens.graphs[r].row_ptr)
        assert np.array_equal(g.col, ens.graphs[r].col)


def _sm64(seed, c):
    """One counter draw, plain Python integers."""
    M = 2**64 - 1
    z = (seed + (c + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def _edges(g):
    return {(i, int(j)) for i in range(g.n) for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]] if i < j}


def test_ws_statement_equals_plain_loop():
    n, k, seed, r = 40, 6, 123, 3
    for p in (0.0, 0.3, 1.0):
        thr = synth.ws_threshold(p)
        want = set()
        for i in range(n):
            for d in range(1, k // 2 + 1):
                z = _sm64(seed, (r << 32) + i * (k // 2) + d - 1)
                j = (i + d) % n
                if (z >> 32) < thr:
                    j = ((z & 0xFFFFFFFF) * n) >> 32
                if j != i:
                    want.add((min(i, j), max(i, j)))
        assert _edges(synth.ws_generated(n, k, p, seed, r)) == want, p


def test_ws_without_rewiring_is_the_ring_lattice():
    n, k = 50, 8
    g = synth.ws_generated(n, k, 0.0, 9, 0)
    assert np.all(np.diff(g.row_ptr) == k)
    assert _edges(g) == {(min(i, (i + d) % n), max(i, (i + d) % n)) for i in range(n) for d in range(1, 5)}


def _ba_target_plain(n, m, seed, r, t):
    while True:
        T = t // m
        if T == 0:
            return t
        z = _sm64(seed, (r << 32) + t)
        pos = ((z & 0xFFFFFFFF) * (2 * m * T)) >> 32
        if pos % 2 == 0:
            return m + (pos // 2) // m
        t = pos // 2


def test_ba_statement_equals_plain_loop():
    for n, m in [(60, 1), (80, 3), (50, 5)]:
        seed, r = 77, 2
        want = set()
        for t in range(m * (n - m)):
            u, v = m + t // m, _ba_target_plain(n, m, seed, r, t)
            want.add((min(u, v), max(u, v)))
        assert _edges(synth.ba_generated(n, m, seed, r)) == want, (n, m)


def test_ba_structure():
    # m = 1: each new node links to one earlier node, a tree on n nodes
    g = synth.ba_generated(500, 1, 5, 0)
    assert len(_edges(g)) == 499
    seen, stack = {0}, [0]
    while stack:
        i = stack.pop()
        for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]]:
            if int(j) not in seen:
                seen.add(int(j))
                stack.append(int(j))
    assert len(seen) == 500
    # the first new node links to every seed; degrees are heavy-tailed
    m = 3
    g = synth.ba_generated(20_000, m, 6, 0)
    assert set(int(x) for x in g.col[g.row_ptr[m]:g.row_ptr[m + 1]]) >= set(range(m))
    deg = np.diff(g.row_ptr.astype(np.int64))
    assert deg.max() > 20 * deg.mean() and deg.min() >= 1

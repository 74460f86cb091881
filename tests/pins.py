"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each ``check_*`` takes the oracle module (``oracle.communicability``, or a
copy with a planted mistake) and raises AssertionError when the oracle
disagrees with:

* closed forms of e^A 1 (eq. 4) on graphs whose spectrum is known: the
  empty graph, K_n, the cycle C_n, complete bipartite K_{a,b} (stars
  included), the path P_n, and disjoint unions;
* exact integer walk counts sum_k A^k 1 / k! on graphs with n <= 12;
* an independent library expm (scipy's Pade scaling-and-squaring);
* invariants: the lower bound 1 + d + (A^2 1)/2, permutation
  equivariance, monotonicity under edge addition, the spectral identity
  1^T e^A 1 = sum_j e^{lambda_j} (q_j^T 1)^2;
* exactness of the Lanczos approximation once m reaches the dimension of
  the Krylov space K(A, 1);
* linearity of the ensemble sum (eq. 5) and its N = 1 reduction;
* the top-k rule (a full sort, the paper's selection in "Identification algorithm")
  against a brute-force Python sort with ties.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from paper_1409_5000_gb300 import synth


def graph(n, edges):
    g = synth.from_edges(n, np.asarray(edges, dtype=np.uint32).reshape(-1, 2))
    return g.n, g.row_ptr, g.col


def complete(n):
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


def path(n):
    return [(i, i + 1) for i in range(n - 1)]


def bipartite(a, b):
    return [(i, a + j) for i in range(a) for j in range(b)]


def path_closed_form(n):
    """e^A 1 for P_n from its spectrum: lambda_j = 2 cos(pi j/(n+1)),
    q_j(i) = sqrt(2/(n+1)) sin(pi i j/(n+1)), i, j = 1..n."""
    i = np.arange(1, n + 1)
    s = np.zeros(n)
    for j in range(1, n + 1):
        q = math.sqrt(2.0 / (n + 1)) * np.sin(math.pi * i * j / (n + 1))
        s += math.exp(2.0 * math.cos(math.pi * j / (n + 1))) * q * q.sum()
    return s


def bipartite_closed_form(a, b):
    """K_{a,b}: a-side cosh(s) + sqrt(b/a) sinh(s), b-side cosh(s) + sqrt(a/b) sinh(s),
    s = sqrt(ab)."""
    s = math.sqrt(a * b)
    return np.concatenate([np.full(a, math.cosh(s) + math.sqrt(b / a) * math.sinh(s)),
                           np.full(b, math.cosh(s) + math.sqrt(a / b) * math.sinh(s))])


def rel(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1e-300))) if ref.size else 0.0


def krylov_scores(mod, g, m):
    theta, y, m_eff = mod.krylov_expv(*g, m)
    return math.exp(theta) * y, m_eff


CLOSED = [
    ("empty6", lambda: (graph(6, []), np.ones(6), 1)),
    ("K7", lambda: (graph(7, complete(7)), np.full(7, math.exp(6)), 1)),
    ("C9", lambda: (graph(9, cycle(9)), np.full(9, math.exp(2)), 1)),
    ("K3,5", lambda: (graph(8, bipartite(3, 5)), bipartite_closed_form(3, 5), 2)),
    ("star1,6", lambda: (graph(7, bipartite(1, 6)), bipartite_closed_form(1, 6), 2)),
    ("P11", lambda: (graph(11, path(11)), path_closed_form(11), 6)),
    ("P10", lambda: (graph(10, path(10)), path_closed_form(10), 5)),
]


def check_closed_forms_dense(mod):
    for name, mk in CLOSED:
        g, ref, _ = mk()
        err = rel(mod.total_communicability_dense(*g), ref)
        assert err < 1e-13, (name, err)


def check_closed_forms_krylov(mod):
    """Lanczos is exact once m >= dim K(A, 1) (breakdown, or m = dim)."""
    for name, mk in CLOSED:
        g, ref, dim = mk()
        s, m_eff = krylov_scores(mod, g, 20)
        assert m_eff == dim, (name, m_eff, dim)
        err = rel(s, ref)
        assert err < 1e-12, (name, err)
        # exactly at m = dim as well
        s2, _ = krylov_scores(mod, g, dim)
        assert rel(s2, ref) < 1e-12, (name, "m=dim")


def check_disjoint_union(mod):
    # K4 on 0..3, P5 on 4..8, isolated 9, star K_{1,3} on 10..13
    edges = complete(4) + [(4 + a, 4 + b) for a, b in path(5)] + [(10, 11), (10, 12), (10, 13)]
    g = graph(14, edges)
    ref = np.concatenate([np.full(4, math.exp(3)), path_closed_form(5), [1.0],
                          bipartite_closed_form(1, 3)])
    assert rel(mod.total_communicability_dense(*g), ref) < 1e-13
    s, _ = krylov_scores(mod, g, 14)
    assert rel(s, ref) < 1e-11


def _small_random(seed, n):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.15, 0.6)
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return n, edges


def check_walk_counts(mod):
    for seed, n in [(1, 5), (2, 8), (3, 10), (4, 12), (5, 12)]:
        n, edges = _small_random(seed, n)
        g = graph(n, edges)
        ref = mod.total_communicability_walks(n, edges)
        assert rel(mod.total_communicability_dense(*g), ref) < 1e-13, seed
        s, _ = krylov_scores(mod, g, n)  # m = n spans the whole Krylov space
        assert rel(s, ref) < 1e-11, seed


def check_library_expm(mod):
    rng = np.random.default_rng(7)
    for n in (3, 17, 40):
        M = rng.normal(size=(n, n)) * 2.0
        M = M + M.T
        assert rel(mod.expm_taylor(M), sla.expm(M)) < 1e-11
    g = synth.er(120, 0.08, 99)
    A = mod.dense_adjacency(g.n, g.row_ptr, g.col)
    assert rel(mod.expm_taylor(A), sla.expm(A)) < 1e-11


def check_invariants(mod):
    g = synth.er(80, 0.07, 5)
    n, rp, col = g.n, g.row_ptr, g.col
    A = mod.dense_adjacency(n, rp, col)
    s = mod.total_communicability_dense(n, rp, col)
    d = A.sum(axis=1)
    assert np.all(s >= 1.0 + d + 0.5 * (A @ d) - 1e-9)
    # spectral identity 1^T e^A 1 = sum_j e^{lam_j} (q_j^T 1)^2
    lam, Q = np.linalg.eigh(A)
    assert abs(s.sum() - np.sum(np.exp(lam) * (Q.sum(axis=0)) ** 2)) < 1e-10 * s.sum()
    # permutation equivariance s(P A P^T) = P s(A), dense and Krylov
    perm = np.random.default_rng(3).permutation(n)
    inv = np.argsort(perm)
    edges = [(int(inv[i]), int(inv[j])) for i in range(n) for j in col[rp[i]:rp[i + 1]] if i < j]
    gp = graph(n, edges)
    sp_ = mod.total_communicability_dense(*gp)
    assert rel(sp_[inv], s) < 1e-12
    k1, _ = krylov_scores(mod, (n, rp, col), 40)
    k2, _ = krylov_scores(mod, gp, 40)
    assert rel(k2[inv], k1) < 1e-10
    # monotone under edge addition
    extra = [(0, 1), (2, 3), (4, 50)]
    edges0 = [(i, int(j)) for i in range(n) for j in col[rp[i]:rp[i + 1]] if i < j]
    g2 = graph(n, edges0 + extra)
    assert np.all(mod.total_communicability_dense(*g2) >= s - 1e-12)


def check_krylov_converges(mod):
    """At m well above the degree of the exp polynomial needed for the
    spectral width, the Lanczos approximation equals dense e^A 1."""
    for seed, (n, p) in enumerate([(300, 0.03), (200, 0.1)]):
        g = synth.er(n, p, 100 + seed)
        ref = mod.total_communicability_dense(g.n, g.row_ptr, g.col)
        s, _ = krylov_scores(mod, (g.n, g.row_ptr, g.col), 60)
        assert rel(s, ref) < 1e-10, seed
    g = synth.ba(400, 3, 11)
    ref = mod.total_communicability_dense(g.n, g.row_ptr, g.col)
    s, _ = krylov_scores(mod, (g.n, g.row_ptr, g.col), 60)
    assert rel(s, ref) < 1e-10


def check_lanczos_relation(mod):
    """A V^T = V^T T + beta_m v_{m+1} e_m^T with orthonormal V (FP64)."""
    g = synth.er(500, 0.016, 21)
    A = mod.csr_matrix(g.n, g.row_ptr, g.col)
    alpha, beta, V, beta0, m_eff = mod.lanczos(A, 20)
    assert m_eff == 20
    assert abs(beta0 - math.sqrt(g.n)) < 1e-12
    assert np.max(np.abs(V @ V.T - np.eye(20))) < 1e-13
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    R = (A @ V.T) - V.T @ T
    R[:, -1] = 0.0  # last column holds beta_m v_{m+1}
    assert np.max(np.abs(R)) < 1e-12
    assert abs(alpha[0] - g.nnz / g.n) < 1e-12  # alpha_1 = 1^T A 1 / n = mean degree


def check_tridiag(mod):
    # 2x2: T = [[a, b], [b, c]] has exp(T) e1 in closed form
    a, b, c = 1.3, 0.7, -0.4
    theta, v = mod.tridiag_exp_e1(np.array([a, c]), np.array([b, 0.0]))
    ref = sla.expm(np.array([[a, b], [b, c]]))[:, 0]
    mu = (a + c) / 2 + math.sqrt(((a - c) / 2) ** 2 + b * b)
    assert abs(theta - mu) < 1e-14
    assert rel(math.exp(theta) * v, ref) < 1e-14
    rng = np.random.default_rng(1)
    al, be = rng.normal(size=30) * 3, np.abs(rng.normal(size=30))
    theta, v = mod.tridiag_exp_e1(al, be)
    T = np.diag(al) + np.diag(be[:29], 1) + np.diag(be[:29], -1)
    ref = sla.expm(T)[:, 0]
    # normwise: the far entries of e^T e1 are tiny and carry no relative accuracy
    assert np.max(np.abs(math.exp(theta) * v - ref)) < 1e-12 * np.max(np.abs(ref))


def check_ensemble(mod):
    ens = synth.er_ensemble([60, 75, 50], 4.0, 6, 2, config=901)
    gs = [(g.n, g.row_ptr, g.col) for g in ens.graphs]
    theta_star, S = mod.ensemble_scores(gs, 40)
    ref = np.zeros(75)
    for (n, rp, col) in gs:
        ref[:n] += mod.total_communicability_dense(n, rp, col)
    assert rel(math.exp(theta_star) * S, ref) < 1e-10
    t1, s1 = mod.ensemble_scores(gs[:1], 40)
    t0, y0, _ = mod.krylov_expv(*gs[0], 40)
    assert t1 == t0 and rel(s1, y0) < 1e-15


def check_topk(mod):
    rng = np.random.default_rng(5)
    for n, k in [(50, 7), (200, 20), (13, 13), (1, 1)]:
        S = rng.integers(0, 6, size=n).astype(np.float64)  # many ties
        idx, val = mod.topk(S, k)
        ref = sorted(range(n), key=lambda i: (-S[i], i))[:k]
        assert list(idx) == ref
        assert np.array_equal(val, S[ref])


def _closed_walk_sc(n, edges, kmax=60):
    """SC_i = sum_k (A^k)_ii / k! from exact integer closed-walk counts."""
    from fractions import Fraction

    A = [[0] * n for _ in range(n)]
    for u, v in edges:
        A[u][v] = A[v][u] = 1
    P = [[int(i == j) for j in range(n)] for i in range(n)]
    tot = [Fraction(1)] * n
    fact = 1
    for k in range(1, kmax + 1):
        P = [[sum(P[i][q] * A[q][j] for q in range(n)) for j in range(n)] for i in range(n)]
        fact *= k
        tot = [tot[i] + Fraction(P[i][i], fact) for i in range(n)]
    return np.array([float(t) for t in tot])


def check_subgraph_centrality(mod):
    """SC = diag(e^A) (eq. 3): dense and Gauss-quadrature forms."""
    s6 = math.sqrt(6.0)
    cases = [
        (graph(5, []), np.ones(5)),
        (graph(7, complete(7)), np.full(7, (math.exp(6) + 6 * math.exp(-1)) / 7)),
        (graph(7, bipartite(1, 6)),  # star: centre cosh(sqrt s), leaves 1 + (cosh(sqrt s) - 1)/s
         np.concatenate([[math.cosh(s6)], np.full(6, 1 + (math.cosh(s6) - 1) / 6)])),
        (graph(9, cycle(9)),
         np.full(9, sum(math.exp(2 * math.cos(2 * math.pi * j / 9)) for j in range(9)) / 9)),
    ]
    for g, ref in cases:
        assert rel(mod.subgraph_centrality_dense(*g), ref) < 1e-13
        th, c0 = mod.subgraph_centrality_krylov(*g, range(g[0]), g[0])
        assert rel(np.exp(th) * c0, ref) < 1e-11
    for seed, n in [(11, 6), (12, 9), (13, 10)]:
        n, edges = _small_random(seed, n)
        g = graph(n, edges)
        ref = _closed_walk_sc(n, edges)
        assert rel(mod.subgraph_centrality_dense(*g), ref) < 1e-13, seed
        th, c0 = mod.subgraph_centrality_krylov(*g, range(n), n)  # exact at m = n
        assert rel(np.exp(th) * c0, ref) < 1e-11, seed
    # Gauss rule for exp: a lower bound that grows with m
    g = synth.er(80, 0.06, 21)
    dense = mod.subgraph_centrality_dense(g.n, g.row_ptr, g.col)
    nodes = [0, 7, 33, 79]
    prev = np.zeros(len(nodes))
    for m in (1, 2, 3, 5, 8):
        th, c0 = mod.subgraph_centrality_krylov(g.n, g.row_ptr, g.col, nodes, m)
        est = np.exp(th) * c0
        assert np.all(est >= prev * (1 - 1e-13)) and np.all(est <= dense[nodes] * (1 + 1e-12)), m
        prev = est
    th, c0 = mod.subgraph_centrality_krylov(g.n, g.row_ptr, g.col, nodes, 40)
    assert rel(np.exp(th) * c0, dense[nodes]) < 1e-10


def check_restarted(mod):
    """Restarted Lanczos (the paper's ref [10]): one cycle is the plain
    m-step approximation; the cycles converge to e^A 1 (dense form and
    closed forms); a cycle whose start vector spans an invariant subspace
    makes the result exact."""
    g = synth.er(60, 0.1, 77)
    gg = (g.n, g.row_ptr, g.col)
    ref = mod.total_communicability_dense(*gg)
    th0, y0, _ = mod.krylov_expv(*gg, 6)
    th1, y1, run = mod.krylov_expv_restarted(*gg, 6, 1)
    assert run == 1 and abs(th0 - th1) < 1e-13 * th0 and rel(y1, y0) < 1e-13
    errs = []
    for cyc in (1, 2, 3, 4, 6):
        th, y, run = mod.krylov_expv_restarted(*gg, 5, cyc)
        assert run == cyc
        errs.append(rel(np.exp(th) * y, ref))
    assert errs[0] > 1e-3 and all(b < 1e-2 * a for a, b in zip(errs[:3], errs[1:4])), errs
    assert errs[-1] < 1e-12, errs
    b = synth.ba(400, 3, 11)
    bb = (b.n, b.row_ptr, b.col)
    th, y, _ = mod.krylov_expv_restarted(*bb, 8, 4)
    assert rel(np.exp(th) * y, mod.total_communicability_dense(*bb)) < 1e-12
    # closed forms: path (m = 2) and star (m = 1) need many cycles
    th, y, _ = mod.krylov_expv_restarted(*graph(9, path(9)), 2, 8)
    assert rel(np.exp(th) * y, path_closed_form(9)) < 1e-12
    th, y, _ = mod.krylov_expv_restarted(*graph(7, bipartite(1, 6)), 1, 20)
    assert rel(np.exp(th) * y, bipartite_closed_form(1, 6)) < 1e-12
    th, y, _ = mod.krylov_expv_restarted(*graph(7, bipartite(3, 4)), 3, 6)
    assert rel(np.exp(th) * y, bipartite_closed_form(3, 4)) < 1e-12
    # 1 is an eigenvector of a regular graph: the first cycle breaks down, exact
    th, y, run = mod.krylov_expv_restarted(*graph(7, complete(7)), 3, 5)
    assert run == 1 and rel(np.exp(th) * y, np.full(7, math.exp(6))) < 1e-14
    # a start vector other than 1 (an indicator): column 0 of e^A
    e0 = np.zeros(g.n)
    e0[0] = 1.0
    th, y, _ = mod.krylov_expv_restarted(*gg, 6, 6, b=e0)
    col0 = sla.expm(mod.dense_adjacency(*gg))[:, 0]
    assert np.max(np.abs(np.exp(th) * y - col0)) < 1e-12 * np.max(col0)


ALL_CHECKS = [check_closed_forms_dense, check_closed_forms_krylov, check_disjoint_union,
              check_walk_counts, check_library_expm, check_invariants, check_krylov_converges,
              check_lanczos_relation, check_tridiag, check_ensemble, check_topk,
              check_subgraph_centrality, check_restarted]

"""FP64 oracle: total communicability, its Krylov approximation, eq. 5, top-k.

TEST INFRASTRUCTURE ONLY (see the package docstring): not for the product
path.

Notation follows the paper: A is the symmetric 0/1 adjacency matrix of a
simple graph ("Signal processing on graphs"), SC = diag(e^A) (eq. 3),
EBTC = e^A 1, the row sums of e^A (eq. 4), and the ensemble score is the
plain sum of EBTC over N realisations (eq. 5).  The Krylov evaluation of
e^A 1 ("Identification algorithm": the row sums are obtained directly as
e^A 1 with a Krylov method) is the m-step Lanczos approximation

    f_m = beta0 * V_m exp(T_m) e1,  beta0 = ||1|| = sqrt(n),

with V_m the Lanczos basis of K_m(A, 1) and T_m the tridiagonal matrix of
recurrence coefficients.  Scores are returned as the pair (theta, y) with
score = exp(theta) * y, theta = lambda_max(T_m), so that large graphs do
not overflow.

Readings where the paper is silent (Krylov depth, breakdown rule,
reorthogonalisation, shift, tie order) are fixed here and listed in the
design notes: fixed m (krylov_expv_restarted adds the restarted form of
the paper's ref [10]); start vector 1; full
reorthogonalisation (two classical Gram-Schmidt passes); breakdown when
beta_j <= 1e-12 (|alpha_j| + beta_{j-1}) + 1e-300, after which the result
is exact; ties in the top-k go to the smaller node index.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import scipy.sparse as sp

BREAKDOWN_RTOL = 1e-12


# --------------------------------------------------------------------------
# Graph plumbing
# --------------------------------------------------------------------------

def csr_matrix(n, row_ptr, col, weight=None):
    """A as a scipy CSR matrix (float64); `weight` optional per entry."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    data = np.ones(len(col)) if weight is None else np.asarray(weight, dtype=np.float64)
    return sp.csr_matrix((data, col, row_ptr), shape=(n, n))


def dense_adjacency(n, row_ptr, col, weight=None):
    return csr_matrix(n, row_ptr, col, weight).toarray()


# --------------------------------------------------------------------------
# Dense definitions (eq. 3, eq. 4) for small n
# --------------------------------------------------------------------------

def expm_taylor(M):
    """e^M by scaling and squaring a truncated Taylor series (FP64).

    Moler & Van Loan, "Nineteen dubious ways to compute the exponential of
    a matrix": scale M by 2^-s until ||M||_1 / 2^s <= 1/2, sum the Taylor
    series until a term is below 1e-18 of the partial sum (1-norm), then
    square s times.
    """
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    if n == 0:
        return np.zeros((0, 0))
    norm = np.abs(M).sum(axis=0).max()
    s = 0
    while norm / (2.0 ** s) > 0.5:
        s += 1
    X = M / (2.0 ** s)
    E = np.eye(n)
    term = np.eye(n)
    for k in range(1, 200):
        term = term @ X / k
        E = E + term
        tn = np.abs(term).sum(axis=0).max()
        if tn <= 1e-18 * np.abs(E).sum(axis=0).max():
            break
    for _ in range(s):
        E = E @ E
    return E


def total_communicability_dense(n, row_ptr, col, weight=None):
    """EBTC = e^A 1, the row sums of e^A (eq. 4), by dense expm."""
    A = dense_adjacency(n, row_ptr, col, weight)
    return expm_taylor(A) @ np.ones(n)


def subgraph_centrality_dense(n, row_ptr, col):
    """SC_i = (e^A)_ii (eq. 3), by dense expm."""
    return np.diag(expm_taylor(dense_adjacency(n, row_ptr, col))).copy()


def subgraph_centrality_krylov(n, row_ptr, col, nodes, m):
    """SC_i = (e^A)_ii (eq. 3) by Gauss quadrature, for each i in `nodes`.

    e_i^T f(A) e_i is the integral of f against the spectral measure of A
    seen from e_i; the m-step Lanczos process started at e_i (beta0 = 1) gives
    its m-point Gauss rule e1^T f(T_m) e1 (Golub & Meurant, "Matrices,
    Moments and Quadrature with Applications", 2010).  For f = exp every
    derivative is positive, so the rule is a lower bound that increases with
    m, and it is exact once the Krylov space is invariant (breakdown).

    Returns (theta[k], c0[k]) with SC_i ~= exp(theta) * c0.
    """
    A = csr_matrix(n, row_ptr, col)
    thetas, c0 = [], []
    for i in nodes:
        b = np.zeros(n)
        b[int(i)] = 1.0
        alpha, beta, _, _, m_eff = lanczos(A, m, b)
        theta, c = tridiag_exp_e1(alpha, beta)
        thetas.append(theta)
        c0.append(float(c[0]))
    return np.asarray(thetas), np.asarray(c0)


def total_communicability_walks(n, edges, kmax=60):
    """e^A 1 from exact integer walk counts: sum_k (A^k 1) / k!, k <= kmax.

    Pure Python integers and fractions; for n <= 12 only.  The series
    truncation error is below ||A||^(kmax+1) / (kmax+1)! * e^||A||.
    """
    adj = [[0] * n for _ in range(n)]
    for u, v in edges:
        if u != v:
            adj[u][v] = 1
            adj[v][u] = 1
    x = [1] * n
    acc = [Fraction(1)] * n
    fact = 1
    for k in range(1, kmax + 1):
        x = [sum(adj[i][j] * x[j] for j in range(n)) for i in range(n)]
        fact *= k
        acc = [acc[i] + Fraction(x[i], fact) for i in range(n)]
    return np.array([float(a) for a in acc])


# --------------------------------------------------------------------------
# Krylov (Lanczos) approximation of e^A 1
# --------------------------------------------------------------------------

def lanczos(A, m, b=None):
    """m steps of Lanczos on symmetric A from b (default: the ones vector).

    Returns (alpha[m_eff], beta[m_eff] (beta[j] couples v_{j+1} and v_{j+2};
    the last entry is the residual norm beta_m), V[m_eff, n], beta0, m_eff).
    Full reorthogonalisation: two classical Gram-Schmidt passes against all
    previous basis vectors.  Stops early at breakdown (invariant subspace).
    """
    n = A.shape[0]
    b = np.ones(n) if b is None else np.asarray(b, dtype=np.float64)
    beta0 = float(np.linalg.norm(b))
    if n == 0 or beta0 == 0.0:
        return np.zeros(0), np.zeros(0), np.zeros((0, n)), beta0, 0
    V = np.zeros((m, n))
    alpha = np.zeros(m)
    beta = np.zeros(m)
    V[0] = b / beta0
    m_eff = m
    for j in range(m):
        w = A @ V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        alpha[j] = V[j] @ w
        w = w - alpha[j] * V[j]
        for _ in range(2):
            w = w - V[: j + 1].T @ (V[: j + 1] @ w)
        beta[j] = float(np.linalg.norm(w))
        prev = beta[j - 1] if j > 0 else 0.0
        if beta[j] <= BREAKDOWN_RTOL * (abs(alpha[j]) + prev) + 1e-300:
            m_eff = j + 1
            break
        if j + 1 < m:
            V[j + 1] = w / beta[j]
    return alpha[:m_eff], beta[:m_eff], V[:m_eff], beta0, m_eff


def tridiag_exp_e1(alpha, beta_off):
    """(theta, c) with theta = lambda_max(T), c = exp(T - theta I) e1.

    T = tridiag(beta_off, alpha, beta_off).  Dense symmetric
    eigendecomposition T = Q diag(lam) Q^T, then
    c = Q diag(exp(lam - theta)) Q^T e1.
    """
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta_off[: k - 1], 1) + np.diag(beta_off[: k - 1], -1)
    lam, Q = np.linalg.eigh(T)
    theta = float(lam.max())
    c = Q @ (np.exp(lam - theta) * Q[0, :])
    return theta, c


def krylov_expv(n, row_ptr, col, m, weight=None, b=None):
    """m-step Lanczos approximation of e^A b (b = 1 gives EBTC, eq. 4).

    Returns (theta, y, m_eff) with e^A b ~= exp(theta) * y.
    """
    A = csr_matrix(n, row_ptr, col, weight)
    alpha, beta, V, beta0, m_eff = lanczos(A, m, b)
    if m_eff == 0:
        return 0.0, np.zeros(n), 0
    theta, c = tridiag_exp_e1(alpha, beta)
    y = beta0 * (V.T @ c)
    return theta, y, m_eff


def krylov_expv_restarted(n, row_ptr, col, m, cycles, b=None):
    """Restarted Lanczos approximation of e^A b with `cycles` cycles of m steps
    (the restarted Krylov method of the paper's ref [10], Afanasjew, Eiermann,
    Ernst & Guettel 2008).  Cycle k + 1 starts from the (m+1)-th Lanczos vector
    of cycle k, and only the current cycle's basis is needed.  After k cycles
    the approximation is, by definition (Eiermann & Ernst 2006),

        f_k = beta0 [V_1 ... V_k] exp(H_k) e1,

    with H_k block lower bidiagonal: the cycles' tridiagonals T_i on the
    diagonal, and beta^(i) (the last residual norm of cycle i) coupling the
    first row of block i + 1 to the last column of block i.  Evaluated here
    from that definition, with the stacked basis and H_k in full and a dense
    exponential.  A cycle that breaks down ends the process (the result is
    then exact).  Returns (theta, y, cycles_run): f_k = exp(theta) y,
    theta = lambda_max(T_1).
    """
    A = csr_matrix(n, row_ptr, col)
    v = np.ones(n) if b is None else np.asarray(b, dtype=np.float64)
    beta0 = float(np.linalg.norm(v))
    blocks, Vs, couple = [], [], []
    run = 0
    for _ in range(cycles):
        alpha, beta, V, _, m_eff = lanczos(A, m + 1, v)  # step m + 1 only supplies v_{m+1}
        run += 1
        if m_eff <= m:  # breakdown within the cycle: invariant subspace, exact
            blocks.append((alpha, beta))
            Vs.append(V)
            break
        blocks.append((alpha[:m], beta[:m]))
        Vs.append(V[:m])
        couple.append(beta[m - 1])
        v = V[m]
    sizes = [len(a) for a, _ in blocks]
    K = sum(sizes)
    H = np.zeros((K, K))
    o = 0
    for i, (a, bt) in enumerate(blocks):
        k = len(a)
        H[o:o + k, o:o + k] = np.diag(a) + np.diag(bt[: k - 1], 1) + np.diag(bt[: k - 1], -1)
        if i > 0:
            H[o, o - 1] = couple[i - 1]
        o += k
    a1, b1 = blocks[0]
    T1 = np.diag(a1) + np.diag(b1[: len(a1) - 1], 1) + np.diag(b1[: len(a1) - 1], -1)
    theta = float(np.linalg.eigvalsh(T1).max())
    c = expm_taylor(H - theta * np.eye(K))[:, 0]
    y = beta0 * (np.concatenate(Vs, axis=0).T @ c)
    return theta, y, run


def ensemble_scores(graphs, m, n_out=None):
    """Eq. 5: EBTC(i) = sum_r EBTC_r(i), with a common shift.

    `graphs` is a list of (n_r, row_ptr_r, col_r).  Realisation r
    contributes 0 to nodes i >= n_r.  Returns (theta_star, S) with
    EBTC(i) = exp(theta_star) * S[i], theta_star = max_r theta_r; the sum
    runs in realisation order.
    """
    parts = [krylov_expv(n, rp, c, m) for (n, rp, c) in graphs]
    n_out = max(g[0] for g in graphs) if n_out is None else n_out
    theta_star = max(p[0] for p in parts)
    S = np.zeros(n_out)
    for (n, _, _), (theta, y, _) in zip(graphs, parts):
        S[:n] += math.exp(theta - theta_star) * y
    return theta_star, S


def topk(S, k):
    """The k largest scores (section "Identification algorithm"), by a full sort.

    Order: score descending, ties to the smaller node index.  Returns
    (idx int64[k], val float64[k]).
    """
    S = np.asarray(S, dtype=np.float64)
    idx = np.arange(len(S))
    order = np.lexsort((idx, -S))[:k]
    return order.astype(np.int64), S[order]

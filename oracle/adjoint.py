"""FP64 oracle: edge gradient of the summed top-k total communicability.

TEST INFRASTRUCTURE ONLY (see the package docstring): not for the product
path.

The paper has no gradient; this is the adjoint of its scores, defined by
the derivative itself.  With w the indicator of a fixed node set (the
top-k of eq. 5's summed EBTC), one realisation contributes

    L(A) = w^T e^A 1                      (eq. 4 restricted to the set)

and for the undirected weight a_ij = a_ji of an existing edge

    dL/da_ij = G_ij + G_ji,   G = int_0^1 e^{sA} w 1^T e^{(1-s)A} ds,

because the directional derivative of e^A along E is the Frechet derivative
int_0^1 e^{sA} E e^{(1-s)A} ds, and w^T (.) 1 contracts it with E.  The
ensemble gradient (eq. 5) is the sum of the realisations' gradients.

Three independent evaluations:
* ``frechet_block`` -- G as the upper-right block of exp([[A, w 1^T], [0, A]])
  (Van Loan, "Computing integrals involving the matrix exponential", 1978);
* ``frechet_eig`` -- G = Q (F o (Q^T w 1^T Q)) Q^T, F_ab the divided
  differences of exp at the eigenvalues (Daleckii-Krein);
* ``krylov_edge_grad`` -- the m-step Krylov form used at scale: Lanczos
  bases V_w (from w) and V_1 (from 1), G ~ V_w M V_1^T with
  M_ab = ||w|| sqrt(n) int_0^1 (e^{s T_w} e1)_a (e^{(1-s) T_1} e1)_b ds,
  evaluated through the eigendecompositions of T_w and T_1.
"""
from __future__ import annotations

import math

import numpy as np

from .communicability import csr_matrix, dense_adjacency, expm_taylor, lanczos, krylov_expv


def edge_list(n, row_ptr, col):
    """(i, j) of every CSR entry, in CSR order."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    i = np.repeat(np.arange(n), np.diff(rp))
    return i, np.asarray(col, dtype=np.int64)


def frechet_block(A, w):
    """G = int_0^1 e^{sA} w 1^T e^{(1-s)A} ds via one 2n x 2n exponential."""
    n = A.shape[0]
    big = np.zeros((2 * n, 2 * n))
    big[:n, :n] = A
    big[n:, n:] = A
    big[:n, n:] = np.outer(w, np.ones(n))
    return expm_taylor(big)[:n, n:]


def divided_exp(lam):
    """F_ab = (e^{l_a} - e^{l_b}) / (l_a - l_b), F_aa = e^{l_a}."""
    la = lam[:, None]
    lb = lam[None, :]
    d = la - lb
    with np.errstate(invalid="ignore", divide="ignore"):
        F = np.exp(lb) * np.expm1(d) / d
    diag = np.abs(d) < 1e-300
    F[diag] = np.exp(np.broadcast_to(la, d.shape)[diag])
    return F


def frechet_eig(A, w):
    """The same G from A = Q diag(lam) Q^T (Daleckii-Krein)."""
    lam, Q = np.linalg.eigh(A)
    C = Q.T @ np.outer(w, np.ones(A.shape[0])) @ Q
    return Q @ (divided_exp(lam) * C) @ Q.T


def dense_edge_grad(n, row_ptr, col, w, how="block"):
    """dL/da_ij = G_ij + G_ji for every CSR entry (i, j)."""
    A = dense_adjacency(n, row_ptr, col)
    G = frechet_block(A, w) if how == "block" else frechet_eig(A, w)
    i, j = edge_list(n, row_ptr, col)
    return G[i, j] + G[j, i]


def krylov_edge_grad(n, row_ptr, col, w, m):
    """m-step Krylov gradient (theta, g) with dL/da_e ~= exp(theta) * g[e].

    theta = max(lambda_max(T_w), lambda_max(T_1)) is the shift that keeps
    the exponentials bounded.  Returns (0, zeros) when w is zero.
    """
    A = csr_matrix(n, row_ptr, col)
    i, j = edge_list(n, row_ptr, col)
    w = np.asarray(w, dtype=np.float64)
    if not np.any(w):
        return 0.0, np.zeros(len(i))
    aw, bw, Vw, b0w, mw = lanczos(A, m, w)
    a1, b1, V1, b01, m1 = lanczos(A, m, None)

    def eig_T(al, be):
        k = len(al)
        T = np.diag(al) + np.diag(be[: k - 1], 1) + np.diag(be[: k - 1], -1)
        return np.linalg.eigh(T)

    mu, Qw = eig_T(aw, bw)
    nu, Q1 = eig_T(a1, b1)
    theta = float(max(mu.max(), nu.max()))
    # int_0^1 e^{s mu_p} e^{(1-s) nu_q} ds, shifted by theta
    d = mu[:, None] - nu[None, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        Phi = np.exp(nu[None, :] - theta) * np.expm1(d) / d
    same = np.abs(d) < 1e-300
    Phi[same] = np.exp(np.broadcast_to(mu[:, None], d.shape)[same] - theta)
    M = b0w * b01 * (Qw * Qw[0, :]) @ Phi @ (Q1 * Q1[0, :]).T
    P = Vw.T @ M  # n x m1
    U = V1.T  # n x m1
    g = np.einsum("ek,ek->e", P[i], U[j]) + np.einsum("ek,ek->e", P[j], U[i])
    return theta, g


def topk_loss(n, row_ptr, col, nodes, m, weight=None):
    """(theta, l) with sum_{i in nodes} (e^A 1)_i ~= exp(theta) * l (m-step
    Lanczos, optional edge weights: the loss the gradient differentiates)."""
    theta, y, _ = krylov_expv(n, row_ptr, col, m, weight=weight)
    return theta, float(np.sum(y[np.asarray(nodes, dtype=np.int64)]))


def fd_edge_grad(n, row_ptr, col, nodes, m, edges, h=1e-3):
    """Central finite differences of the m-step loss on undirected edges.

    `edges` are CSR entry indices; the weight of the entry and of its
    mirror (j, i) move together by +-h.  Returns values in absolute units.
    """
    i, j = edge_list(n, row_ptr, col)
    rp = np.asarray(row_ptr, dtype=np.int64)
    out = []
    for e in edges:
        a, b = int(i[e]), int(j[e])
        mirror = rp[b] + int(np.searchsorted(col[rp[b]:rp[b + 1]], a))
        vals = []
        for sgn in (1.0, -1.0):
            wgt = np.ones(len(col))
            wgt[e] += sgn * h
            wgt[mirror] += sgn * h
            th, l = topk_loss(n, row_ptr, col, nodes, m, weight=wgt)
            vals.append((th, l))
        th0 = max(vals[0][0], vals[1][0])
        lp = vals[0][1] * math.exp(vals[0][0] - th0)
        lm = vals[1][1] * math.exp(vals[1][0] - th0)
        out.append((th0, (lp - lm) / (2 * h)))
    return out


def ensemble_edge_grad(graphs, nodes, m):
    """Gradient of sum_r sum_{i in nodes, i < n_r} EBTC_r(i) (eq. 5 restricted
    to the set) for every CSR entry of every realisation, concatenated in
    realisation order.  Returns (theta_star, g) with grad = exp(theta_star) g."""
    parts = []
    for (n, rp, col) in graphs:
        w = np.zeros(n)
        sel = np.asarray([x for x in nodes if x < n], dtype=np.int64)
        w[sel] = 1.0
        parts.append(krylov_edge_grad(n, rp, col, w, m))
    theta_star = max(p[0] for p in parts)
    return theta_star, np.concatenate([math.exp(t - theta_star) * g for t, g in parts])

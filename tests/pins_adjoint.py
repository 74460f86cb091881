"""Pins of the FP64 adjoint oracle (edge gradient of the summed top-k score).

Each ``check_*`` takes the adjoint oracle module (or a copy with a planted
mistake) and raises AssertionError when it disagrees with:
* a closed form on the complete graph K_n with w = e_0;
* the other dense evaluation (block exponential vs Daleckii-Krein);
* the scalar identity sum_ij A_ij G_ij = w^T A e^A 1 (the derivative along
  t -> e^{tA} at t = 1);
* central finite differences of w^T e^A 1 in the edge weights (FP64);
* exactness of the Krylov form once m spans the Krylov spaces;
* for the ensemble gradient (eq. 5 restricted to the node set): the dense
  gradient of every realisation, concatenated, and central differences of
  the summed loss sum_r w_r^T e^{A_r} 1, on realisations of uneven n and
  clearly different largest eigenvalues.
"""
from __future__ import annotations

import math

import numpy as np

import oracle.communicability as oc
from paper_1409_5000_gb300 import synth
from tests.pins import complete, graph, rel


def kn_closed_form(n):
    """K_n, w = e_0: G_ij = delta_{i0} a + c, a = e^{n-1}(1 - e^{-n})/n,
    c = (e^{n-1} - a)/n (from e^{sA} e_0 = e^{-s} e_0 + (e^{s(n-1)} - e^{-s})/n 1)."""
    a = math.exp(n - 1) * (1 - math.exp(-n)) / n
    c = (math.exp(n - 1) - a) / n
    G = np.full((n, n), c)
    G[0, :] += a
    return G


def _er60():
    g = synth.er(60, 0.1, 77)
    w = np.zeros(60)
    w[[3, 10, 11, 42, 59]] = 1.0
    return g, w


def check_kn_closed_form(adj):
    n = 9
    rp_g = graph(n, complete(n))
    A = oc.dense_adjacency(*rp_g)
    w = np.zeros(n)
    w[0] = 1.0
    Gref = kn_closed_form(n)
    assert rel(adj.frechet_block(A, w), Gref) < 1e-12
    assert rel(adj.frechet_eig(A, w), Gref) < 1e-11
    i, j = adj.edge_list(*rp_g)
    theta, g = adj.krylov_edge_grad(*rp_g, w, 5)
    assert rel(math.exp(theta) * g, Gref[i, j] + Gref[j, i]) < 1e-11


def check_two_dense_ways(adj):
    g, w = _er60()
    A = oc.dense_adjacency(g.n, g.row_ptr, g.col)
    G1, G2 = adj.frechet_block(A, w), adj.frechet_eig(A, w)
    assert np.max(np.abs(G1 - G2)) < 1e-12 * np.max(np.abs(G1))


def check_scalar_identity(adj):
    g, w = _er60()
    A = oc.dense_adjacency(g.n, g.row_ptr, g.col)
    lhs = w @ A @ oc.expm_taylor(A) @ np.ones(g.n)
    for G in (adj.frechet_block(A, w), adj.frechet_eig(A, w)):
        assert abs(np.sum(A * G) - lhs) < 1e-11 * abs(lhs)
    # the edge gradients sum the same way: sum over CSR entries of g_e / 2 * ... each
    # undirected edge appears twice with the same value G_ij + G_ji
    ge = adj.dense_edge_grad(g.n, g.row_ptr, g.col, w)
    assert abs(0.5 * ge.sum() - lhs) < 1e-11 * abs(lhs)


def check_finite_differences(adj):
    g, w = _er60()
    n = g.n
    A0 = oc.dense_adjacency(n, g.row_ptr, g.col)
    ge = adj.dense_edge_grad(n, g.row_ptr, g.col, w, how="eig")
    i, j = adj.edge_list(n, g.row_ptr, g.col)
    h = 1e-5
    for e in [0, 17, 55, len(i) - 1]:
        a, b = int(i[e]), int(j[e])
        vals = []
        for sgn in (1, -1):
            A = A0.copy()
            A[a, b] += sgn * h
            A[b, a] += sgn * h
            vals.append(w @ oc.expm_taylor(A) @ np.ones(n))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - ge[e]) < 1e-7 * abs(ge[e]), (e, fd, ge[e])


def check_krylov_exact(adj):
    g, w = _er60()
    ge = adj.dense_edge_grad(g.n, g.row_ptr, g.col, w)
    theta, gk = adj.krylov_edge_grad(g.n, g.row_ptr, g.col, w, 60)
    assert rel(math.exp(theta) * gk, ge) < 1e-9


def check_krylov_fd(adj):
    """The m-step loss's own finite differences equal the m-step gradient
    once m has converged (FP64, weights moved by +-1e-4)."""
    g = synth.er(400, 6.0 / 400, 5)
    nodes = [1, 50, 222]
    w = np.zeros(g.n)
    w[nodes] = 1.0
    theta, gk = adj.krylov_edge_grad(g.n, g.row_ptr, g.col, w, 50)
    for e, (th, fd) in zip([3, 700], adj.fd_edge_grad(g.n, g.row_ptr, g.col, nodes, 50, [3, 700],
                                                     h=1e-4)):
        ref = math.exp(theta) * gk[e]
        assert abs(math.exp(th) * fd - ref) < 1e-6 * abs(ref), (e, math.exp(th) * fd, ref)


def _ensemble3():
    """Three realisations of uneven n and spread shifts: a sparse ER(30)
    (lambda_max ~ 3), a denser ER(45) (~ 11) and a star K_{1,20} beside
    isolated nodes (sqrt(20) ~ 4.5).  The node set reaches past n for the
    smaller ones, so each realisation keeps only its own nodes."""
    g0 = synth.er(30, 0.1, 11)
    g1 = synth.er(45, 0.25, 12)
    g2 = synth.from_edges(40, [(5, q) for q in range(20, 40)])
    nodes = [2, 5, 21, 29, 33, 44]
    return [(g.n, g.row_ptr, g.col) for g in (g0, g1, g2)], nodes


def check_ensemble_grad_dense(adj):
    """exp(theta*) g equals the dense FP64 gradient of each realisation,
    concatenated in realisation order, with w_r = 1 on the nodes < n_r
    (m spans every Krylov space, so the Krylov form is exact)."""
    graphs, nodes = _ensemble3()
    theta_s, g = adj.ensemble_edge_grad(graphs, nodes, 50)
    ref = []
    for (n, rp, col) in graphs:
        w = np.zeros(n)
        w[[x for x in nodes if x < n]] = 1.0
        ref.append(adj.dense_edge_grad(n, rp, col, w, how="eig"))
    ref = np.concatenate(ref)
    assert g.shape == ref.shape, (g.shape, ref.shape)
    got = math.exp(theta_s) * g
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
    # entry by entry where the value is not tiny against the largest
    big = np.abs(ref) > 1e-6 * np.max(np.abs(ref))
    assert rel(got[big], ref[big]) < 1e-8
    # theta* is the largest shift: some realisation carries weight exp(0) = 1
    lam = [np.linalg.eigvalsh(oc.dense_adjacency(*gr)).max() for gr in graphs]
    assert theta_s >= max(lam) - 1e-8


def check_ensemble_grad_fd(adj):
    """Central differences of L = sum_r w_r^T e^{A_r} 1 (dense expm, FP64)
    on one edge of every realisation equal the ensemble gradient."""
    graphs, nodes = _ensemble3()
    theta_s, g = adj.ensemble_edge_grad(graphs, nodes, 50)
    h = 1e-5
    off = 0
    for (n, rp, col) in graphs:
        w = np.zeros(n)
        w[[x for x in nodes if x < n]] = 1.0
        A0 = oc.dense_adjacency(n, rp, col)
        i, j = adj.edge_list(n, rp, col)
        e = len(i) // 2
        vals = []
        for sgn in (1, -1):
            A = A0.copy()
            A[i[e], j[e]] += sgn * h
            A[j[e], i[e]] += sgn * h
            # the other realisations' terms do not move
            vals.append(w @ oc.expm_taylor(A) @ np.ones(n))
        fd = (vals[0] - vals[1]) / (2 * h)
        got = math.exp(theta_s) * g[off + e]
        assert abs(fd - got) < 1e-6 * abs(fd), (off, e, fd, got)
        off += len(i)
    assert off == len(g)


ADJ_CHECKS = [check_kn_closed_form, check_two_dense_ways, check_scalar_identity,
              check_finite_differences, check_krylov_exact, check_krylov_fd,
              check_ensemble_grad_dense, check_ensemble_grad_fd]

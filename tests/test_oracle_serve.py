"""Pins for the serving-form oracle (resident gallery, frozen degrees), CPU only."""
import math

import numpy as np
import pytest

import oracle
from tests import bruteforce as bf


def _rand(seed, n, d):
    return np.random.default_rng(seed).standard_normal((n, d))


@pytest.mark.parametrize("symmetric", [True, False])
def test_serve_matches_bruteforce(symmetric):
    G0 = _rand(0, 14, 3)
    Q = _rand(1, 4, 3)
    layers, degs = oracle.gallery_layers(G0, 3, 0.7, 2, symmetric)
    idx, dist, xq = oracle.serve_queries(Q, layers, degs, 3, 0.7, 2, 6, symmetric)
    ref = bf.serve(Q.tolist(), G0.tolist(), 3, 0.7, 2, 6, symmetric)
    assert [list(r) for r in idx] == ref
    # distances are the squared distances on the last gallery layer
    for i in range(4):
        for s, g in enumerate(idx[i]):
            assert abs(dist[i, s] - bf.sqd(xq[i], layers[2][g])) < 1e-12


def test_gallery_layers_are_offline_gcr():
    G0 = _rand(2, 30, 5)
    layers, _ = oracle.gallery_layers(G0, 4, 0.5, 2)
    np.testing.assert_allclose(layers[2], oracle.gcr(G0, 4, 0.5, 2), atol=1e-14)


def test_no_neighbours_leaves_queries_unchanged():
    """k = 0: the query's row holds only its self loop, so it ranks like plain re-ranking on G_T."""
    G0 = _rand(3, 20, 4)
    Q = _rand(4, 5, 4)
    layers, degs = oracle.gallery_layers(G0, 0, 0.5, 2)
    idx, dist, xq = oracle.serve_queries(Q, layers, degs, 0, 0.5, 2, 20)
    np.testing.assert_allclose(xq, oracle.l2_normalize(Q), atol=1e-15)
    ridx, _ = oracle.rerank(oracle.l2_normalize(Q), layers[2])
    assert np.array_equal(idx, ridx)


def test_batch_invariance():
    G0 = _rand(5, 40, 6)
    Q = _rand(6, 7, 6)
    layers, degs = oracle.gallery_layers(G0, 5, 0.4, 2)
    idx_all, d_all, _ = oracle.serve_queries(Q, layers, degs, 5, 0.4, 2, 10)
    for i in range(7):
        idx_1, d_1, _ = oracle.serve_queries(Q[i:i + 1], layers, degs, 5, 0.4, 2, 10)
        assert np.array_equal(idx_1[0], idx_all[i])
        np.testing.assert_allclose(d_1[0], d_all[i], atol=0)


@pytest.mark.parametrize("symmetric", [True, False])
def test_query_row_is_the_row_of_the_augmented_operator(symmetric):
    """One serving step is the query's row of Eq. 7 (or Eq. 6) on the gallery with the query
    appended as one more node.

    The appended node has its self loop and edges to its k nearest gallery rows (Eq. 4); no
    gallery row gains an edge to it, and the gallery nodes keep the degrees of the gallery-only
    graph (frozen). The augmented matrix is built densely with loops, symmetrised as
    (A~ + A~^T)/2 for Eq. 7, and its query row of D^{-1/2} A D^{-1/2} (D_r^{-1/2} A~ D_c^{-1/2}
    for Eq. 6) applied to the stacked features; the query's own degree comes from that matrix.
    """
    k, gamma, d = 3, 0.6, 4
    G0 = _rand(7, 12, d)
    Q = _rand(8, 3, d)
    layers, degs = oracle.gallery_layers(G0, k, gamma, 2, symmetric)
    for t in range(2):
        L = layers[t].tolist()
        n = len(L)
        At = bf.affinity(L, bf.knn_lists(L, k), gamma)           # the gallery-only graph
        if symmetric:
            frozen = [sum((At[i][j] + At[j][i]) / 2.0 for j in range(n)) for i in range(n)]
        else:
            frozen = [sum(At[i][j] for i in range(n)) for j in range(n)]
        np.testing.assert_allclose(degs[t], frozen, atol=1e-13)
        _, _, y = oracle.serve_queries(Q, layers[t:], degs[t:], k, gamma, 1, n, symmetric)
        for qi, q in enumerate(bf.normalize(list(r)) for r in Q.tolist()):
            A = [row[:] + [0.0] for row in At] + [[0.0] * (n + 1)]
            A[n][n] = 1.0
            for j in sorted(range(n), key=lambda j: (bf.sqd(q, L[j]), j))[:k]:
                A[n][j] = math.exp(-bf.sqd(q, L[j]) / gamma)
            X = L + [q]
            if symmetric:
                S = [(A[n][j] + A[j][n]) / 2.0 for j in range(n + 1)]
                D = frozen + [sum(S)]
                row = [S[j] / math.sqrt(D[n] * D[j]) for j in range(n + 1)]
            else:
                Dc = frozen + [sum(A[i][n] for i in range(n + 1))]
                row = [A[n][j] / math.sqrt(sum(A[n]) * Dc[j]) for j in range(n + 1)]
            ref = bf.normalize([sum(row[j] * X[j][c] for j in range(n + 1)) for c in range(d)])
            np.testing.assert_allclose(y[qi], ref, atol=1e-13)

"""Pins for the serving-form oracle (resident gallery, frozen degrees), CPU only."""
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

"""Pins for the FP64 DSFP oracle (Algorithm 1; CPU only).

Each test checks the oracle against something other than itself: closed forms that
Algorithm 1 fixes for special inputs (no neighbours, infinite temperature, one neighbour
worked by hand), the global method's own oracle on data where the two must agree (cliques
of exactly k+1 mutual neighbours, fixed graph), and invariances. Two tests plant a
plausible mistake in a copy of the oracle and check that a pin catches it.
"""
import math

import numpy as np
import pytest

import oracle


def _rand(seed, n, d):
    return np.random.default_rng(seed).standard_normal((n, d))


def _cliques(seed, n_cl, size, d, noise=1.0):
    """n_cl well-separated groups of `size` points: every point's size-1 nearest neighbours
    are exactly its own group."""
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((n_cl, d)) * 4.0
    lab = np.repeat(np.arange(n_cl), size)
    X = C[lab] + noise * rng.standard_normal((n_cl * size, d))
    perm = rng.permutation(n_cl * size)
    return X[perm], lab[perm]


def test_no_neighbours_is_identity():
    X = _rand(0, 9, 5)
    out, _ = oracle.dsfp(X, 0, 0.2, 3)
    np.testing.assert_allclose(out, oracle.l2_normalize(X), atol=1e-15)


def test_zero_iterations_is_identity():
    X = _rand(1, 12, 4)
    out, _ = oracle.dsfp(X, 4, 0.2, 0)
    np.testing.assert_allclose(out, oracle.l2_normalize(X), atol=1e-15)


@pytest.mark.parametrize("T", [1, 2, 3])
def test_infinite_temperature_gives_normalised_local_mean(T):
    # gamma -> inf: every A^i_uv = 1, D = k+1, the operator is the local mean; after the
    # first iteration all local rows are equal, so every later one leaves them unchanged
    X = _rand(2, 15, 6)
    k = 4
    out, nbr = oracle.dsfp(X, k, 1e300, T)
    U = oracle.l2_normalize(X)
    for i in range(X.shape[0]):
        loc = [i] + list(nbr[i])
        mean = U[loc].mean(axis=0)
        np.testing.assert_allclose(out[i], mean / np.linalg.norm(mean), atol=1e-13)


@pytest.mark.parametrize("gamma", [0.2, 0.7])
def test_one_neighbour_worked_by_hand(gamma):
    # k = 1, local set {i, j}: A = [[1, a], [a, 1]], a = exp(-||x_i - x_j||^2 / gamma),
    # D = 1 + a for both. T = 1: x_i + a x_j (normalised). Both rows of X_1 have the same
    # norm (unit inputs), so T = 2: (x_i + a x_j) + a (x_j + a x_i) = (1 + a^2) x_i + 2a x_j.
    X = _rand(3, 10, 7)
    U = oracle.l2_normalize(X)
    out1, nbr = oracle.dsfp(X, 1, gamma, 1)
    out2, _ = oracle.dsfp(X, 1, gamma, 2)
    for i in range(X.shape[0]):
        j = int(nbr[i, 0])
        a = math.exp(-float(np.sum((U[i] - U[j]) ** 2)) / gamma)
        y1 = U[i] + a * U[j]
        y2 = (1 + a * a) * U[i] + 2 * a * U[j]
        np.testing.assert_allclose(out1[i], y1 / np.linalg.norm(y1), atol=1e-14)
        np.testing.assert_allclose(out2[i], y2 / np.linalg.norm(y2), atol=1e-14)


@pytest.mark.parametrize("T", [1, 2, 3])
def test_cliques_match_global_propagation_on_a_fixed_graph(T):
    # groups of exactly k+1 mutual nearest neighbours: the global symmetric operator of
    # Eq. 7, restricted to a group, is the local operator of Algorithm 1 (every pair of the
    # group is an edge both ways, so A = A~ and D = D_r = D_c). With the graph kept fixed
    # the global method then gives the local result row by row.
    k = 5
    X, lab = _cliques(4, 7, k + 1, 16)
    out, nbr = oracle.dsfp(X, k, 0.3, T)
    for i in range(X.shape[0]):
        assert set(nbr[i].tolist()) == set(np.nonzero(lab == lab[i])[0].tolist()) - {i}
    U = oracle.l2_normalize(X)
    g = oracle.build_graph(U, k, 0.3, symmetric=True)
    Y = U
    for _ in range(T):
        Y = oracle.propagate(Y, g["M"])
    np.testing.assert_allclose(out, Y, atol=1e-13)


def test_neighbour_order_does_not_matter():
    X = _rand(5, 20, 6)
    k = 5
    out, nbr = oracle.dsfp(X, k, 0.25, 2)
    rng = np.random.default_rng(9)
    shuffled = np.array([rng.permutation(r) for r in nbr])
    out2, _ = oracle.dsfp(X, k, 0.25, 2, nbr=shuffled)
    np.testing.assert_allclose(out2, out, atol=1e-14)


def test_absent_neighbours_are_skipped():
    # k larger than the other samples: the local set is every sample, the -1 slots are skipped
    X = _rand(6, 4, 3)
    out, nbr = oracle.dsfp(X, 6, 1e300, 1)
    assert (nbr[:, 3:] == -1).all()
    U = oracle.l2_normalize(X)
    mean = U.mean(axis=0)
    np.testing.assert_allclose(out, np.tile(mean / np.linalg.norm(mean), (4, 1)), atol=1e-13)


# ----------------------------------------------------------------------------- planted mistakes
def _dsfp_local_variant(X, i, nbr_i, gamma, T, mistake):
    X = np.asarray(X, dtype=np.float64)
    local = [int(i)] + [int(j) for j in nbr_i if j >= 0]
    Xl = X[local].copy()
    m = len(local)
    A = np.empty((m, m))
    for u in range(m):
        for v in range(m):
            diff = Xl[u] - Xl[v]
            A[u, v] = np.exp(-np.dot(diff, diff) / gamma)
    s = 1.0 / np.sqrt(A.sum(axis=1))
    M = s[:, None] * A * s[None, :]
    if mistake == "normalise_once":
        for _ in range(T):
            Xl = M @ Xl
        return oracle.l2_normalize(Xl)[0]
    for _ in range(T):
        Xl = oracle.l2_normalize(M @ Xl)
    return Xl[1 if mistake == "wrong_row" else 0]


@pytest.mark.parametrize("mistake", ["normalise_once", "wrong_row"])
def test_planted_mistakes_are_caught(mistake):
    k, T = 5, 2
    X, _lab = _cliques(4, 7, k + 1, 16)
    U = oracle.l2_normalize(X)
    nbr, _ = oracle.knn(U, k)
    bad = np.array([_dsfp_local_variant(U, i, nbr[i], 0.3, T, mistake) for i in range(U.shape[0])])
    g = oracle.build_graph(U, k, 0.3, symmetric=True)
    Y = U
    for _ in range(T):
        Y = oracle.propagate(Y, g["M"])
    assert np.max(np.abs(bad - Y)) > 1e-4

"""Pins for the FP64 GCR oracle (CPU only).

Each test checks the oracle against something other than itself: pure-Python brute
force on tiny inputs (tests/bruteforce.py), closed forms that the equations fix for
special inputs, invariants of the operators, and a worked example derived by hand.
A few tests plant a plausible mistake in a copy of an oracle function and check that
the pins catch it.
"""
import math

import numpy as np
import pytest

import oracle
from tests import bruteforce as bf


def _rand(seed, n, d, cams=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    cam = rng.integers(0, cams, size=n) if cams else None
    return X, cam


# ----------------------------------------------------------------------------- distances
def test_sq_dist_expansion_matches_difference_formula():
    X, _ = _rand(1, 17, 9)
    Y, _ = _rand(2, 11, 9)
    np.testing.assert_allclose(oracle.sq_dist(X, Y), oracle.sq_dist_direct(X, Y), rtol=0, atol=1e-12)


def test_unit_rows_distance_is_two_minus_two_cos():
    X, _ = _rand(3, 10, 6)
    U = oracle.l2_normalize(X)
    cos = U @ U.T
    np.testing.assert_allclose(oracle.sq_dist_direct(U, U), 2 - 2 * cos, atol=1e-13)


def test_normalize_zero_row_stays_zero():
    X = np.array([[3.0, 4.0], [0.0, 0.0]])
    np.testing.assert_allclose(oracle.l2_normalize(X), [[0.6, 0.8], [0.0, 0.0]])


# ----------------------------------------------------------------------------- kNN
@pytest.mark.parametrize("seed,n,d,k", [(0, 9, 3, 3), (1, 12, 4, 5), (2, 7, 2, 6), (3, 6, 3, 10)])
def test_knn_matches_bruteforce(seed, n, d, k):
    X, _ = _rand(seed, n, d)
    idx, d2 = oracle.knn(X, k)
    ref = bf.knn_lists(X.tolist(), k)
    for i in range(n):
        got = [int(j) for j in idx[i] if j >= 0]
        assert got == ref[i]                          # same set and same order
        for s, j in enumerate(got):
            assert abs(d2[i, s] - bf.sqd(X[i], X[j])) < 1e-12


def test_knn_rows_in_blocks_match_bruteforce():
    """Rows searched in blocks (here 4 rows per block, a ragged last block) and a row subset
    in an arbitrary order give each row's own N_i."""
    X, cam = _rand(20, 11, 3, cams=3)
    rows = np.array([10, 3, 0, 7, 7, 5, 1, 9, 2])
    ref = bf.knn_lists(X.tolist(), 3)
    ref_cr = bf.knn_lists(X.tolist(), 3, cam.tolist(), cross=True)
    idx, d2 = oracle.knn_rows(X, rows, 3, block=4)
    idx_cr, _ = oracle.knn_rows(X, rows, 3, cam, cross_camera=True, block=4)
    for t, i in enumerate(rows):
        assert [int(j) for j in idx[t] if j >= 0] == ref[i]
        assert [int(j) for j in idx_cr[t] if j >= 0] == ref_cr[i]
        for s, j in enumerate(ref[i]):
            assert abs(d2[t, s] - bf.sqd(X[i], X[j])) < 1e-12


def test_knn_ties_go_to_smaller_index():
    # integer lattice: many exactly equal distances
    X = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [2, 0]], dtype=np.float64)
    idx, _ = oracle.knn(X, 4)
    ref = bf.knn_lists(X.tolist(), 4)
    assert [list(r) for r in idx] == ref
    assert list(idx[0]) == [1, 2, 3, 4]               # four points at distance 1 from the origin


@pytest.mark.parametrize("seed", [4, 5])
def test_cross_camera_knn_matches_bruteforce(seed):
    X, cam = _rand(seed, 13, 3, cams=3)
    idx, _ = oracle.knn(X, 4, cam, cross_camera=True)
    ref = bf.knn_lists(X.tolist(), 4, cam.tolist(), cross=True)
    for i in range(13):
        got = [int(j) for j in idx[i] if j >= 0]
        assert got == ref[i]
        assert all(cam[j] != cam[i] for j in got)


def test_knn_clamps_to_eligible_count():
    X, cam = _rand(6, 5, 3, cams=2)
    cam = np.array([0, 0, 0, 0, 1])
    idx, d2 = oracle.knn(X, 3, cam, cross_camera=True)
    assert list(idx[0]) == [4, -1, -1] and np.isinf(d2[0, 1:]).all()
    assert list(idx[4]) == bf.knn_lists(X.tolist(), 3, cam.tolist(), cross=True)[4]
    assert -1 not in list(idx[4])


# ----------------------------------------------------------------------------- graph (Eq. 4-7)
def test_affinity_and_degrees_match_loops():
    X, _ = _rand(7, 10, 4)
    k, gamma = 3, 0.7
    idx, d2 = oracle.knn(X, k)
    At = oracle.affinity(10, idx, d2, gamma).toarray()
    ref = bf.affinity(X.tolist(), bf.knn_lists(X.tolist(), k), gamma)
    np.testing.assert_allclose(At, np.array(ref), atol=1e-14)
    np.testing.assert_allclose(oracle.affinity_dense(X, idx, gamma), np.array(ref), atol=1e-14)
    Dr, Dc = oracle.degrees(oracle.affinity(10, idx, d2, gamma))
    np.testing.assert_allclose(Dr, [sum(r) for r in ref], atol=1e-13)
    np.testing.assert_allclose(Dc, [sum(ref[i][j] for i in range(10)) for j in range(10)], atol=1e-13)


@pytest.mark.parametrize("symmetric", [True, False])
def test_operator_matches_loops_and_dense(symmetric):
    X, _ = _rand(8, 11, 3)
    idx, d2 = oracle.knn(X, 4)
    At = oracle.affinity(11, idx, d2, 0.5)
    M = oracle.propagation_operator(At, symmetric).toarray()
    ref = bf.operator(At.toarray().tolist(), symmetric)
    np.testing.assert_allclose(M, np.array(ref), atol=1e-14)
    np.testing.assert_allclose(oracle.propagation_operator_dense(At.toarray(), symmetric), M, atol=1e-14)


def test_symmetric_operator_invariants():
    """M = M^T and M D^{1/2} 1 = D^{1/2} 1 (the Perron vector of D^{-1/2} A D^{-1/2})."""
    X, _ = _rand(9, 40, 5)
    idx, d2 = oracle.knn(X, 6)
    At = oracle.affinity(40, idx, d2, 0.3)
    M = oracle.propagation_operator(At, True).toarray()
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    Atd = At.toarray()
    D = 0.5 * (Atd.sum(0) + Atd.sum(1))              # D = (D_r + D_c)/2 for A = (A~ + A~^T)/2
    v = np.sqrt(D)
    np.testing.assert_allclose(M @ v, v, atol=1e-12)
    assert abs(np.max(np.abs(np.linalg.eigvalsh(M))) - 1.0) < 1e-12


def test_asymmetric_operator_invariants():
    """Eq. 6: M D_c^{1/2} 1 = D_r^{1/2} 1 and 1^T D_r^{1/2} M = (D_c^{1/2} 1)^T."""
    X, _ = _rand(10, 30, 4)
    idx, d2 = oracle.knn(X, 5)
    At = oracle.affinity(30, idx, d2, 0.4)
    M = oracle.propagation_operator(At, False).toarray()
    Dr, Dc = oracle.degrees(At)
    np.testing.assert_allclose(M @ np.sqrt(Dc), np.sqrt(Dr), atol=1e-12)
    np.testing.assert_allclose(np.sqrt(Dr) @ M, np.sqrt(Dc), atol=1e-12)


def test_worked_example_three_points():
    """Hand-derived example (Eq. 4-7), three unit vectors at 0, 60 and 180 degrees, k = 1.

    Squared distances: d01 = 1, d12 = 3, d02 = 4, so N_0 = {1}, N_1 = {0}, N_2 = {1}.
    With gamma = 1/ln 2 every weight is 2^-d: w01 = w10 = 1/2, w21 = 1/8.
    A~ = [[1, 1/2, 0], [1/2, 1, 0], [0, 1/8, 1]], D_r = (3/2, 3/2, 9/8), D_c = (3/2, 13/8, 1).
    Symmetric A = [[1, 1/2, 0], [1/2, 1, 1/16], [0, 1/16, 1]], D = (3/2, 25/16, 17/16).
    M = D^{-1/2} A D^{-1/2}: M00 = 2/3, M01 = 2 sqrt(6)/15, M11 = 16/25, M12 = 1/(5 sqrt(17)),
    M22 = 16/17, M02 = 0.
    """
    ang = np.deg2rad([0.0, 60.0, 180.0])
    X = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    g = oracle.build_graph(X, 1, 1.0 / math.log(2.0))
    assert [list(r) for r in g["nbr"]] == [[1], [0], [1]]
    np.testing.assert_allclose(g["At"].toarray(), [[1, .5, 0], [.5, 1, 0], [0, .125, 1]], atol=1e-14)
    Dr, Dc = oracle.degrees(g["At"])
    np.testing.assert_allclose(Dr, [1.5, 1.5, 1.125], atol=1e-14)
    np.testing.assert_allclose(Dc, [1.5, 1.625, 1.0], atol=1e-14)
    M = g["M"].toarray()
    exp = np.array([[2 / 3, 2 * math.sqrt(6) / 15, 0.0],
                    [2 * math.sqrt(6) / 15, 16 / 25, 1 / (5 * math.sqrt(17))],
                    [0.0, 1 / (5 * math.sqrt(17)), 16 / 17]])
    np.testing.assert_allclose(M, exp, atol=1e-14)
    # propagated first row: (2/3) x0 + (2 sqrt 6 / 15) x1, then normalised
    y0 = exp[0, 0] * X[0] + exp[0, 1] * X[1]
    np.testing.assert_allclose(oracle.propagate(X, g["M"])[0], y0 / np.linalg.norm(y0), atol=1e-14)


# ----------------------------------------------------------------------------- propagation
@pytest.mark.parametrize("symmetric", [True, False])
@pytest.mark.parametrize("cross", [False, True])
def test_layer_matches_bruteforce(symmetric, cross):
    X, cam = _rand(11, 12, 3, cams=3)
    U = oracle.l2_normalize(X)
    Y, _ = oracle.gcr_layer(U, 4, 0.6, cam, cross, symmetric, alpha=0.7)
    ref = bf.layer(U.tolist(), 4, 0.6, cam.tolist(), cross, symmetric, 0.7)
    np.testing.assert_allclose(Y, np.array(ref), atol=1e-13)


def test_gcr_iterations_match_bruteforce():
    X, cam = _rand(12, 14, 4, cams=2)
    Y = oracle.gcr(X, 3, 0.5, 3, cam, cross_camera=True, alpha=0.7)
    ref = bf.gcr(X.tolist(), 3, 0.5, 3, cam.tolist(), cross=True, alpha=0.7)
    np.testing.assert_allclose(Y, np.array(ref), atol=1e-12)


@pytest.mark.parametrize("symmetric", [True, False])
def test_full_graph_uniform_weights_collapse_to_mean(symmetric):
    """k = n-1 and gamma -> inf: every weight is 1, so every output row is normalise(mean X)."""
    X, _ = _rand(13, 9, 5)
    U = oracle.l2_normalize(X)
    Y, _ = oracle.gcr_layer(U, 8, 1e300, symmetric=symmetric)
    m = U.mean(axis=0)
    np.testing.assert_allclose(Y, np.tile(m / np.linalg.norm(m), (9, 1)), atol=1e-13)


@pytest.mark.parametrize("symmetric", [True, False])
def test_self_loop_only_is_identity(symmetric):
    """k = 0 (only the self loop of Eq. 4) and gamma -> 0+ (all neighbour weights underflow)."""
    X, _ = _rand(14, 10, 4)
    U = oracle.l2_normalize(X)
    Y0, _ = oracle.gcr_layer(U, 0, 0.2, symmetric=symmetric)
    np.testing.assert_allclose(Y0, U, atol=1e-15)
    Y1, _ = oracle.gcr_layer(U, 3, 1e-6, symmetric=symmetric)
    np.testing.assert_allclose(Y1, U, atol=1e-15)


def test_one_neighbour_is_not_identity():
    X, _ = _rand(15, 8, 3)
    U = oracle.l2_normalize(X)
    Y, _ = oracle.gcr_layer(U, 1, 0.5)
    assert np.max(np.abs(Y - U)) > 1e-3


def test_alpha_mix_endpoints_and_linearity():
    X, cam = _rand(16, 15, 4, cams=3)
    U = oracle.l2_normalize(X)
    g1 = oracle.build_graph(U, 4, 0.5, cam, True, alpha=1.0)
    g0 = oracle.build_graph(U, 4, 0.5, cam, True, alpha=0.0)
    gh = oracle.build_graph(U, 4, 0.5, cam, True, alpha=0.3)
    gg = oracle.build_graph(U, 4, 0.5, cam, False)
    np.testing.assert_allclose(g1["M"].toarray(), gg["M"].toarray(), atol=1e-15)
    Mc = oracle.propagation_operator(g0["At_cr"], True).toarray()
    np.testing.assert_allclose(g0["M"].toarray(), Mc, atol=1e-15)
    np.testing.assert_allclose(gh["M"].toarray(), 0.3 * gg["M"].toarray() + 0.7 * Mc, atol=1e-15)


def test_permutation_equivariance():
    X, cam = _rand(17, 20, 5, cams=3)
    p = np.random.default_rng(0).permutation(20)
    Y = oracle.gcr(X, 4, 0.4, 2, cam, True, alpha=0.6)
    Yp = oracle.gcr(X[p], 4, 0.4, 2, cam[p], True, alpha=0.6)
    np.testing.assert_allclose(Yp, Y[p], atol=1e-13)


def test_given_neighbours_reproduce_search():
    X, cam = _rand(18, 25, 4, cams=2)
    U = oracle.l2_normalize(X)
    g = oracle.build_graph(U, 5, 0.3, cam, True, alpha=0.7)
    g2 = oracle.build_graph(U, 5, 0.3, cam, True, alpha=0.7, nbr=g["nbr"], nbr_cr=g["nbr_cr"])
    np.testing.assert_allclose(g2["M"].toarray(), g["M"].toarray(), atol=1e-15)


# ----------------------------------------------------------------------------- re-ranking
def test_rerank_matches_bruteforce_with_ties():
    Q = np.array([[0, 0], [1, 1]], dtype=np.float64)
    G = np.array([[1, 0], [0, 1], [-1, 0], [2, 2], [1, 1], [0, 0]], dtype=np.float64)
    idx, dist = oracle.rerank(Q, G)
    assert [list(r) for r in idx] == bf.rerank(Q.tolist(), G.tolist())
    assert list(idx[0]) == [5, 0, 1, 2, 4, 3]
    idx3, _ = oracle.rerank(Q, G, topk=3)
    assert [list(r) for r in idx3] == [r[:3] for r in bf.rerank(Q.tolist(), G.tolist())]


def test_rerank_random_matches_bruteforce():
    X, _ = _rand(19, 14, 3)
    idx, dist = oracle.rerank(X[:4], X[4:])
    assert [list(r) for r in idx] == bf.rerank(X[:4].tolist(), X[4:].tolist())
    assert np.all(np.diff(dist, axis=1) >= 0)


# ----------------------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant mistakes in a copy of the oracle's operator and check the pins above fail."""
    X, _ = _rand(20, 12, 3)
    U = oracle.l2_normalize(X)
    idx, d2 = oracle.knn(U, 4)
    At = oracle.affinity(12, idx, d2, 0.6)
    ref = np.array(bf.operator(At.toarray().tolist(), False))

    def swapped_degrees(At):        # transposed operand: D_c on the left, D_r on the right
        Dr, Dc = oracle.degrees(At)
        import scipy.sparse as sp
        return (sp.diags(1 / np.sqrt(Dc)) @ At @ sp.diags(1 / np.sqrt(Dr))).toarray()

    assert np.max(np.abs(swapped_degrees(At) - ref)) > 1e-6

    wrong_sign = oracle.affinity(12, idx, -d2, 0.6).toarray()      # exp(+d/gamma)
    assert np.max(np.abs(wrong_sign - np.array(bf.affinity(U.tolist(), bf.knn_lists(U.tolist(), 4), 0.6)))) > 1e-3

    no_self = At.toarray() - np.eye(12)                             # dropped self loop
    Md = oracle.propagation_operator_dense(no_self + 1e-300, True)
    Mref = oracle.propagation_operator(At, True).toarray()
    assert np.max(np.abs(Md - Mref)) > 1e-3


def test_paper_default_hyperparameters_fixture():
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_defaults.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    assert vals == {"gamma": 0.2, "k": 15, "T": 3, "lambda": 10, "alpha": 0.7}

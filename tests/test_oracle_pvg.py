"""Pins for the FP64 profile-vector oracle (Eq. 10, Eq. 16-17), CPU only."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle


def _video(seed, C, d, cams, max_len=5):
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, max_len + 1, size=C)
    off = np.zeros(C + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    frames = rng.standard_normal((int(off[-1]), d))
    cam = rng.integers(0, cams, size=C)
    return frames, off, cam


def test_mean_profile_by_loops():
    frames, off, _ = _video(0, 6, 4, 2)
    mp = oracle.mean_profiles(frames, off)
    for c in range(6):
        acc = [0.0] * 4
        for f in range(off[c], off[c + 1]):
            for t in range(4):
                acc[t] += frames[f, t]
        np.testing.assert_allclose(mp[c], [a / (off[c + 1] - off[c]) for a in acc], atol=1e-14)


def test_worked_example_orthogonal_frames():
    """Camera with two one-frame tracklets e1 and e2 (d = 2).

    X^T X = e1 e1^T + e2 e2^T = I, n = 2, mu = (e1 + e2)/2, mu_1 - mu = (e1 - e2)/2, so
    Eq. 17 gives w_1 = (e1 - e2) / (2 (1 + 2 lambda)) and w_2 = -w_1.
    """
    frames = np.array([[1.0, 0.0], [0.0, 1.0]])
    off = np.array([0, 1, 2])
    cam = np.array([0, 0])
    lam = 10.0
    W = oracle.pvg_profiles(frames, off, cam, lam)
    w1 = np.array([1.0, -1.0]) / (2 * (1 + 2 * lam))
    np.testing.assert_allclose(W, [w1, -w1], atol=1e-15)


@pytest.mark.parametrize("gram_scale", [1.0, 2.0])
def test_profile_minimises_the_quadratic_bound(gram_scale):
    """Eq. 16 with the Gram term weighted gram_scale/(2n) is minimised by Eq. 17's w_c.

    The objective is written out from Eq. 16 and minimised with L-BFGS (an iterative
    method unrelated to the oracle's Cholesky solve); its minimiser must point along the
    oracle's profile. gram_scale = 2 is the bound exactly as printed (1/n ||Xw||^2);
    gram_scale = 1 is the printed closed form of Eq. 17.
    """
    frames, off, cam = _video(1, 5, 6, 1, max_len=6)
    lam = 0.05
    Xf = oracle.l2_normalize(frames)
    n = Xf.shape[0]
    W = oracle.pvg_profiles(frames, off, cam, lam, gram_scale=gram_scale)
    for c in range(5):
        mu = Xf.mean(axis=0)
        mu_c = Xf[off[c]:off[c + 1]].mean(axis=0)

        def f(w):
            Xw = Xf @ w
            return (mu @ w - mu_c @ w + gram_scale / (2 * n) * (Xw @ Xw) + lam / 2 * (w @ w))

        def g(w):
            return mu - mu_c + gram_scale / n * (Xf.T @ (Xf @ w)) + lam * w

        r = minimize(f, np.zeros(6), jac=g, method="L-BFGS-B", options=dict(gtol=1e-14, ftol=1e-16, maxiter=5000))
        a = r.x / np.linalg.norm(r.x)
        b = W[c] / np.linalg.norm(W[c])
        np.testing.assert_allclose(a, b, atol=1e-6)


def test_large_lambda_tends_to_mean_difference():
    frames, off, cam = _video(2, 8, 5, 2)
    W = oracle.pvg_profiles(frames, off, cam, 1e9)
    Xf = oracle.l2_normalize(frames)
    for c in range(8):
        m = np.nonzero(cam == cam[c])[0]
        if m.shape[0] == 1:
            continue
        Xs = np.concatenate([Xf[off[t]:off[t + 1]] for t in m])
        v = Xf[off[c]:off[c + 1]].mean(0) - Xs.mean(0)
        np.testing.assert_allclose(W[c] / np.linalg.norm(W[c]), v / np.linalg.norm(v), atol=1e-7)


def test_normal_equation_residual():
    frames, off, cam = _video(3, 12, 7, 3)
    lam = 10.0
    W = oracle.pvg_profiles(frames, off, cam, lam)
    Xf = oracle.l2_normalize(frames)
    for c in range(12):
        m = np.nonzero(cam == cam[c])[0]
        if m.shape[0] == 1:
            continue
        Xs = np.concatenate([Xf[off[t]:off[t + 1]] for t in m])
        n = Xs.shape[0]
        lhs = np.zeros(7)
        for row in Xs:                                 # (X^T X) w by explicit rank-1 sums
            lhs += row * (row @ W[c])
        lhs += lam * n * W[c]
        rhs = Xf[off[c]:off[c + 1]].mean(0) - Xs.mean(0)
        assert np.linalg.norm(lhs - rhs) <= 1e-12 * max(1.0, np.linalg.norm(rhs))


def test_single_tracklet_camera_keeps_mean_profile():
    frames, off, cam = _video(4, 4, 3, 2)
    cam = np.array([0, 0, 0, 1])
    W = oracle.pvg_profiles(frames, off, cam, 10.0)
    Xf = oracle.l2_normalize(frames)
    np.testing.assert_allclose(W[3], Xf[off[3]:off[4]].mean(0), atol=1e-15)


def test_gcrv_runs_cross_camera_gcr_on_profiles():
    frames, off, cam = _video(5, 16, 4, 3)
    Y = oracle.gcrv(frames, off, cam, 10.0, 3, 0.5, 2, alpha=0.7)
    W = oracle.pvg_profiles(frames, off, cam, 10.0)
    ref = oracle.gcr(W, 3, 0.5, 2, cam=cam, cross_camera=True, alpha=0.7)
    np.testing.assert_allclose(Y, ref, atol=0)
    np.testing.assert_allclose(np.linalg.norm(Y, axis=1), 1.0, atol=1e-14)

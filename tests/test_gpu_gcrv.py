"""GPU parity tests for the GCRV profile vectors (Eq. 10, Eq. 17) and Algorithm 2.

Tolerances: the profiles come out of FP32 conjugate gradients whose iteration count is set
for a relative error of ~1e-7 (cond <= 1 + 1/lambda), on FP32 frame statistics; rows are
compared after normalisation to 2e-5 absolute, and the FP64 normal-equation residual
||(X_s^T X_s + lambda n_s I) w - (mu_c - mu_s)|| must stay below 1e-4 of the right-hand side.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gcr():
    import paper_2306_08792_gb300 as g
    from paper_2306_08792_gb300 import build
    build.build()
    return g


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _small(seed=0, C=180, d=128, cams=4, max_len=24):
    v = workloads.video(seed=seed, n_query=C // 5, n_gallery=C - C // 5, d=d, n_ids=40, max_len=max_len,
                        n_cams=cams)
    return v


def _unit(A):
    return A / np.linalg.norm(A, axis=1, keepdims=True)


@pytest.mark.parametrize("seed,d,lam", [(0, 128, 10.0), (1, 200, 10.0), (2, 64, 0.5)])
def test_profiles_match_oracle(gcr, seed, d, lam):
    v = _small(seed=seed, d=d)
    cam = v.trk_cam.copy()
    cam[cam == 3] = 2
    cam[7] = 3                                    # camera 3 holds a single tracklet
    W = gcr.gcrv_profiles(_dev(v.frames), _dev(v.trk_off, torch.int64), _dev(cam, torch.int32), 4, lam)
    torch.cuda.synchronize()
    Wg = W.double().cpu().numpy()
    Wo = oracle.pvg_profiles(v.frames, v.trk_off, cam, lam)
    np.testing.assert_allclose(_unit(Wg), _unit(Wo), atol=2e-5, rtol=0)
    np.testing.assert_allclose(np.linalg.norm(Wg, axis=1), np.linalg.norm(Wo, axis=1), rtol=1e-4)
    # the single-tracklet camera keeps its mean profile (Eq. 10)
    np.testing.assert_allclose(Wg[7], oracle.mean_profiles(oracle.l2_normalize(v.frames), v.trk_off)[7], atol=1e-6)


@pytest.mark.parametrize("seed,d", [(3, 128), (4, 260)])
def test_mean_profiles_match_oracle(gcr, seed, d):
    # Eq. 10 on the normalised frames (the ablation baseline of the profile vectors)
    v = _small(seed=seed, d=d)
    W = gcr.gcrv_mean_profiles(_dev(v.frames), _dev(v.trk_off, torch.int64)).double().cpu().numpy()
    Wo = oracle.mean_profiles(oracle.l2_normalize(v.frames), v.trk_off)
    np.testing.assert_allclose(W, Wo, atol=1e-6, rtol=0)


def test_gcrv_algorithm2_staged(gcr):
    """Algorithm 2: GPU profiles, then GPU GCR with both graphs; the oracle's GCR is run on the
    GPU's profiles (staged) and X_T must agree."""
    v = _small(seed=3, C=400, d=128, cams=6, max_len=12)
    lam, k, T = 10.0, 10, 2
    W = gcr.gcrv_profiles(_dev(v.frames), _dev(v.trk_off, torch.int64), _dev(v.trk_cam, torch.int32), 6, lam)
    p = gcr.default_params(k=k, T=T, cross_camera=1, alpha=0.7)
    idx, dist, XT, st = gcr.gcr_pipeline(W, v.n_query, p, _dev(v.trk_cam, torch.int32))
    torch.cuda.synchronize()
    Xo = oracle.gcr(W.double().cpu().numpy(), k, p.gamma, T, cam=v.trk_cam, cross_camera=True, alpha=0.7)
    assert float(np.max(np.abs(XT.cpu().numpy() - Xo))) < 1e-4
    err, viol = parity.ranking_errors(Xo[:v.n_query], Xo[v.n_query:], idx.cpu().numpy(), dist.cpu().numpy())
    assert err < 1e-4 and viol < 2e-4


def test_profiles_full_size_residual(gcr):
    """MARS-shaped workload at full size (13,290 tracklets, ~678k frames, d = 2048): FP64
    normal-equation residual and Eq. 10 means on a sample of tracklets of every camera."""
    v = workloads.video()
    W = gcr.gcrv_profiles(_dev(v.frames), _dev(v.trk_off, torch.int64), _dev(v.trk_cam, torch.int32), 6, v.lam)
    torch.cuda.synchronize()
    Wg = W.double().cpu().numpy()
    rng = np.random.default_rng(0)
    off = v.trk_off
    for s in range(6):
        members = np.nonzero(v.trk_cam == s)[0]
        fr = np.concatenate([np.arange(off[c], off[c + 1]) for c in members])
        Xs = oracle.l2_normalize(v.frames[fr])
        mu_s = Xs.mean(axis=0)
        for c in rng.choice(members, 3, replace=False):
            mu_c = oracle.l2_normalize(v.frames[off[c]:off[c + 1]]).mean(axis=0)
            rhs = mu_c - mu_s
            w = Wg[c]
            lhs = Xs.T @ (Xs @ w) + v.lam * Xs.shape[0] * w
            assert np.linalg.norm(lhs - rhs) <= 1e-4 * np.linalg.norm(rhs), (s, c)

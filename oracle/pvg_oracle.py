"""Plain FP64 oracle for the tracklet profiles of GCRV (Sec. III-D, Eq. 10 and Eq. 17).

Test infrastructure, not product code (see the package docstring).

* Eq. 10: the mean profile of tracklet c is the average of its frame features.
* Eq. 17: the profile vector w_c = (X^T X + lambda n I)^{-1} (mu_c - mu), where X
  stacks the frames of every tracklet recorded by the same camera as c, n is the
  number of those frames, mu their mean and mu_c the mean of c's frames.

Readings (each is listed with its reason in the repository's design notes):

* The printed matrix in Eq. 17 is X X^T (n x n), which cannot multiply a
  d-vector; the Taylor term ||X w_c||^2 of Eq. 16 and the text after Eq. 17
  ("covariance matrix X^T X") fix it as the d x d matrix X^T X.
* The exact minimiser of the Eq. 16 bound has 2 X^T X / n + lambda I; Eq. 17 as
  printed has weight 1 on X^T X. ``gram_scale`` selects 1 (printed, default) or 2.
* Frames are L2-normalised first (Sec. III-D assumes ||x_i|| = 1).
* A camera holding a single tracklet has mu_c = mu and hence w_c = 0; such a
  tracklet keeps its mean profile (Eq. 10) instead.
* Algorithm 2 then runs GCR on the profiles with both the global and the
  cross-camera graph (Eq. 9).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .gcr_oracle import l2_normalize, gcr

__all__ = ["mean_profiles", "pvg_profiles", "gcrv"]


def mean_profiles(frames, trk_off):
    """Eq. 10: x^_c = (1/m_c) sum of the frames of tracklet c (frames taken as given)."""
    F = np.asarray(frames, dtype=np.float64)
    C = len(trk_off) - 1
    out = np.empty((C, F.shape[1]))
    for c in range(C):
        out[c] = F[trk_off[c]:trk_off[c + 1]].mean(axis=0)
    return out


def pvg_profiles(frames, trk_off, trk_cam, lam, gram_scale=1.0):
    """Eq. 17 profile vectors for every tracklet, camera by camera (float64, not normalised).

    Returns W float64 [C, d].
    """
    Xf = l2_normalize(frames)
    trk_off = np.asarray(trk_off, dtype=np.int64)
    trk_cam = np.asarray(trk_cam)
    C = trk_cam.shape[0]
    d = Xf.shape[1]
    mu_c = mean_profiles(Xf, trk_off)
    W = np.empty((C, d))
    for s in np.unique(trk_cam):
        members = np.nonzero(trk_cam == s)[0]
        if members.shape[0] == 1:
            W[members[0]] = mu_c[members[0]]
            continue
        Xs = np.concatenate([Xf[trk_off[c]:trk_off[c + 1]] for c in members], axis=0)
        n_s = Xs.shape[0]
        mu_s = Xs.mean(axis=0)
        G = gram_scale * (Xs.T @ Xs) + lam * n_s * np.eye(d)
        rhs = (mu_c[members] - mu_s[None, :]).T          # d x |members|
        W[members] = sla.cho_solve(sla.cho_factor(G), rhs).T
    return W


def gcrv(frames, trk_off, trk_cam, lam, k, gamma, T, alpha=0.7, symmetric=True, gram_scale=1.0):
    """Algorithm 2: profiles by Eq. 17, then T rounds of global + cross-camera GCR on them."""
    W = pvg_profiles(frames, trk_off, trk_cam, lam, gram_scale)
    return gcr(W, k, gamma, T, cam=np.asarray(trk_cam), cross_camera=True,
               symmetric=symmetric, alpha=alpha)

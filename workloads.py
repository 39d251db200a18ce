"""Seeded synthetic workloads for Graph Convolution based Re-ranking (GCR / GCRV).

This module only draws random numbers. It holds none of the re-ranking arithmetic
(no normalisation, no distances, no graphs): both the FP64 oracle and the CUDA path
receive the raw arrays produced here and apply the method themselves.

The paper evaluates on person re-identification benchmarks (Market-1501, MARS, ...)
with features from trained backbones (Sec. IV-A, IV-B). Neither the data nor the
weights are available, so every workload below is a stand-in with the shape and the
structure of those inputs: identity clusters in feature space, distractors, camera
labels and ragged tracklets. All draws come from ``numpy.random.default_rng(seed)``.

Workloads (n = queries + gallery):

* ``plain``      500 q + 2,000 g, d=256, 100 clusters, sigma=0.3, no cameras.
* ``crosscam``   3,368 q + 15,913 g, d=2048 (Market-1501 shape), 751 clusters,
                 20% distractors, ReLU (non-negative features), 6 cameras.
* ``camera_bias`` the crosscam shape with look-alike identities and per-camera offsets
                 (retrieval-quality measurements).
* ``zipf``       1,000 q + 200,000 g, d=512, 10,000 clusters, Zipf(1.1) sizes.
* ``video``      1,980 q + 11,310 g tracklets (MARS shape), 1,261 identities,
                 2..100 frames each, frame noise sigma=0.2, d=2048, 6 cameras.
* ``serving``    500,000 gallery x d=256 from 25,000 clusters; Poisson arrivals.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class ImageWorkload:
    name: str
    X: np.ndarray               # float32 [n, d], raw (not normalised)
    n_query: int                # rows [0, n_query) are queries, the rest gallery
    cam: Optional[np.ndarray]   # int32 [n] camera id, or None
    label: np.ndarray           # int32 [n] cluster id, -1 for distractors
    k: int
    T: int
    gamma: float = 0.2
    alpha: float = 1.0
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])


@dataclass
class VideoWorkload:
    name: str
    frames: np.ndarray          # float32 [F, d], raw frame features
    trk_off: np.ndarray         # int64 [C+1] frame offsets of each tracklet
    trk_cam: np.ndarray         # int32 [C] camera of each tracklet
    trk_label: np.ndarray       # int32 [C] identity of each tracklet
    n_query: int                # tracklets [0, n_query) are queries
    k: int
    T: int
    lam: float = 10.0
    gamma: float = 0.2
    alpha: float = 0.7

    @property
    def C(self) -> int:
        return int(self.trk_cam.shape[0])


def _clustered(rng, n, d, n_clusters, sigma, cluster_of):
    """x = centroid[cluster] + sigma * eps, generated in row blocks (float32)."""
    cent = rng.standard_normal((n_clusters, d), dtype=np.float32)
    X = np.empty((n, d), dtype=np.float32)
    blk = 8192
    for s in range(0, n, blk):
        e = min(n, s + blk)
        X[s:e] = cent[cluster_of[s:e]]
        X[s:e] += np.float32(sigma) * rng.standard_normal((e - s, d), dtype=np.float32)
    return X


def plain(seed: int = 0, n_query: int = 500, n_gallery: int = 2000, d: int = 256,
          n_clusters: int = 100, sigma: float = 0.3, k: int = 20, T: int = 2) -> ImageWorkload:
    """Plain GCR workload: Gaussian identity clusters, no cameras."""
    rng = np.random.default_rng(seed)
    n = n_query + n_gallery
    lab = rng.integers(0, n_clusters, size=n).astype(np.int32)
    X = _clustered(rng, n, d, n_clusters, sigma, lab)
    return ImageWorkload("plain", X, n_query, None, lab, k=k, T=T, gamma=0.2, alpha=1.0,
                         params=dict(seed=seed, n_clusters=n_clusters, sigma=sigma))


def crosscam(seed: int = 0, n_query: int = 3368, n_gallery: int = 15913, d: int = 2048,
             n_clusters: int = 751, distractor_frac: float = 0.2, sigma: float = 0.3,
             n_cams: int = 6, k: int = 20, T: int = 2, alpha: float = 0.7) -> ImageWorkload:
    """Cross-camera workload with the Market-1501 shape.

    80% of the samples belong to one of ``n_clusters`` identities (x = c + sigma*eps),
    20% are distractors (x = eps, label -1); a ReLU makes every feature non-negative,
    as a ReLU-terminated backbone would. Camera ids are uniform in [0, n_cams).
    """
    rng = np.random.default_rng(seed)
    n = n_query + n_gallery
    lab = rng.integers(0, n_clusters, size=n).astype(np.int32)
    distract = rng.random(n) < distractor_frac
    lab[distract] = -1
    cent = rng.standard_normal((n_clusters, d), dtype=np.float32)
    X = np.empty((n, d), dtype=np.float32)
    blk = 4096
    for s in range(0, n, blk):
        e = min(n, s + blk)
        eps = rng.standard_normal((e - s, d), dtype=np.float32)
        li = lab[s:e]
        base = np.where((li >= 0)[:, None], cent[np.maximum(li, 0)], np.float32(0.0))
        scale = np.where(li >= 0, np.float32(sigma), np.float32(1.0))[:, None]
        X[s:e] = base + scale * eps
    np.maximum(X, 0.0, out=X)
    cam = rng.integers(0, n_cams, size=n).astype(np.int32)
    return ImageWorkload("crosscam", X, n_query, cam, lab, k=k, T=T, gamma=0.2, alpha=alpha,
                         params=dict(seed=seed, n_clusters=n_clusters, sigma=sigma,
                                     distractor_frac=distractor_frac, n_cams=n_cams))


def camera_bias(seed: int = 0, n_query: int = 3368, n_gallery: int = 15913, d: int = 2048,
                n_clusters: int = 751, ids_per_group: int = 5, distractor_frac: float = 0.2,
                tau: float = 0.32, sigma: float = 0.28, cam_bias: float = 0.3, n_cams: int = 6,
                k: int = 20, T: int = 2, alpha: float = 0.7) -> ImageWorkload:
    """Market-1501-shaped workload for retrieval-quality measurements, with the two traits
    that make re-identification hard and that the paper's cross-camera graph addresses
    (Sec. III-C): look-alike identities and camera bias. Identities come in groups of
    ``ids_per_group`` that share a group centre g; identity centre c = g + tau*u; an image is
    x = c + sigma*eps + cam_bias*b_cam with b_cam a per-camera offset. Per unit of variance,
    the same identity on two cameras then shares 1 + tau^2, a look-alike on the same camera
    1 + cam_bias^2, a look-alike on another camera 1. With cam_bias below tau the true match
    on another camera stays the closer one (with cam_bias = 0.3, tau = 0.32 the original
    features give mAP ~0.64 under the cross-camera protocol); past tau a same-camera
    look-alike wins and no method of this family recovers (mAP ~0.2-0.3 for all of them).
    Distractors (label -1) are a group centre plus noise: look-alikes of no identity."""
    rng = np.random.default_rng(seed)
    n = n_query + n_gallery
    n_groups = max(1, (n_clusters + ids_per_group - 1) // ids_per_group)
    lab = rng.integers(0, n_clusters, size=n).astype(np.int32)
    distract = rng.random(n) < distractor_frac
    lab[distract] = -1
    grp = rng.standard_normal((n_groups, d), dtype=np.float32)
    cent = grp[np.arange(n_clusters) // ids_per_group] + np.float32(tau) * rng.standard_normal(
        (n_clusters, d), dtype=np.float32)
    dgrp = rng.integers(0, n_groups, size=n)
    bias = rng.standard_normal((n_cams, d), dtype=np.float32)
    cam = rng.integers(0, n_cams, size=n).astype(np.int32)
    X = np.empty((n, d), dtype=np.float32)
    blk = 4096
    for s in range(0, n, blk):
        e = min(n, s + blk)
        li = lab[s:e]
        base = np.where((li >= 0)[:, None], cent[np.maximum(li, 0)], grp[dgrp[s:e]])
        eps = rng.standard_normal((e - s, d), dtype=np.float32)
        X[s:e] = base + np.float32(sigma) * eps + np.float32(cam_bias) * bias[cam[s:e]]
    return ImageWorkload("camera_bias", X, n_query, cam, lab, k=k, T=T, gamma=0.2, alpha=alpha,
                         params=dict(seed=seed, n_clusters=n_clusters, ids_per_group=ids_per_group,
                                     tau=tau, sigma=sigma, cam_bias=cam_bias,
                                     distractor_frac=distractor_frac, n_cams=n_cams))


def zipf(seed: int = 0, n_query: int = 1000, n_gallery: int = 200000, d: int = 512,
         n_clusters: int = 10000, s: float = 1.1, sigma: float = 0.3, k: int = 30,
         T: int = 3) -> ImageWorkload:
    """Large-scale workload: cluster sizes follow P(r) ~ r^-s over ranks 1..n_clusters."""
    rng = np.random.default_rng(seed)
    n = n_query + n_gallery
    p = np.arange(1, n_clusters + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    lab = rng.choice(n_clusters, size=n, p=p).astype(np.int32)
    X = _clustered(rng, n, d, n_clusters, sigma, lab)
    return ImageWorkload("zipf", X, n_query, None, lab, k=k, T=T, gamma=0.2, alpha=1.0,
                         params=dict(seed=seed, n_clusters=n_clusters, zipf_s=s, sigma=sigma))


def video(seed: int = 0, n_query: int = 1980, n_gallery: int = 11310, d: int = 2048,
          n_ids: int = 1261, min_len: int = 2, max_len: int = 100, sigma_trk: float = 0.3,
          sigma_frame: float = 0.2, n_cams: int = 6, k: int = 20, T: int = 2,
          lam: float = 10.0, cam_bias: float = 0.0) -> VideoWorkload:
    """Video workload with the MARS shape: ragged tracklets of per-frame features.

    Tracklet centre = identity centroid + sigma_trk*eps; each frame = centre +
    sigma_frame*eps. Lengths are uniform in [min_len, max_len]; each tracklet has one
    camera, uniform in [0, n_cams). With cam_bias > 0 every frame also gets its camera's
    offset cam_bias*b_cam (drawn after everything else, so the other draws do not change).
    """
    rng = np.random.default_rng(seed)
    C = n_query + n_gallery
    ident = rng.integers(0, n_ids, size=C).astype(np.int32)
    lens = rng.integers(min_len, max_len + 1, size=C).astype(np.int64)
    cam = rng.integers(0, n_cams, size=C).astype(np.int32)
    off = np.zeros(C + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    cent = rng.standard_normal((n_ids, d), dtype=np.float32)
    centre = cent[ident] + np.float32(sigma_trk) * rng.standard_normal((C, d), dtype=np.float32)
    F = int(off[-1])
    frames = np.empty((F, d), dtype=np.float32)
    blk = 256
    for c0 in range(0, C, blk):
        c1 = min(C, c0 + blk)
        f0, f1 = int(off[c0]), int(off[c1])
        owner = np.repeat(np.arange(c0, c1), lens[c0:c1])
        frames[f0:f1] = centre[owner]
        frames[f0:f1] += np.float32(sigma_frame) * rng.standard_normal((f1 - f0, d), dtype=np.float32)
    if cam_bias > 0:
        bias = rng.standard_normal((n_cams, d), dtype=np.float32)
        for c0 in range(0, C, blk):
            c1 = min(C, c0 + blk)
            f0, f1 = int(off[c0]), int(off[c1])
            frames[f0:f1] += np.float32(cam_bias) * bias[np.repeat(cam[c0:c1], lens[c0:c1])]
    return VideoWorkload("video", frames, off, cam, ident, n_query, k=k, T=T, lam=lam)


@dataclass
class ServingWorkload:
    gallery: np.ndarray          # float32 [ng, d] raw
    centroids: np.ndarray        # float32 [n_clusters, d]
    sigma: float
    k: int
    T: int
    arrivals: np.ndarray         # float64 [R] arrival times (s)
    batch: np.ndarray            # int32 [R] queries per request
    seed: int

    def queries_of(self, b: int, tag: int = 1 << 30) -> np.ndarray:
        """b query rows drawn like a request's (seeded by b and a tag outside request indices)."""
        rng = np.random.default_rng((self.seed, tag, b))
        cl = rng.integers(0, self.centroids.shape[0], size=b)
        q = self.centroids[cl] + np.float32(self.sigma) * rng.standard_normal(
            (b, self.centroids.shape[1]), dtype=np.float32)
        return q.astype(np.float32)

    def queries(self, r: int) -> np.ndarray:
        """Query features of request r (seeded by the request index)."""
        rng = np.random.default_rng((self.seed, r))
        b = int(self.batch[r])
        cl = rng.integers(0, self.centroids.shape[0], size=b)
        q = self.centroids[cl] + np.float32(self.sigma) * rng.standard_normal(
            (b, self.centroids.shape[1]), dtype=np.float32)
        return q.astype(np.float32)


def serving(seed: int = 0, n_gallery: int = 500000, d: int = 256, n_clusters: int = 25000,
            sigma: float = 0.3, k: int = 20, T: int = 2, n_requests: int = 10000,
            rate: float = 200.0, max_batch: int = 512) -> ServingWorkload:
    """Serving workload: resident gallery, Poisson arrivals, log-uniform batch sizes."""
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, n_clusters, size=n_gallery).astype(np.int32)
    cent = rng.standard_normal((n_clusters, d), dtype=np.float32)
    G = np.empty((n_gallery, d), dtype=np.float32)
    blk = 65536
    for s in range(0, n_gallery, blk):
        e = min(n_gallery, s + blk)
        G[s:e] = cent[lab[s:e]] + np.float32(sigma) * rng.standard_normal((e - s, d), dtype=np.float32)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    arrivals = np.cumsum(gaps)
    b = np.floor(np.exp(rng.uniform(0.0, np.log(max_batch), size=n_requests)))
    b = np.clip(b, 1, max_batch).astype(np.int32)
    return ServingWorkload(G, cent, sigma, k, T, arrivals, b, seed)


def random_unit_like(seed: int, n: int, d: int, cams: int = 0):
    """Small unstructured inputs for edge-case tests: Gaussian rows (+ optional cameras)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    cam = rng.integers(0, cams, size=n).astype(np.int32) if cams > 0 else None
    return X, cam

"""Plain FP64 oracle for re-ranking against a resident gallery (serving form of GCR).

Test infrastructure, not product code (see the package docstring).

Sec. IV-F2 notes that with the gallery's graphs computed and stored in advance the cost per
query drops to O(N log N). The serving form follows that remark:

* Offline: GCR over the gallery alone gives layers G_0 .. G_T (G_0 = normalised gallery,
  G_t = normalise(M_t G_{t-1}), graph rebuilt per layer, Eq. 3) and, for each layer t < T,
  the degrees of that layer's gallery graph (Eq. 5, and D = (D_r + D_c)/2 for Eq. 7).
* Per query q (the gallery frozen, no query-query edges, the query never enters a gallery
  row's neighbour list): for t = 1..T, N_q = the k nearest rows of G_{t-1} to x_q, weights
  w_qj = exp(-||x_q - g_j||^2 / gamma) (Eq. 4), and the query's row of the operator:
    symmetric (Eq. 7): A_qq = 1, A_qj = w_qj / 2, D_q = (1 + sum_j w_qj + 1) / 2,
                       y = x_q / D_q + sum_j (w_qj / 2) g_j / sqrt(D_q D_j)
    asymmetric (Eq. 6): y = x_q / sqrt(r_q * 1) + sum_j w_qj g_j / sqrt(r_q Dc_j),
                        r_q = 1 + sum_j w_qj
  then x_q <- normalise(y).
* Finally the gallery is ranked by ||x_q - g||^2 on G_T (ties to the smaller index) and the
  top K are returned.

These readings (frozen degrees, the query's own column degree 1, no query-query edges) are
listed in the repository's design notes.
"""
from __future__ import annotations

import numpy as np

from .gcr_oracle import build_graph, degrees, l2_normalize, propagate, sq_dist

__all__ = ["gallery_layers", "serve_queries"]


def gallery_layers(Xg, k, gamma, T, symmetric=True):
    """Layers G_0..G_T of offline GCR on the gallery and the degrees used by queries."""
    G = l2_normalize(Xg)
    layers, degs = [G], []
    for _ in range(T):
        g = build_graph(G, k, gamma, symmetric=symmetric)
        Dr, Dc = degrees(g["At"])
        degs.append(0.5 * (Dr + Dc) if symmetric else Dc)
        G = propagate(G, g["M"])
        layers.append(G)
    return layers, degs


def _query_step(xq, G, deg, k, gamma, symmetric):
    Y = np.empty_like(xq)
    for i in range(xq.shape[0]):
        D = sq_dist(xq[i:i + 1], G)[0]
        idx = np.argsort(D, kind="stable")[:k]
        w = np.exp(-D[idx] / gamma)
        if symmetric:
            Dq = 0.5 * (1.0 + w.sum() + 1.0)
            Y[i] = xq[i] / Dq + ((0.5 * w) / np.sqrt(Dq * deg[idx])) @ G[idx]
        else:
            r = 1.0 + w.sum()
            Y[i] = xq[i] / np.sqrt(r) + (w / np.sqrt(r * deg[idx])) @ G[idx]
    return l2_normalize(Y)


def serve_queries(Q, layers, degs, k, gamma, T, K, symmetric=True):
    """Top-K gallery indices and squared distances of each query (rows of Q, raw features)."""
    xq = l2_normalize(Q)
    for t in range(T):
        xq = _query_step(xq, layers[t], degs[t], k, gamma, symmetric)
    D = sq_dist(xq, layers[T])
    K = min(K, D.shape[1])
    idx = np.argsort(D, axis=1, kind="stable")[:, :K]
    return idx, np.take_along_axis(D, idx, axis=1), xq

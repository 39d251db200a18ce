"""Plain FP64 oracle for GCR (Graph Convolution based Re-ranking, arXiv 2306.08792).

Test infrastructure, not product code: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline arm of ``bench.py`` use it. It shares no code with the CUDA
path. Everything here is computed in float64 with numpy / scipy.sparse; it is slow
on purpose and follows the paper's equations in their order:

* Sec. III-A, Eq. 2-3: X_t = G(X_{t-1}), G(X) = D^{-1/2} A D^{-1/2} X (W = I).
* Sec. III-B, Eq. 4: A~_ij = exp(-||x_i - x_j||^2 / gamma) for j in N_i, 1 on the
  diagonal, 0 elsewhere; N_i = the k nearest samples of i (i itself excluded).
* Eq. 5: row degree D_r(i,i) = sum_j A~_ij, column degree D_c(j,j) = sum_i A~_ij.
* Eq. 6: asymmetric operator D_r^{-1/2} A~ D_c^{-1/2}.
* Eq. 7: symmetric A = (A~ + A~^T)/2 with D = diag(A 1), operator D^{-1/2} A D^{-1/2}.
* Sec. III-C, Eq. 8-9: the cross-camera graph (neighbours restricted to other
  cameras) and the alpha-mix of the two operators.
* Sec. III-A (retrieval by Euclidean distance): the re-ranked distance is the squared
  Euclidean distance between the final features, and each query's gallery list is
  sorted by it.

Readings where the paper is silent (each one is listed with its reason in the
design notes of the repository):

1. N_i excludes i (Eq. 4 gives j = i its own case; Algorithm 1 adds i to N_i).
2. The graphs are rebuilt from the current features at every iteration
   (Sec. III-C: the similarity matrices and neighbour graphs change across
   iterations; Algorithm 2 rebuilds them inside its loop).
3. The symmetric operator (Eq. 7) is the default, for both graphs of Eq. 9.
4. Rows are L2-normalised on input and after every propagation layer (Sec. III-D
   assumes unit features); a row of norm 0 stays 0.
5. Ties in the kNN search go to the smaller index; the final sort is stable in the
   gallery index.
6. When fewer than k samples are eligible (k >= n, or few other-camera samples), a
   row keeps all eligible samples.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = [
    "l2_normalize", "sq_dist_direct", "sq_dist", "knn", "knn_rows",
    "affinity", "degrees", "propagation_operator", "build_graph", "propagate",
    "gcr_layer", "gcr", "rerank", "affinity_dense", "propagation_operator_dense",
]


# ----------------------------------------------------------------------------
# features and distances
# ----------------------------------------------------------------------------
def l2_normalize(X):
    """x_i <- x_i / ||x_i||_2 in float64 (Sec. III-D assumes ||x_i|| = 1); zero rows stay 0."""
    X = np.asarray(X, dtype=np.float64)
    nrm = np.sqrt(np.sum(X * X, axis=1, keepdims=True))
    out = np.zeros_like(X)
    nz = nrm[:, 0] > 0
    out[nz] = X[nz] / nrm[nz]
    return out


def sq_dist_direct(A, B):
    """||a_i - b_j||^2 written out as sum_k (a_ik - b_jk)^2 (Eq. 4). O(na*nb*d) memory-chunked."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.empty((A.shape[0], B.shape[0]), dtype=np.float64)
    for i in range(A.shape[0]):
        diff = B - A[i][None, :]
        out[i] = np.sum(diff * diff, axis=1)
    return out


def sq_dist(A, B):
    """||a_i - b_j||^2 = ||a_i||^2 + ||b_j||^2 - 2 a_i.b_j, with a float64 matmul.

    Same quantity as :func:`sq_dist_direct` (a pin checks the two against each other);
    used wherever the direct form would be too slow.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    na = np.sum(A * A, axis=1)[:, None]
    nb = np.sum(B * B, axis=1)[None, :]
    return na + nb - 2.0 * (A @ B.T)


# ----------------------------------------------------------------------------
# k-nearest-neighbour search (Sec. III-B, N_i; Sec. III-C, N_i^cr)
# ----------------------------------------------------------------------------
def _select_row(drow, k):
    """Indices of the k smallest entries of drow (inf = ineligible), ties to the smaller index."""
    finite = np.isfinite(drow)
    m = int(np.count_nonzero(finite))
    kk = min(k, m)
    if kk == 0:
        return np.empty(0, dtype=np.int64)
    vk = np.partition(drow, kk - 1)[kk - 1]
    cand = np.nonzero(drow <= vk)[0]                 # ascending index order
    order = np.argsort(drow[cand], kind="stable")    # stable: equal distance -> smaller index
    return cand[order][:kk]


def knn_rows(X, rows, k, cam=None, cross_camera=False, block=512):
    """kNN of the given rows of X against all rows of X.

    N_i = the k samples j != i with the smallest ||x_i - x_j||^2 (Eq. 4). With
    ``cross_camera`` the candidates are restricted to cam_j != cam_i (Sec. III-C, Eq. 8).
    Returns (idx int64 [m, k], d2 float64 [m, k]); a row with fewer than k eligible
    samples is padded with idx -1 and d2 inf.
    """
    X = np.asarray(X, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    m = rows.shape[0]
    idx = np.full((m, k), -1, dtype=np.int64)
    d2 = np.full((m, k), np.inf, dtype=np.float64)
    for s in range(0, m, block):
        r = rows[s:s + block]
        D = sq_dist(X[r], X)
        D[np.arange(r.shape[0]), r] = np.inf         # i itself is not in N_i
        if cross_camera:
            D[cam[r][:, None] == cam[None, :]] = np.inf
        for t in range(r.shape[0]):
            sel = _select_row(D[t], k)
            idx[s + t, :sel.shape[0]] = sel
            d2[s + t, :sel.shape[0]] = D[t, sel]
    return idx, d2


def knn(X, k, cam=None, cross_camera=False):
    """kNN of every row of X (see :func:`knn_rows`)."""
    return knn_rows(X, np.arange(np.asarray(X).shape[0]), k, cam, cross_camera)


# ----------------------------------------------------------------------------
# graph, degrees and propagation operator (Eq. 4-9), sparse formulation
# ----------------------------------------------------------------------------
def affinity(n, nbr, d2, gamma):
    """A~ as an n x n sparse matrix: 1 on the diagonal, exp(-d2/gamma) at (i, nbr[i, s]) (Eq. 4, Eq. 8)."""
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [np.ones(n)]
    valid = nbr >= 0
    r = np.repeat(np.arange(n), nbr.shape[1]).reshape(nbr.shape)[valid]
    rows.append(r)
    cols.append(nbr[valid])
    vals.append(np.exp(-d2[valid] / gamma))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n), dtype=np.float64)


def degrees(At):
    """Eq. 5: D_r(i,i) = sum_j A~_ij and D_c(j,j) = sum_i A~_ij (returned as vectors)."""
    Dr = np.asarray(At.sum(axis=1)).ravel()
    Dc = np.asarray(At.sum(axis=0)).ravel()
    return Dr, Dc


def propagation_operator(At, symmetric=True):
    """The propagation matrix applied to X.

    symmetric: A = (A~ + A~^T)/2 (Eq. 7), D(i,i) = sum_j A_ij, M = D^{-1/2} A D^{-1/2} (Eq. 2).
    otherwise: M = D_r^{-1/2} A~ D_c^{-1/2} (Eq. 6).
    """
    if symmetric:
        A = (At + At.T) * 0.5
        D = np.asarray(A.sum(axis=1)).ravel()
        s = sp.diags(1.0 / np.sqrt(D))
        return (s @ A @ s).tocsr()
    Dr, Dc = degrees(At)
    return (sp.diags(1.0 / np.sqrt(Dr)) @ At @ sp.diags(1.0 / np.sqrt(Dc))).tocsr()


def build_graph(X, k, gamma, cam=None, cross_camera=False, symmetric=True, alpha=1.0,
                nbr=None, nbr_cr=None):
    """One graph construction step on the current features X (Sec. III-B/C).

    Returns a dict with the kNN sets, their float64 squared distances, A~ (and A~^cr)
    and the mixed operator M_mix = alpha*M + (1-alpha)*M^cr of Eq. 9 (M_mix = M when
    the cross-camera graph is off). If ``nbr`` / ``nbr_cr`` are given, those
    neighbour sets are used instead of searching (their distances are recomputed here).
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    out = {}
    if nbr is None:
        nbr, d2 = knn(X, k, cam)
    else:
        nbr = np.asarray(nbr, dtype=np.int64)
        d2 = _edge_d2(X, nbr)
    out["nbr"], out["d2"] = nbr, d2
    out["At"] = affinity(n, nbr, d2, gamma)
    M = propagation_operator(out["At"], symmetric)
    if cross_camera:
        if nbr_cr is None:
            nbr_cr, d2c = knn(X, k, cam, cross_camera=True)
        else:
            nbr_cr = np.asarray(nbr_cr, dtype=np.int64)
            d2c = _edge_d2(X, nbr_cr)
        out["nbr_cr"], out["d2_cr"] = nbr_cr, d2c
        out["At_cr"] = affinity(n, nbr_cr, d2c, gamma)
        Mc = propagation_operator(out["At_cr"], symmetric)
        out["M"] = (alpha * M + (1.0 - alpha) * Mc).tocsr()
    else:
        out["M"] = M
    return out


def _edge_d2(X, nbr):
    d2 = np.full(nbr.shape, np.inf)
    for i in range(nbr.shape[0]):
        v = nbr[i] >= 0
        diff = X[nbr[i, v]] - X[i][None, :]
        d2[i, v] = np.sum(diff * diff, axis=1)
    return d2


def propagate(X, M):
    """One layer: X_t = normalise(M X_{t-1}) (Eq. 2 / Eq. 9, then the row L2 normalisation)."""
    return l2_normalize(M @ np.asarray(X, dtype=np.float64))


def gcr_layer(X, k, gamma, cam=None, cross_camera=False, symmetric=True, alpha=1.0):
    """G(X): rebuild the graph(s) from X, then propagate once (Eq. 3 step)."""
    g = build_graph(X, k, gamma, cam, cross_camera, symmetric, alpha)
    return propagate(X, g["M"]), g


def gcr(X0, k, gamma, T, cam=None, cross_camera=False, symmetric=True, alpha=1.0):
    """Full GCR feature update: X_0 = normalise(input), X_t = G(X_{t-1}) for t = 1..T (Eq. 3)."""
    X = l2_normalize(X0)
    for _ in range(T):
        X, _g = gcr_layer(X, k, gamma, cam, cross_camera, symmetric, alpha)
    return X


# ----------------------------------------------------------------------------
# re-ranking (Sec. III-A): distances on the updated features, then a stable sort
# ----------------------------------------------------------------------------
def rerank(Xq, Xg, topk=0):
    """Per query: gallery indices sorted by ascending ||x_q - x_g||^2 (ties -> smaller index).

    Returns (idx int64 [nq, K], dist float64 [nq, K]); K = ng when topk == 0.
    """
    D = sq_dist(Xq, Xg)
    K = D.shape[1] if topk in (0, None) else min(int(topk), D.shape[1])
    idx = np.argsort(D, axis=1, kind="stable")[:, :K]
    return idx, np.take_along_axis(D, idx, axis=1)


# ----------------------------------------------------------------------------
# dense formulation (explicit n x n matrices) -- a second, independent spelling of
# Eq. 4-7 used on small inputs to cross-check the sparse one
# ----------------------------------------------------------------------------
def affinity_dense(X, nbr, gamma):
    """Dense A~ (Eq. 4): loops over the neighbour lists, distances by the difference formula."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    At = np.zeros((n, n))
    for i in range(n):
        At[i, i] = 1.0
        for j in nbr[i]:
            if j < 0:
                continue
            diff = X[i] - X[j]
            At[i, j] = np.exp(-np.dot(diff, diff) / gamma)
    return At


def propagation_operator_dense(At, symmetric=True):
    """Dense Eq. 6 / Eq. 7 operator built from explicit degree vectors."""
    At = np.asarray(At, dtype=np.float64)
    if symmetric:
        A = 0.5 * (At + At.T)
        d = A.sum(axis=1)
        return A / np.sqrt(np.outer(d, d))
    dr = At.sum(axis=1)
    dc = At.sum(axis=0)
    return At / np.sqrt(np.outer(dr, dc))

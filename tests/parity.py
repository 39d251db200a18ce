"""Comparison helpers for the GPU-vs-oracle parity tests.

kNN sets must be identical except where the oracle's own FP64 distances tie at the k-th
neighbour (gap below 1e-9): such swaps are certified ties.
"""
import numpy as np

import oracle

TIE_TOL = 1e-9


def row_d2(X64, i, js):
    diff = X64[np.asarray(js, dtype=np.int64)] - X64[i][None, :]
    return np.sum(diff * diff, axis=1)


def compare_knn(X64, rows, gpu_nbr, k, cam=None, cross=False):
    """Returns dict(rows, mismatched, certified_ties, worst_gap) for the given rows.

    gpu_nbr[t] is the GPU's neighbour list of rows[t] (-1 padded).
    """
    rows = np.asarray(rows)
    o_idx, o_d2 = oracle.knn_rows(X64, rows, k, cam, cross)
    mism, ties, worst = 0, 0, 0.0
    for t, r in enumerate(rows):
        g = set(int(j) for j in gpu_nbr[t] if j >= 0)
        o = set(int(j) for j in o_idx[t] if j >= 0)
        if g == o:
            continue
        valid = o_d2[t][np.isfinite(o_d2[t])]
        if len(g) != len(o) or valid.size == 0:
            mism += 1
            continue
        dk = valid[-1]
        diff = sorted(g ^ o)
        gaps = np.abs(row_d2(X64, r, diff) - dk)
        worst = max(worst, float(gaps.max()))
        if np.all(gaps < TIE_TOL):
            ties += 1
        else:
            mism += 1
    return dict(rows=len(rows), mismatched=mism, certified_ties=ties, worst_gap=worst)


def dense_from_csr(rowptr, length, col, val, n):
    M = np.zeros((n, n))
    for i in range(n):
        b = rowptr[i]
        for e in range(b, b + length[i]):
            M[i, col[e]] += val[e]
    return M


def ranking_errors(X64q, X64g, idx, dist):
    """Max |dist - FP64 distance| and the worst order violation along the returned ranking."""
    D = oracle.sq_dist(X64q, X64g)
    dq = np.take_along_axis(D, idx.astype(np.int64), axis=1)
    err = float(np.max(np.abs(dist.astype(np.float64) - dq)))
    viol = float(np.max(np.maximum(0.0, dq[:, :-1] - dq[:, 1:]))) if dq.shape[1] > 1 else 0.0
    return err, viol

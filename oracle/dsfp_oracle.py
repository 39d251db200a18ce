"""Plain FP64 oracle for DSFP, the decentralized and synchronous feature propagation of
GCR (Algorithm 1, Sec. III-B; "GCR_Local" in Sec. IV-F's timing table).

Test infrastructure, not product code: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline arm of ``bench.py`` use it. It shares no code with the CUDA path.
It follows Algorithm 1 step by step, for one image at a time, in float64:

1. N_i = the k nearest samples of i on the given (normalised) features, i excluded,
   ties to the smaller index (the same search as the global method, Eq. 4).
2. The local node set is N_i together with i.
3. The local similarity matrix over every pair (u, v) of that set:
   A^i_uv = exp(-||x_u - x_v||^2 / gamma), written with the explicit differences
   (so A^i_uu = 1 and A^i is symmetric).
4. The local features X^i_0: the rows of the local node set.
5. The local degrees D^i(u, u) = sum_v A^i_uv.
6. T times: X^i_{t+1} = (D^i)^{-1/2} A^i (D^i)^{-1/2} X^i_t.

Readings where the paper is silent or garbled (each one is listed with its reason in the
design notes of the repository):

a. The output feature of image i is the row of i in its own X^i_T; every image is
   updated from its own local graph only ("renew features for each image").
b. The degree of step 5 is printed with a garbled index (D^i(i,i) summed over j); it is
   read as the row sum of A^i for every local node u.
c. The local graph is built once, from the input features, and kept for the T
   iterations (step 3 precedes the loop; unlike the global method's Algorithm 2, nothing
   rebuilds it).
d. As in the global method, rows are L2-normalised on input and after every iteration
   (a row of norm 0 stays 0).
e. Algorithm 1 is stated for the plain graph: there is no cross-camera form.
"""
from __future__ import annotations

import numpy as np

from .gcr_oracle import knn, l2_normalize

__all__ = ["dsfp_local", "dsfp"]


def dsfp_local(X, i, nbr_i, gamma, T):
    """Steps 2-6 of Algorithm 1 for image i: returns the row of i in X^i_T (float64).

    X: the normalised features (all rows); nbr_i: N_i (entries < 0 are absent neighbours).
    """
    X = np.asarray(X, dtype=np.float64)
    local = [int(i)] + [int(j) for j in nbr_i if j >= 0]        # step 2: N_i with i first
    Xl = X[local].copy()                                         # step 4
    m = len(local)
    A = np.empty((m, m), dtype=np.float64)                       # step 3
    for u in range(m):
        for v in range(m):
            diff = Xl[u] - Xl[v]
            A[u, v] = np.exp(-np.dot(diff, diff) / gamma)
    D = A.sum(axis=1)                                            # step 5
    s = 1.0 / np.sqrt(D)
    M = s[:, None] * A * s[None, :]
    for _ in range(T):                                           # step 6, then reading d
        Xl = l2_normalize(M @ Xl)
    return Xl[0]


def dsfp(X0, k, gamma, T, nbr=None):
    """Algorithm 1 for every image: X_0 = normalise(input), N_i by the exact kNN search
    of X_0 (step 1) unless ``nbr`` is given, then each image's local propagation.
    Returns (X_T float64 [n, d], nbr int64 [n, k])."""
    X = l2_normalize(X0)
    if nbr is None:
        nbr, _d2 = knn(X, k)
    nbr = np.asarray(nbr, dtype=np.int64)
    out = np.empty_like(X)
    for i in range(X.shape[0]):
        out[i] = dsfp_local(X, i, nbr[i], gamma, T)
    return out, nbr

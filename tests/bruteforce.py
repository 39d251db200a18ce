"""Pure-Python brute force of one GCR layer, for tiny inputs only.

Written from the paper's definitions with plain loops and lists (no numpy), so that
it shares no code and no library routine with the oracle it pins:
Eq. 4 (weights of the k nearest samples, self weight 1), Eq. 5 (row / column
degrees), Eq. 6 / Eq. 7 (asymmetric / symmetric operator), Eq. 8-9 (cross-camera
graph and the alpha mix), then the row L2 normalisation.
"""
import math


def sqd(a, b):
    return sum((x - y) * (x - y) for x, y in zip(a, b))


def knn_lists(X, k, cam=None, cross=False):
    """N_i by repeated extraction of the nearest remaining sample (ties -> smaller index)."""
    n = len(X)
    out = []
    for i in range(n):
        elig = [j for j in range(n) if j != i and (not cross or cam[j] != cam[i])]
        chosen = []
        while len(chosen) < k and elig:
            best = None
            for j in elig:
                dj = sqd(X[i], X[j])
                if best is None or dj < best[0] or (dj == best[0] and j < best[1]):
                    best = (dj, j)
            chosen.append(best[1])
            elig.remove(best[1])
        out.append(chosen)
    return out


def affinity(X, lists, gamma):
    n = len(X)
    A = [[0.0] * n for _ in range(n)]
    for i in range(n):
        A[i][i] = 1.0
        for j in lists[i]:
            A[i][j] = math.exp(-sqd(X[i], X[j]) / gamma)
    return A


def operator(At, symmetric):
    n = len(At)
    if symmetric:
        A = [[(At[i][j] + At[j][i]) / 2.0 for j in range(n)] for i in range(n)]
        D = [sum(A[i]) for i in range(n)]
        return [[A[i][j] / math.sqrt(D[i] * D[j]) for j in range(n)] for i in range(n)]
    Dr = [sum(At[i]) for i in range(n)]
    Dc = [sum(At[i][j] for i in range(n)) for j in range(n)]
    return [[At[i][j] / math.sqrt(Dr[i] * Dc[j]) for j in range(n)] for i in range(n)]


def normalize(v):
    s = math.sqrt(sum(x * x for x in v))
    return [x / s for x in v] if s > 0 else [0.0 for _ in v]


def layer(X, k, gamma, cam=None, cross=False, symmetric=True, alpha=1.0):
    n, d = len(X), len(X[0])
    M = operator(affinity(X, knn_lists(X, k), gamma), symmetric)
    if cross:
        Mc = operator(affinity(X, knn_lists(X, k, cam, True), gamma), symmetric)
        M = [[alpha * M[i][j] + (1 - alpha) * Mc[i][j] for j in range(n)] for i in range(n)]
    Y = [[sum(M[i][j] * X[j][c] for j in range(n)) for c in range(d)] for i in range(n)]
    return [normalize(y) for y in Y]


def gcr(X0, k, gamma, T, cam=None, cross=False, symmetric=True, alpha=1.0):
    X = [normalize(list(map(float, r))) for r in X0]
    for _ in range(T):
        X = layer(X, k, gamma, cam, cross, symmetric, alpha)
    return X


def rerank(Q, G):
    """Per query: gallery indices by ascending squared distance, ties by index."""
    out = []
    for q in Q:
        keyed = sorted(range(len(G)), key=lambda g: (sqd(q, G[g]), g))
        out.append(keyed)
    return out


def serve(Q, G0, k, gamma, T, K, symmetric=True):
    """Serving form: gallery layers by offline GCR on the gallery alone, then each query's
    row of the operator against the frozen layer (no query-query edges), then top-K."""
    G = [normalize(list(map(float, r))) for r in G0]
    ng = len(G)
    layers, degs = [G], []
    for _ in range(T):
        lists = knn_lists(G, k)
        At = affinity(G, lists, gamma)
        Dr = [sum(At[i]) for i in range(ng)]
        Dc = [sum(At[i][j] for i in range(ng)) for j in range(ng)]
        degs.append([(Dr[j] + Dc[j]) / 2.0 for j in range(ng)] if symmetric else Dc)
        M = operator(At, symmetric)
        d = len(G[0])
        G = [normalize([sum(M[i][j] * G[j][c] for j in range(ng)) for c in range(d)]) for i in range(ng)]
        layers.append(G)
    out = []
    for q in Q:
        x = normalize(list(map(float, q)))
        for t in range(T):
            L = layers[t]
            order = sorted(range(ng), key=lambda j: (sqd(x, L[j]), j))[:k]
            w = [math.exp(-sqd(x, L[j]) / gamma) for j in order]
            d = len(x)
            if symmetric:
                Dq = (1.0 + sum(w) + 1.0) / 2.0
                y = [x[c] / Dq + sum(w[s] / 2.0 * L[j][c] / math.sqrt(Dq * degs[t][j]) for s, j in enumerate(order))
                     for c in range(d)]
            else:
                r = 1.0 + sum(w)
                y = [x[c] / math.sqrt(r) + sum(w[s] * L[j][c] / math.sqrt(r * degs[t][j]) for s, j in enumerate(order))
                     for c in range(d)]
            x = normalize(y)
        ranked = sorted(range(ng), key=lambda g: (sqd(x, layers[T][g]), g))[:K]
        out.append(ranked)
    return out

"""Planted mistakes in the FP64 oracle: each one must fail at least one pin (CPU only).

Every mutant edits one oracle function's source in a plausible way (a dropped term, a wrong
sign, a transposed operand, a wrong index or axis, ties broken the other way) and runs all
pins of the matching test module against it. The unmutated oracle passes them all; a mutant
that every pin let through would be a mistake the pins cannot see.
"""
import pytest

import oracle.dsfp_oracle as dsfp_o
import oracle.eval_oracle as eval_o
import oracle.gcr_oracle as gcr_o
import oracle.pvg_oracle as pvg_o
import oracle.serve_oracle as serve_o
from tests import mutation
from tests import test_oracle_dsfp, test_oracle_eval, test_oracle_gcr, test_oracle_pvg, test_oracle_serve

# (module, function, text, replacement)
GCR = [
    # Sec. III-D: unit rows
    (gcr_o, "l2_normalize", "nrm = np.sqrt(np.sum(X * X, axis=1, keepdims=True))",
     "nrm = np.sum(X * X, axis=1, keepdims=True)"),
    # Eq. 4 distance, expanded form
    (gcr_o, "sq_dist", "return na + nb - 2.0 * (A @ B.T)", "return na + nb - (A @ B.T)"),
    (gcr_o, "sq_dist", "return na + nb - 2.0 * (A @ B.T)", "return na + nb + 2.0 * (A @ B.T)"),
    (gcr_o, "sq_dist_direct", "out[i] = np.sum(diff * diff, axis=1)", "out[i] = np.sum(np.abs(diff), axis=1)"),
    # N_i: i excluded, nearest first, ties to the smaller index, other cameras only (Eq. 8)
    (gcr_o, "knn_rows", "D[np.arange(r.shape[0]), r] = np.inf", "pass"),
    (gcr_o, "knn_rows", "cam[r][:, None] == cam[None, :]", "cam[r][:, None] != cam[None, :]"),
    (gcr_o, "knn_rows", "idx[s + t, :sel.shape[0]] = sel", "idx[t, :sel.shape[0]] = sel"),
    (gcr_o, "knn_rows", "D[np.arange(r.shape[0]), r] = np.inf", "D[np.arange(r.shape[0]), np.arange(r.shape[0])] = np.inf"),
    (gcr_o, "_select_row", "cand = np.nonzero(drow <= vk)[0]", "cand = np.nonzero(drow <= vk)[0][::-1]"),
    (gcr_o, "_select_row", 'order = np.argsort(drow[cand], kind="stable")',
     'order = np.argsort(-drow[cand], kind="stable")'),
    (gcr_o, "_select_row", "kk = min(k, m)", "kk = min(k, m - 1)"),
    # Eq. 4 weights and the self loop
    (gcr_o, "affinity", "vals.append(np.exp(-d2[valid] / gamma))", "vals.append(np.exp(d2[valid] / gamma))"),
    (gcr_o, "affinity", "vals.append(np.exp(-d2[valid] / gamma))", "vals.append(np.exp(-d2[valid] * gamma))"),
    (gcr_o, "affinity", "[np.ones(n)]", "[np.zeros(n)]"),
    (gcr_o, "affinity", "(np.concatenate(rows), np.concatenate(cols))",
     "(np.concatenate(cols), np.concatenate(rows))"),
    # Eq. 5 degrees
    (gcr_o, "degrees", "Dr = np.asarray(At.sum(axis=1)).ravel()", "Dr = np.asarray(At.sum(axis=0)).ravel()"),
    (gcr_o, "degrees", "Dc = np.asarray(At.sum(axis=0)).ravel()", "Dc = np.asarray(At.sum(axis=1)).ravel()"),
    # Eq. 6 / Eq. 7 operators
    (gcr_o, "propagation_operator", "A = (At + At.T) * 0.5", "A = At"),
    (gcr_o, "propagation_operator", "s = sp.diags(1.0 / np.sqrt(D))", "s = sp.diags(1.0 / D)"),
    (gcr_o, "propagation_operator", "D = np.asarray(A.sum(axis=1)).ravel()",
     "D = np.asarray(At.sum(axis=1)).ravel()"),
    (gcr_o, "propagation_operator", "sp.diags(1.0 / np.sqrt(Dr)) @ At @ sp.diags(1.0 / np.sqrt(Dc))",
     "sp.diags(1.0 / np.sqrt(Dc)) @ At @ sp.diags(1.0 / np.sqrt(Dr))"),
    # Eq. 9 mix and the cross-camera search
    (gcr_o, "build_graph", "(alpha * M + (1.0 - alpha) * Mc)", "((1.0 - alpha) * M + alpha * Mc)"),
    (gcr_o, "build_graph", "nbr_cr, d2c = knn(X, k, cam, cross_camera=True)", "nbr_cr, d2c = knn(X, k, cam)"),
    (gcr_o, "_edge_d2", "diff = X[nbr[i, v]] - X[i][None, :]", "diff = X[nbr[i, v]] + X[i][None, :]"),
    # Eq. 2-3 propagation and the layer loop
    (gcr_o, "propagate", "l2_normalize(M @ np.asarray(X, dtype=np.float64))",
     "l2_normalize(M.T @ np.asarray(X, dtype=np.float64))"),
    (gcr_o, "propagate", "l2_normalize(M @ np.asarray(X, dtype=np.float64))", "M @ np.asarray(X, dtype=np.float64)"),
    (gcr_o, "gcr", "X = l2_normalize(X0)", "X = np.asarray(X0, dtype=np.float64)"),
    (gcr_o, "gcr_layer", 'return propagate(X, g["M"]), g', 'return propagate(X, g["At"]), g'),
    # Sec. III-A ranking
    (gcr_o, "rerank", 'idx = np.argsort(D, axis=1, kind="stable")[:, :K]',
     'idx = np.argsort(D, axis=1, kind="stable")[:, ::-1][:, :K]'),
    (gcr_o, "rerank", 'idx = np.argsort(D, axis=1, kind="stable")[:, :K]',
     'idx = np.argsort(D[:, ::-1], axis=1, kind="stable")[:, :K]'),
    # the dense spelling used as a cross-check
    (gcr_o, "affinity_dense", "At[i, i] = 1.0", "At[i, i] = 0.0"),
    (gcr_o, "propagation_operator_dense", "A = 0.5 * (At + At.T)", "A = 0.5 * (At + At)"),
]

PVG = [
    # Eq. 10
    (pvg_o, "mean_profiles", "out[c] = F[trk_off[c]:trk_off[c + 1]].mean(axis=0)",
     "out[c] = F[trk_off[c]:trk_off[c + 1]].sum(axis=0)"),
    (pvg_o, "mean_profiles", "out[c] = F[trk_off[c]:trk_off[c + 1]].mean(axis=0)",
     "out[c] = F[trk_off[c]:trk_off[c + 1] + 1].mean(axis=0)"),
    # Eq. 17: normalised frames, the camera's mean, lambda n I, the sign of mu_c - mu
    (pvg_o, "pvg_profiles", "Xf = l2_normalize(frames)", "Xf = np.asarray(frames, dtype=np.float64)"),
    (pvg_o, "pvg_profiles", "mu_s = Xs.mean(axis=0)", "mu_s = Xf.mean(axis=0)"),
    (pvg_o, "pvg_profiles", "mu_s = Xs.mean(axis=0)", "mu_s = mu_c[members].mean(axis=0)"),
    (pvg_o, "pvg_profiles", "lam * n_s * np.eye(d)", "lam * np.eye(d)"),
    (pvg_o, "pvg_profiles", "gram_scale * (Xs.T @ Xs)", "gram_scale * (Xs.T @ Xs) / n_s"),
    (pvg_o, "pvg_profiles", "rhs = (mu_c[members] - mu_s[None, :]).T", "rhs = (mu_s[None, :] - mu_c[members]).T"),
    (pvg_o, "pvg_profiles", "W[members[0]] = mu_c[members[0]]", "W[members[0]] = 0.0"),
    (pvg_o, "pvg_profiles", "if members.shape[0] == 1:", "if False:"),
    # Algorithm 2 on the profiles
    (pvg_o, "gcrv", "cross_camera=True", "cross_camera=False"),
    (pvg_o, "gcrv", "symmetric=symmetric, alpha=alpha", "symmetric=symmetric, alpha=1.0 - alpha"),
]

SERVE = [
    # gallery layers and frozen degrees
    (serve_o, "gallery_layers", "0.5 * (Dr + Dc) if symmetric else Dc", "Dr if symmetric else Dc"),
    (serve_o, "gallery_layers", "0.5 * (Dr + Dc) if symmetric else Dc", "0.5 * (Dr + Dc) if symmetric else Dr"),
    (serve_o, "gallery_layers", "layers, degs = [G], []", "layers, degs = [Xg], []"),
    # the query's row of Eq. 7 / Eq. 6
    (serve_o, "_query_step", 'idx = np.argsort(D, kind="stable")[:k]', 'idx = np.argsort(D, kind="stable")[:k + 1]'),
    (serve_o, "_query_step", "w = np.exp(-D[idx] / gamma)", "w = np.exp(D[idx] / gamma)"),
    (serve_o, "_query_step", "Dq = 0.5 * (1.0 + w.sum() + 1.0)", "Dq = 0.5 * (1.0 + w.sum())"),
    (serve_o, "_query_step", "Dq = 0.5 * (1.0 + w.sum() + 1.0)", "Dq = 1.0 + w.sum()"),
    (serve_o, "_query_step", "((0.5 * w) / np.sqrt(Dq * deg[idx]))", "(w / np.sqrt(Dq * deg[idx]))"),
    (serve_o, "_query_step", "((0.5 * w) / np.sqrt(Dq * deg[idx]))", "((0.5 * w) / np.sqrt(Dq))"),
    (serve_o, "_query_step", "Y[i] = xq[i] / Dq +", "Y[i] = xq[i] / np.sqrt(Dq) +"),
    (serve_o, "_query_step", "Y[i] = xq[i] / np.sqrt(r) +", "Y[i] = xq[i] / r +"),
    (serve_o, "_query_step", "(w / np.sqrt(r * deg[idx])) @ G[idx]", "(w / np.sqrt(r)) @ G[idx]"),
    (serve_o, "_query_step", "return l2_normalize(Y)", "return Y"),
    # the layer loop and the final ranking
    (serve_o, "serve_queries", "xq = _query_step(xq, layers[t], degs[t],", "xq = _query_step(xq, layers[t + 1], degs[t],"),
    (serve_o, "serve_queries", "D = sq_dist(xq, layers[T])", "D = sq_dist(xq, layers[T - 1])"),
    (serve_o, "serve_queries", "xq = l2_normalize(Q)", "xq = np.asarray(Q, dtype=np.float64)"),
]

DSFP = [
    # Algorithm 1: local node set, local weights, degrees, T normalised steps, the row of i
    (dsfp_o, "dsfp_local", "local = [int(i)] + [int(j) for j in nbr_i if j >= 0]",
     "local = [int(j) for j in nbr_i if j >= 0] + [int(i)]"),
    (dsfp_o, "dsfp_local", "A[u, v] = np.exp(-np.dot(diff, diff) / gamma)",
     "A[u, v] = np.exp(-np.dot(diff, diff) / gamma) if u != v else 0.0"),
    (dsfp_o, "dsfp_local", "A[u, v] = np.exp(-np.dot(diff, diff) / gamma)",
     "A[u, v] = np.exp(np.dot(diff, diff) / gamma)"),
    (dsfp_o, "dsfp_local", "D = A.sum(axis=1)", "D = A.sum(axis=1) ** 2"),
    (dsfp_o, "dsfp_local", "s = 1.0 / np.sqrt(D)", "s = 1.0 / D"),
    (dsfp_o, "dsfp_local", "Xl = l2_normalize(M @ Xl)", "Xl = M @ Xl"),
    (dsfp_o, "dsfp_local", "return Xl[0]", "return l2_normalize(Xl)[-1]"),
    (dsfp_o, "dsfp", "X = l2_normalize(X0)", "X = np.asarray(X0, dtype=np.float64)"),
    (dsfp_o, "dsfp", "out[i] = dsfp_local(X, i, nbr[i], gamma, T)", "out[i] = dsfp_local(X, i, nbr[i], gamma, max(T - 1, 0))"),
]

EVAL = [
    # relevance, junk removal, the precision at each hit, missing items, the first hit
    (eval_o, "query_ap", "if protocol == 1 and same and g_cam[g] == q_cam:", "if False:"),
    (eval_o, "query_ap", "if g_label[g] == q_label and not (protocol == 1 and g_cam[g] == q_cam):",
     "if g_label[g] == q_label:"),
    (eval_o, "query_ap", "s += hits / (pos + 1)", "s += hits / pos if pos else 1.0"),
    (eval_o, "query_ap", "s += hits / (pos + 1)", "s += 1.0 / (pos + 1)"),
    (eval_o, "query_ap", "return s / R, first", "return s / max(hits, 1), first"),
    (eval_o, "query_ap", "        pos += 1\n", "        if same:\n            pos += 1\n"),
    (eval_o, "query_ap", "if q_label < 0:", "if q_label < -1:"),
    (eval_o, "query_ap", "first = pos", "first = pos + 1"),
    (eval_o, "summarise", "(first[ok] >= 0) & (first[ok] < k)", "(first[ok] >= 0) & (first[ok] <= k)"),
]

TABLES = [(GCR, test_oracle_gcr), (PVG, test_oracle_pvg), (SERVE, test_oracle_serve),
          (DSFP, test_oracle_dsfp), (EVAL, test_oracle_eval)]


def _id(case):
    (module, fname, old, _new), _tests = case
    return f"{module.__name__.split('.')[-1]}.{fname}:{old[:40]}"


@pytest.mark.parametrize("tests_module", [m for _t, m in TABLES], ids=lambda m: m.__name__.split(".")[-1])
def test_unmutated_oracle_passes_every_pin(tests_module):
    assert mutation.failing_pins(mutation.pin_cases(tests_module), []) == []


@pytest.mark.parametrize("case", [(row, mod) for table, mod in TABLES for row in table], ids=_id)
def test_planted_mistake_fails_a_pin(monkeypatch, case):
    (module, fname, old, new), tests_module = case
    mutation.plant(monkeypatch, module, fname, old, new)
    skipped = []
    failed = mutation.failing_pins(mutation.pin_cases(tests_module), skipped)
    if not failed and skipped:
        pytest.skip(f"pins skipped here: {skipped}")
    assert failed, f"no pin catches {fname}: {old!r} -> {new!r}"

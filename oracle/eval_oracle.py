"""Plain oracle for the retrieval-quality evaluation of re-ranked lists (mean average precision
and the CMC / Rank-k accuracy that Sec. IV reports for every method), on labelled synthetic
data.

Test infrastructure, not product code: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU arms of ``bench.py`` use it. It shares no code with the CUDA path.

Definitions (the usual ones for person re-identification; the paper reports mAP and Rank-1
without restating them, so these are readings):

* A gallery item is *relevant* to a query when both carry the same label and the label is
  non-negative (label -1 marks a distractor, relevant to no query).
* Protocol 1 (cross-camera, as on Market-1501 and MARS): a gallery item with the query's label
  and the query's camera is *junk*: it is removed from the list before scoring (it counts
  neither as a hit nor as a miss). Protocol 0 removes nothing.
* On the list with junk removed, with the relevant items at 0-based positions
  p_1 < p_2 < ... < p_R (R = the number of relevant items in the whole gallery),
  AP = (1/R) sum_i i / (p_i + 1), the precision at each hit averaged over all relevant items
  (relevant items missing from a truncated list contribute 0). The first hit is p_1 (or -1).
  A query with R = 0 has no AP (reported as NaN) and no first hit.
* mAP = the mean AP over queries with R > 0; Rank-k = the fraction of those queries whose
  first hit is at a position < k.
"""
from __future__ import annotations

import numpy as np

__all__ = ["query_ap", "evaluate", "summarise"]


def query_ap(ranked, q_label, q_cam, g_label, g_cam, protocol):
    """AP and first-hit position of one query's ranked gallery indices (a Python loop)."""
    if q_label < 0:
        return float("nan"), -1
    R = 0
    for g in range(len(g_label)):
        if g_label[g] == q_label and not (protocol == 1 and g_cam[g] == q_cam):
            R += 1
    if R == 0:
        return float("nan"), -1
    pos = 0
    hits = 0
    s = 0.0
    first = -1
    for g in ranked:
        g = int(g)
        if g < 0:
            continue
        same = g_label[g] == q_label
        if protocol == 1 and same and g_cam[g] == q_cam:
            continue                       # junk: removed from the list
        if same:
            hits += 1
            s += hits / (pos + 1)
            if first < 0:
                first = pos
        pos += 1
    return s / R, first


def evaluate(idx, q_label, g_label, q_cam=None, g_cam=None, protocol=0):
    """Per-query AP (float64, NaN without relevant items) and first-hit position (int64)."""
    idx = np.asarray(idx)
    nq = idx.shape[0]
    q_cam = np.zeros(nq, np.int64) if q_cam is None else np.asarray(q_cam)
    g_cam = np.zeros(len(g_label), np.int64) if g_cam is None else np.asarray(g_cam)
    ap = np.empty(nq, np.float64)
    first = np.empty(nq, np.int64)
    for q in range(nq):
        ap[q], first[q] = query_ap(idx[q], int(q_label[q]), int(q_cam[q]), g_label, g_cam, protocol)
    return ap, first


def summarise(ap, first, ranks=(1, 5, 10)):
    """mAP and Rank-k over the queries that have relevant items."""
    ok = ~np.isnan(ap)
    out = {"mAP": float(np.mean(ap[ok])) if ok.any() else float("nan"), "queries": int(ok.sum())}
    for k in ranks:
        out[f"rank{k}"] = float(np.mean((first[ok] >= 0) & (first[ok] < k))) if ok.any() else float("nan")
    return out

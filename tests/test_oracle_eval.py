"""Pins for the retrieval-quality oracle (mAP / Rank-k; CPU only): hand-worked lists,
the junk rule, truncated lists, and an independent library implementation of average
precision (scikit-learn) on random rankings."""
import numpy as np
import pytest

import oracle


def test_hand_worked_lists():
    g_label = np.array([5, 7, 5, 5, 9, 7])
    # query label 5: relevant gallery items 0, 2, 3 (R = 3)
    ap, first = oracle.query_ap([4, 0, 1, 2, 5, 3], 5, 0, g_label, np.zeros(6), 0)
    # hits at positions 1, 3, 5: (1/2 + 2/4 + 3/6) / 3 = 0.5
    assert ap == pytest.approx(0.5, abs=1e-15) and first == 1
    ap, first = oracle.query_ap([0, 2, 3, 1, 4, 5], 5, 0, g_label, np.zeros(6), 0)
    assert ap == 1.0 and first == 0
    ap, first = oracle.query_ap([1, 4, 5, 0, 2, 3], 5, 0, g_label, np.zeros(6), 0)
    # hits at 3, 4, 5: (1/4 + 2/5 + 3/6) / 3
    assert ap == pytest.approx((0.25 + 0.4 + 0.5) / 3, abs=1e-15) and first == 3


def test_junk_is_removed_before_scoring():
    g_label = np.array([5, 7, 5, 5])
    g_cam = np.array([0, 0, 1, 2])
    # protocol 1, query label 5 on camera 0: item 0 (label 5, camera 0) is junk; R = 2
    ap, first = oracle.query_ap([0, 1, 2, 3], 5, 0, g_label, g_cam, 1)
    # list without junk: 1, 2, 3 -> hits at positions 1, 2: (1/2 + 2/3) / 2
    assert ap == pytest.approx((0.5 + 2 / 3) / 2, abs=1e-15) and first == 1
    ap0, first0 = oracle.query_ap([0, 1, 2, 3], 5, 0, g_label, g_cam, 0)
    assert ap0 == pytest.approx((1 + 2 / 3 + 3 / 4) / 3, abs=1e-15) and first0 == 0


def test_no_relevant_items_and_distractor_queries():
    g_label = np.array([1, 2, -1, -1])
    ap, first = oracle.query_ap([0, 1, 2, 3], 3, 0, g_label, np.zeros(4), 0)
    assert np.isnan(ap) and first == -1
    ap, first = oracle.query_ap([2, 3, 0, 1], -1, 0, g_label, np.zeros(4), 0)   # a distractor query
    assert np.isnan(ap) and first == -1


def test_truncated_list_counts_missing_relevant_items_as_zero():
    g_label = np.array([5, 5, 5, 7, 7])
    ap, first = oracle.query_ap([3, 0], 5, 0, g_label, np.zeros(5), 0)
    assert ap == pytest.approx((1 / 2) / 3, abs=1e-15) and first == 1


def test_matches_scikit_learn_average_precision():
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(0)
    ng, nq = 60, 40
    g_label = rng.integers(0, 8, ng)
    q_label = rng.integers(0, 9, nq)           # label 8 has no gallery items
    scores = rng.standard_normal((nq, ng))
    idx = np.argsort(-scores, axis=1, kind="stable")
    ap, first = oracle.evaluate(idx, q_label, g_label)
    for q in range(nq):
        y = (g_label == q_label[q]).astype(int)
        if y.sum() == 0:
            assert np.isnan(ap[q]) and first[q] == -1
            continue
        assert ap[q] == pytest.approx(skm.average_precision_score(y, scores[q]), abs=1e-12)
        assert first[q] == int(np.argmax(y[idx[q]] == 1))
    s = oracle.summarise(ap, first)
    ok = ~np.isnan(ap)
    assert s["queries"] == ok.sum() and s["rank1"] == pytest.approx(np.mean(first[ok] == 0))


def test_perfect_ranking_scores_one():
    g_label = np.repeat(np.arange(5), 4)
    q_label = np.arange(5)
    idx = np.array([np.argsort(g_label != q, kind="stable") for q in q_label])
    ap, first = oracle.evaluate(idx, q_label, g_label)
    assert np.all(ap == 1.0) and np.all(first == 0)


def test_rank_k_and_map_by_hand():
    """Rank-k counts the queries whose first hit lies before position k; queries without
    relevant items (AP NaN) are left out of both figures."""
    ap = np.array([1.0, 0.5, float("nan"), 0.25, 0.0])
    first = np.array([0, 4, -1, 5, -1])
    s = oracle.summarise(ap, first, ranks=(1, 5, 6))
    assert s["queries"] == 4
    assert s["mAP"] == pytest.approx((1.0 + 0.5 + 0.25 + 0.0) / 4, abs=1e-15)
    assert (s["rank1"], s["rank5"], s["rank6"]) == (0.25, 0.5, 0.75)

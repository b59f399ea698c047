"""Pins of the parity checker (oracle/compare.py:check_topk), which decides
every GPU parity test: it must accept the exact answer and answers that
differ only where the rule allows (ties within the tolerance at the k-th
score, FP32 rounding of the scores), and reject each plausible mistake of a
top-k kernel.  Hand-built score vectors; no GPU.
"""
import numpy as np
import pytest

import oracle
from oracle.compare import RTOL, check_topk
from paper_2407_03618_gb300 import synth


def _exact(full, k):
    """The oracle's own answer: top k by (score desc, id asc), FP32 scores."""
    n = full.shape[0]
    order = np.lexsort((np.arange(n), -full))
    kp = min(k, n)
    ids = np.full(k, -1, np.int64)
    sc = np.full(k, -np.inf)
    ids[:kp] = order[:kp]
    sc[:kp] = full[order[:kp]].astype(np.float32)
    return ids, sc


# twelve documents with well separated scores, two exact ties (docs 4 and 9
# at 2.0, docs 6 and 7 at 0.5) and a Robertson-like negative score
FULL = np.array([3.0, 1.0, 5.0, 0.25, 2.0, 4.0, 0.5, 0.5, 1.5, 2.0, -0.75, 0.0])
ABS = np.abs(FULL) + 0.5  # sum_i |S(q_i, D)| >= |B(Q,D)|


def _expect_fail(ids, sc, full=FULL, ab=ABS, k=5, match=None):
    with pytest.raises(AssertionError, match=match):
        check_topk(np.asarray(ids), np.asarray(sc, np.float64), full, ab, k)


def test_accepts_exact_answer():
    for k in (1, 3, 5, 6, 12, 15):
        ids, sc = _exact(FULL, k)
        check_topk(ids, sc, FULL, ABS, k)


def test_accepts_scores_within_tolerance():
    ids, sc = _exact(FULL, 5)
    # 0.4 of the tolerance in either direction (ranks stay separated)
    tol = RTOL * np.maximum(np.abs(FULL[ids]), ABS[ids])
    check_topk(ids, sc + 0.4 * tol * np.array([1, -1, 1, 1, -1]), FULL, ABS, 5)


def test_rejects_score_off_by_2e5_relative():
    ids, sc = _exact(FULL, 5)
    sc = sc.copy()
    sc[1] = FULL[ids[1]] * (1 + 2e-5) + RTOL * ABS[ids[1]]  # beyond max(|B|, sum|S|) * 1e-5
    _expect_fail(ids, sc, match="score mismatch")


def test_rejects_swapped_id_in_strict_top():
    ids, sc = _exact(FULL, 5)  # [2, 5, 0, 4, 9]
    bad = ids.copy()
    bad[1] = 8  # doc 8 (1.5) in place of doc 5 (4.0), with doc 5's score
    _expect_fail(bad, sc, match="score mismatch")
    # ... and with doc 8's own score: the row is then unsorted, and doc 5 missing
    sc2 = sc.copy()
    sc2[1] = 1.5
    _expect_fail(bad, sc2)
    bad3, sc3 = ids.copy(), sc.copy()  # doc 8 last, the true 4.0 dropped, sorted
    bad3 = np.array([2, 0, 4, 9, 8])
    sc3 = np.array([5.0, 3.0, 2.0, 2.0, 1.5])
    _expect_fail(bad3, sc3, match="missing|below the k-th")


def test_rejects_missing_top_doc():
    # k = 4: the top four are 2 (5.0), 5 (4.0), 0 (3.0), 4 (2.0); doc 0 left
    # out, doc 9 (2.0, tied with the k-th) and doc 8 (1.5) in
    ids = np.array([2, 5, 4, 9])
    sc = np.array([5.0, 4.0, 2.0, 2.0])
    _expect_fail(ids, sc, k=4, match="missing")


def test_rejects_duplicate_id():
    ids, sc = _exact(FULL, 5)
    bad = ids.copy()
    bad[4] = bad[3]
    _expect_fail(bad, sc, match="duplicate")


def test_rejects_ascending_row():
    ids, sc = _exact(FULL, 5)
    _expect_fail(ids[::-1], sc[::-1], match="not sorted")


def test_rejects_equal_scores_with_higher_id_first():
    ids, sc = _exact(FULL, 5)  # ... 4 (2.0), 9 (2.0)
    assert list(ids[3:]) == [4, 9]
    bad = ids.copy()
    bad[3], bad[4] = 9, 4
    _expect_fail(bad, sc, match="doc id")


def test_rejects_wrong_padding():
    ids, sc = _exact(FULL, 15)  # 12 documents, 3 padding slots
    for fix in ("id0", "id_other", "score0", "score_nan"):
        i2, s2 = ids.copy(), sc.copy()
        if fix == "id0":
            i2[13] = 0
        elif fix == "id_other":
            i2[14] = 12
        elif fix == "score0":
            s2[12] = 0.0
        else:
            s2[14] = np.nan
        _expect_fail(i2, s2, k=15, match="padding")
    # a real document must not be replaced by padding either
    i3, s3 = ids.copy(), sc.copy()
    i3[11], s3[11] = -1, -np.inf
    _expect_fail(i3, s3, k=15)


def test_rejects_out_of_range_id():
    ids, sc = _exact(FULL, 5)
    bad = ids.copy()
    bad[0] = 12
    _expect_fail(bad, sc, match="out of range")


def test_tie_at_kth_score_either_doc():
    # k = 4: docs 4 and 9 tie exactly at 2.0 for the last slot; both answers pass
    check_topk(np.array([2, 5, 0, 4]), np.array([5.0, 4.0, 3.0, 2.0]), FULL, ABS, 4)
    check_topk(np.array([2, 5, 0, 9]), np.array([5.0, 4.0, 3.0, 2.0]), FULL, ABS, 4)


def test_near_tie_within_one_tolerance_passes_beyond_fails():
    # the 5th best is 1.0; a document 0.5 tolerance below it may replace it,
    # one 1.5 tolerances below may not (the looser 2 tol_k + tol_D rule of an
    # earlier checker accepted up to three tolerances)
    base = np.array([9.0, 8.0, 7.0, 6.0, 1.0, 0.0, 0.0])
    ab = np.abs(base)
    tol_k = RTOL * 1.0
    for delta, ok in ((0.5, True), (1.5, False), (2.5, False)):
        full = base.copy()
        full[5] = 1.0 - delta * tol_k
        ids = np.array([0, 1, 2, 3, 5])
        sc = full[ids].astype(np.float64)
        if ok:
            check_topk(ids, sc, full, ab, 5)
        else:
            _expect_fail(ids, sc, full=full, ab=ab, k=5, match="below the k-th")


def test_negative_and_zero_scores_rank():
    # Robertson: an untouched document (0) outranks a negative one
    full = np.array([-0.2, 0.0, 0.1])
    ab = np.array([0.2, 0.0, 0.1])
    check_topk(np.array([2, 1, 0]), np.array([0.1, 0.0, -0.2]), full, ab, 3)
    _expect_fail([2, 0, 1], [0.1, -0.2, 0.0], full=full, ab=ab, k=3)


def test_against_oracle_on_random_corpora():
    # the oracle's own ranking passes; a ranking one position off at a
    # separated boundary fails
    rng = np.random.default_rng(42)
    checked = 0
    for _ in range(60):
        c = synth.random_tiny_corpus(rng, max_docs=12, max_vocab=6, max_len=6)
        orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.LUCENE, 1.5, 0.75, 0.5)
        q = synth.random_queries(rng, c.vocab, 1, 4, min_len=1).query(0)
        full, ab = oracle.score_all(orc, q, with_abs=True)
        k = min(3, c.n_docs)
        ids, sc = _exact(full, k)
        check_topk(ids, sc, full, ab, k)
        order = np.lexsort((np.arange(full.shape[0]), -full))
        if full.shape[0] > k and full[order[k - 1]] - full[order[k]] > 1e-3 * (1 + abs(full).max()):
            bad = ids.copy()
            bad[k - 1] = order[k]
            s2 = sc.copy()
            s2[k - 1] = full[order[k]]
            _expect_fail(bad, s2, full=full, ab=ab, k=k)
            checked += 1
    assert checked >= 10


def test_list_checker_agrees_with_the_full_checker():
    """check_topk_with_list (the oracle's top-m list in place of its full
    score vector) accepts and rejects what check_topk does, on random
    non-negative score vectors with ties and on perturbed answers."""
    from oracle.compare import check_topk_with_list
    rng = np.random.default_rng(77)
    n_same = 0
    for trial in range(400):
        n = int(rng.integers(5, 60))
        full = np.round(rng.exponential(1.0, n), 2)  # ties
        k = int(rng.integers(1, 8))
        order = np.lexsort((np.arange(n), -full))
        m = min(n, k + 20)
        top_ids, top_sc = order[:m], full[order[:m]]
        ids, sc = _exact(full, k)
        mode = trial % 4
        if mode == 1 and min(k, n) >= 2:  # swap in a document from below
            ids = ids.copy()
            ids[-1] = order[min(n - 1, k + int(rng.integers(0, 5)))]
            sc = sc.copy()
            sc[-1] = full[ids[-1]]
        elif mode == 2:  # a score off
            sc = sc.copy()
            sc[0] *= 1 + 3e-5
        elif mode == 3 and min(k, n) >= 2:  # unsorted
            ids, sc = ids[::-1].copy(), sc[::-1].copy()
        try:
            check_topk(ids, sc, full, full, k)
            ok_full = True
        except AssertionError:
            ok_full = False
        try:
            check_topk_with_list(ids, sc, top_ids, top_sc, k, n)
            ok_list = True
        except AssertionError as e:
            ok_list = False
            if "too short" in str(e):
                continue
        assert ok_full == ok_list, (trial, mode, full, ids, sc)
        n_same += 1
    assert n_same > 300

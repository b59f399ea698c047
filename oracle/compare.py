"""Parity checks of a top-k result against the oracle's exact scores.

TEST INFRASTRUCTURE ONLY (used by tests/, smoke() and bench.py's oracle leg).

The rule (Sec. 2 "Top-k selection": the k highest-scoring documents, ties
broken by the lower doc id; tolerance 1e-5 relative):

  tol(D) = rtol * max(|B(Q,D)|, sum_i |S(q_i, D)|)          rtol = 1e-5

The second term keeps terms of opposite sign (Robertson's negative IDF) from
making a relative bound meaningless.  With k' = min(k, N), `order` the
oracle's ranking (score descending, doc id ascending) and B_k the oracle
score of order[k'-1] (the k-th best), tol_k = tol(order[k'-1]):

  * every returned score is within tol(D) of the oracle's B(Q,D);
  * ids may differ from the oracle's top k' only among documents whose
    oracle score lies within tol_k of B_k: every oracle top-k' document
    scoring more than B_k + tol_k is returned, and every returned document
    scores at least B_k - tol_k;
  * the returned ids are in [0, N) and distinct, and the row is ordered by
    its own scores (descending; equal scores by ascending doc id);
  * slots past k' hold id -1 and score -inf.

check_topk raises AssertionError with a message naming the first violation.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-5


def tolerance(full, abs_full, rtol: float = RTOL):
    """Per-document tolerance rtol * max(|B|, sum |S|)."""
    return rtol * np.maximum(np.abs(full), abs_full)


def check_topk(ids, scores, full, abs_full, k: int, rtol: float = RTOL, where: str = ""):
    ids = np.asarray(ids)
    scores = np.asarray(scores, dtype=np.float64)
    full = np.asarray(full, dtype=np.float64)
    abs_full = np.asarray(abs_full, dtype=np.float64)
    n = full.shape[0]
    kp = min(k, n)
    assert ids.shape[0] == k and scores.shape[0] == k, f"{where}: expected {k} slots"
    if kp < k:
        assert (ids[kp:] == -1).all(), f"{where}: padding ids must be -1, got {ids[kp:][:5]}"
        assert np.isneginf(scores[kp:]).all(), \
            f"{where}: padding scores must be -inf, got {scores[kp:][:5]}"
    got = ids[:kp].astype(np.int64)
    sc = scores[:kp]
    assert ((got >= 0) & (got < n)).all(), f"{where}: id out of range {got[(got < 0) | (got >= n)][:5]}"
    assert np.unique(got).shape[0] == kp, f"{where}: duplicate ids {got}"
    assert np.isfinite(sc).all(), f"{where}: non-finite score among the first {kp} slots"
    tol = tolerance(full, abs_full, rtol)
    err = np.abs(sc - full[got])
    bad = err > tol[got]
    assert not bad.any(), (f"{where}: score mismatch at ranks {np.nonzero(bad)[0][:5]}: "
                           f"got {sc[bad][:5]} want {full[got][bad][:5]}")
    order = np.lexsort((np.arange(n), -full))
    kth_doc = order[kp - 1]
    kth = full[kth_doc]
    tol_k = tol[kth_doc]
    lo = full[got] < kth - tol_k
    assert not lo.any(), (f"{where}: returned ids {got[lo][:5]} (oracle {full[got][lo][:5]}) "
                          f"are below the k-th score {kth} by more than {tol_k}")
    top = order[:kp]
    must = top[full[top] > kth + tol_k]
    missing = np.setdiff1d(must, got)
    assert missing.shape[0] == 0, (f"{where}: top ids {missing[:5]} "
                                   f"(oracle {full[missing][:5]}) missing")
    # the row's own order: scores non-increasing, equal scores by ascending id
    ds = np.diff(sc)
    assert (ds <= 0).all(), f"{where}: scores not sorted descending at {np.nonzero(ds > 0)[0][:5]}"
    eq = ds == 0
    assert (np.diff(got)[eq] > 0).all(), f"{where}: equal scores not ordered by doc id"


def check_topk_with_list(ids, scores, top_ids, top_scores, k: int, n_docs: int,
                         rtol: float = RTOL, where: str = ""):
    """check_topk when the oracle's full score vector is too large to score
    for every query: the oracle's own top m > k list (ids, FP64 scores, as
    oracle.topk returns them) stands in for it.  Valid for score vectors
    whose terms are all >= 0 (sum_i |S| = B: every variant but Robertson).
    Documents outside the list score at most the list's last score; that is
    enough to apply the same rule as check_topk as long as the last score
    lies more than the k-th tolerance below the k-th score (else the list is
    too short to decide, and AssertionError says so)."""
    ids = np.asarray(ids)
    scores = np.asarray(scores, dtype=np.float64)
    top_ids = np.asarray(top_ids, dtype=np.int64)
    top_scores = np.asarray(top_scores, dtype=np.float64)
    m = int((top_ids >= 0).sum())
    kp = min(k, n_docs)
    assert ids.shape[0] == k and scores.shape[0] == k, f"{where}: expected {k} slots"
    if kp < k:
        assert (ids[kp:] == -1).all(), f"{where}: padding ids must be -1"
        assert np.isneginf(scores[kp:]).all(), f"{where}: padding scores must be -inf"
    got = ids[:kp].astype(np.int64)
    sc = scores[:kp]
    assert ((got >= 0) & (got < n_docs)).all(), f"{where}: id out of range"
    assert np.unique(got).shape[0] == kp, f"{where}: duplicate ids {got}"
    kth = top_scores[kp - 1]
    tol_k = rtol * abs(kth)
    if m < n_docs:
        assert top_scores[m - 1] < kth - tol_k, (f"{where}: the oracle list of {m} is too short "
                                                 f"to decide ties at the k-th score")
    pos = {int(d): i for i, d in enumerate(top_ids[:m])}
    for r, d in enumerate(got.tolist()):
        assert d in pos, f"{where}: returned id {d} is not within the tolerance of the top {kp}"
        b = top_scores[pos[d]]
        assert abs(sc[r] - b) <= rtol * abs(b), \
            f"{where}: score mismatch at rank {r}: got {sc[r]} want {b}"
        assert b >= kth - tol_k, f"{where}: returned id {d} ({b}) below the k-th score {kth}"
    must = top_ids[:kp][top_scores[:kp] > kth + tol_k]
    missing = np.setdiff1d(must, got)
    assert missing.shape[0] == 0, f"{where}: top ids {missing[:5]} missing"
    ds = np.diff(sc)
    assert (ds <= 0).all(), f"{where}: scores not sorted descending"
    assert (np.diff(got)[ds == 0] > 0).all(), f"{where}: equal scores not ordered by doc id"

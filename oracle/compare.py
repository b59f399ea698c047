"""Parity checks of a top-k result against the oracle's exact scores.

TEST INFRASTRUCTURE ONLY (used by tests/, smoke() and bench.py's oracle leg).

Tolerance: |s - B(Q,D)| <= rtol * max(|B(Q,D)|, sum_i |S(q_i, D)|), rtol 1e-5.
The second term keeps terms of opposite sign (Robertson's negative IDF) from
making a relative bound meaningless.  Ids must equal the oracle's ranking
except where oracle scores are within that tolerance of each other, so only
what is unique is compared exactly:
  * every returned document's oracle score is at least the k-th best oracle
    score minus the tolerance;
  * every document whose oracle score beats the k-th by more than the
    tolerance is returned;
  * the returned list holds no duplicate and is ordered by its own scores
    (descending, then doc id ascending);
  * slots past min(k, N) hold id -1 and score -inf.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-5


def check_topk(ids, scores, full, abs_full, k: int, rtol: float = RTOL, where: str = ""):
    ids = np.asarray(ids)
    scores = np.asarray(scores, dtype=np.float64)
    n = full.shape[0]
    kp = min(k, n)
    assert ids.shape[0] == k, f"{where}: expected {k} slots"
    if kp < k:
        assert (ids[kp:] == -1).all(), f"{where}: padding ids must be -1"
        assert np.isneginf(scores[kp:]).all(), f"{where}: padding scores must be -inf"
    got = ids[:kp].astype(np.int64)
    sc = scores[:kp]
    assert ((got >= 0) & (got < n)).all(), f"{where}: id out of range {got}"
    assert np.unique(got).shape[0] == kp, f"{where}: duplicate ids {got}"
    tol_doc = rtol * np.maximum(np.abs(full), abs_full)
    err = np.abs(sc - full[got])
    bad = err > tol_doc[got] + 1e-300
    assert not bad.any(), (f"{where}: score mismatch at ranks {np.nonzero(bad)[0][:5]}: "
                           f"got {sc[bad][:5]} want {full[got][bad][:5]}")
    order = np.lexsort((np.arange(n), -full))
    kth = full[order[kp - 1]]
    tol_k = rtol * max(abs(kth), float(abs_full[order[kp - 1]]))
    lo = full[got] < kth - 2 * tol_k - tol_doc[got]
    assert not lo.any(), f"{where}: returned ids {got[lo][:5]} are not in the top {kp}"
    must = order[:kp][full[order[:kp]] > kth + 2 * tol_k + tol_doc[order[:kp]]]
    missing = np.setdiff1d(must, got)
    assert missing.shape[0] == 0, f"{where}: top ids {missing[:5]} missing"
    # own order: scores non-increasing; equal scores by ascending id
    ds = np.diff(sc)
    assert (ds <= 0).all(), f"{where}: scores not sorted"
    eq = ds == 0
    assert (np.diff(got)[eq] > 0).all(), f"{where}: equal scores not ordered by doc id"

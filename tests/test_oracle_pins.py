"""Pins for the FP64 oracle: checks against things other than the oracle.

* a hand-worked 3-document corpus (tests/golden/toy_corpus.json) whose
  intermediate values are exact rationals (Sec. 2 "Calculation of BM25",
  Sec. 2.1);
* closed forms and algebraic identities of the IDF variants;
* invariants the paper states: TF = 0 gives S = 0 for the sparse variants
  (Sec. 2 "Eager index-time scoring"), S0 does not depend on D and
  B = sum S_delta + sum S0 (Sec. 2.1), and the shift leaves the ranking alone;
* brute force on tiny corpora (counting, sets, scipy's CSC, numpy lexsort).
"""
import json
import math
import os
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2407_03618_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toy_corpus.json")
VARIANTS = ["lucene", "robertson", "atire", "bm25l", "bm25+"]
VID = {"lucene": 0, "robertson": 1, "atire": 2, "bm25l": 3, "bm25+": 4}


@pytest.fixture(scope="module")
def toy():
    with open(GOLDEN) as f:
        return json.load(f)


def _toy_corpus(toy):
    docs = toy["docs"]
    tok = np.array([t for d in docs for t in d], np.int32)
    off = np.zeros(len(docs) + 1, np.int64)
    off[1:] = np.cumsum([len(d) for d in docs])
    return tok, off


def _params(toy):
    return (float(Fraction(toy["k1"])), float(Fraction(toy["b"])), float(Fraction(toy["delta"])))


# ---------------------------------------------------------------- toy ----

@pytest.mark.parametrize("variant", VARIANTS)
def test_toy_structure(oracle_mod, toy, variant):
    tok, off = _toy_corpus(toy)
    k1, b, d = _params(toy)
    ix = oracle_mod.build(tok, off, toy["vocab"], VID[variant], k1, b, d)
    assert ix.doc_len.tolist() == toy["doc_len"]
    assert ix.lavg == float(Fraction(toy["lavg"]))
    assert ix.df.tolist() == toy["df"]
    assert ix.nnz == toy["nnz"]
    assert ix.indptr.tolist() == toy["indptr"]
    assert ix.indices.tolist() == toy["indices"]
    for key, tf in toy["tf"].items():
        t, dd = map(int, key.split(","))
        lo, hi = ix.indptr[t], ix.indptr[t + 1]
        j = lo + list(ix.indices[lo:hi]).index(dd)
        assert ix.csc_tf[j] == tf


@pytest.mark.parametrize("variant", VARIANTS)
def test_toy_idf_and_scores(oracle_mod, toy, variant):
    tok, off = _toy_corpus(toy)
    k1, b, d = _params(toy)
    g = toy["variants"][variant]
    ix = oracle_mod.build(tok, off, toy["vocab"], VID[variant], k1, b, d)
    # IDF: hand-evaluated logarithms of exact arguments
    np.testing.assert_allclose(ix.idf, g["idf"], rtol=0, atol=5e-11)
    for t, arg in enumerate(g["idf_arg"]):
        assert ix.idf[t] == pytest.approx(math.log(float(Fraction(arg))), rel=1e-14, abs=1e-15)
    # S0 = IDF * s0_ratio for terms that occur; 0 for the DF = 0 term
    s0r = float(Fraction(g["s0_ratio"]))
    for t in range(toy["vocab"]):
        assert ix.s0[t] == pytest.approx(ix.idf[t] * s0r, rel=1e-13, abs=1e-15)
    # stored S - S0 = IDF * (ratio - s0_ratio), exact rationals from the hand derivation
    for key, ratio in g["ratio"].items():
        t, dd = map(int, key.split(","))
        lo, hi = ix.indptr[t], ix.indptr[t + 1]
        j = lo + list(ix.indices[lo:hi]).index(dd)
        want = ix.idf[t] * float(Fraction(ratio) - Fraction(g["s0_ratio"]))
        assert ix.csc_delta[j] == pytest.approx(want, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("variant", VARIANTS)
def test_toy_lazy_scores_and_order(oracle_mod, toy, variant):
    tok, off = _toy_corpus(toy)
    k1, b, d = _params(toy)
    g = toy["variants"][variant]
    ix = oracle_mod.build(tok, off, toy["vocab"], VID[variant], k1, b, d)
    for case in g["queries"]:
        sc = oracle_mod.score_all(ix, case["q"])
        np.testing.assert_allclose(sc, case["B"], rtol=0, atol=5e-11)
        assert oracle_mod.rank(sc).tolist() == case["order"]
        qo = np.array([0, len(case["q"])], np.int64)
        ids, scs = oracle_mod.topk(ix, np.array(case["q"], np.int32), qo, 3)
        assert ids[0].tolist() == case["order"]


def test_toy_spot_values(oracle_mod, toy):
    """Single S values worked by hand (Lucene S(t0,D0), BM25L and BM25+ shifts)."""
    tok, off = _toy_corpus(toy)
    k1, b, d = _params(toy)
    lu = oracle_mod.build(tok, off, 5, 0, k1, b, d)
    # Lucene S(t0, D0) = ln(8/5) * 80/191
    assert lu.csc_delta[0] == pytest.approx(math.log(1.6) * 80 / 191, rel=1e-14)
    assert lu.csc_delta[0] == pytest.approx(0.1968601588, abs=5e-11)
    bl = oracle_mod.build(tok, off, 5, 3, k1, b, d)
    j = bl.indptr[3]  # (t3, D2)
    assert bl.csc_delta[j] == pytest.approx(0.4904146265, abs=5e-11)
    bp = oracle_mod.build(tok, off, 5, 4, k1, b, d)
    j = bp.indptr[1]  # (t1, D0)
    assert bp.csc_delta[j] == pytest.approx(0.4246229852, abs=5e-11)


# ------------------------------------------------------- closed forms ----

@pytest.mark.parametrize("n", [1, 2, 3, 10, 101, 1000, 10**6])
def test_idf_closed_forms(oracle_mod, n):
    for df in sorted({1, max(1, n // 3), max(1, n // 2), n}):
        lu = oracle_mod.idf(0, n, df)
        ro = oracle_mod.idf(1, n, df)
        at = oracle_mod.idf(2, n, df)
        bl = oracle_mod.idf(3, n, df)
        bp = oracle_mod.idf(4, n, df)
        # (N - DF + 0.5)/(DF + 0.5) + 1 simplifies to (N + 1)/(DF + 0.5):
        # Lucene's IDF equals BM25L's
        assert lu == pytest.approx(bl, rel=1e-14)
        assert lu > 0
        # Robertson is antisymmetric about N/2 and negative exactly above it
        assert ro == pytest.approx(-oracle_mod.idf(1, n, n - df), rel=1e-12, abs=1e-14) if df < n else True
        assert (ro < 0) == (df > n / 2)
        # Lucene - Robertson = ln((N + 1)/(N - DF + 0.5))
        assert lu - ro == pytest.approx(math.log((n + 1) / (n - df + 0.5)), rel=1e-12)
        # ATIRE = ln N - ln DF; BM25+ = ln(N + 1) - ln DF
        assert at == pytest.approx(math.log(n) - math.log(df), rel=1e-12, abs=1e-14)
        assert bp == pytest.approx(math.log(n + 1) - math.log(df), rel=1e-12, abs=1e-14)
    assert oracle_mod.idf(2, n, n) == 0.0
    assert oracle_mod.idf(4, n, n) == pytest.approx(math.log1p(1.0 / n), rel=1e-12)
    if n % 2 == 0:
        assert oracle_mod.idf(1, n, n // 2) == 0.0
    for v in range(5):
        assert oracle_mod.idf(v, n, 0) == 0.0


def test_tf_zero_is_zero_for_sparse_variants(oracle_mod):
    rng = np.random.default_rng(3)
    for _ in range(200):
        idf_t = rng.normal() * 3
        ln, la = rng.uniform(0, 50), rng.uniform(1, 50)
        k1, b, d = rng.uniform(0, 3), rng.uniform(0, 1), rng.uniform(0, 2)
        for v in (0, 1, 2):
            assert oracle_mod.term_score(v, idf_t, 0, ln, la, k1, b, d) == 0.0
            assert oracle_mod.nonoccurrence(v, idf_t, k1, b, d) == 0.0


def test_nonoccurrence_is_free_of_the_document(oracle_mod):
    rng = np.random.default_rng(4)
    for _ in range(200):
        idf_t = abs(rng.normal()) * 3
        k1, b, d = rng.uniform(0.1, 3), rng.uniform(0, 1), rng.uniform(0, 2)
        for v in (3, 4):
            s0 = oracle_mod.nonoccurrence(v, idf_t, k1, b, d)
            for ln in (0, 1, 7, 300):
                assert oracle_mod.term_score(v, idf_t, 0, ln, rng.uniform(1, 50), k1, b, d) == \
                    pytest.approx(s0, rel=1e-14)
        # hand-simplified: BM25L S0 = IDF (k1+1) d/(k1+d); BM25+ S0 = IDF d
        assert oracle_mod.nonoccurrence(3, idf_t, k1, b, d) == pytest.approx(
            idf_t * (k1 + 1) * d / (k1 + d), rel=1e-13, abs=1e-15)
        assert oracle_mod.nonoccurrence(4, idf_t, k1, b, d) == pytest.approx(idf_t * d, rel=1e-13,
                                                                              abs=1e-15)


def test_delta_zero_collapses_variants(oracle_mod):
    """With delta = 0, BM25L, BM25+ and ATIRE all reduce to
    IDF (k1+1) TF/(TF + k1 K_D); Lucene is that without the (k1+1)."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        tf = int(rng.integers(1, 40))
        ln, la = rng.uniform(1, 200), rng.uniform(1, 200)
        k1, b = rng.uniform(0.05, 3), rng.uniform(0, 1)
        at = oracle_mod.term_score(2, 1.0, tf, ln, la, k1, b, 0.0)
        assert oracle_mod.term_score(3, 1.0, tf, ln, la, k1, b, 0.0) == pytest.approx(at, rel=1e-13)
        assert oracle_mod.term_score(4, 1.0, tf, ln, la, k1, b, 0.0) == pytest.approx(at, rel=1e-13)
        assert oracle_mod.term_score(0, 1.0, tf, ln, la, k1, b, 0.0) * (k1 + 1) == \
            pytest.approx(at, rel=1e-13)


def test_b_zero_and_saturation(oracle_mod):
    rng = np.random.default_rng(6)
    for _ in range(100):
        tf = int(rng.integers(1, 20))
        k1 = rng.uniform(0.1, 3)
        for v in range(5):
            # b = 0: no length normalisation, the score ignores |D|
            a = oracle_mod.term_score(v, 1.3, tf, 5, 60, k1, 0.0, 0.5)
            c = oracle_mod.term_score(v, 1.3, tf, 500, 60, k1, 0.0, 0.5)
            assert a == pytest.approx(c, rel=1e-14)
        # TF -> infinity: Lucene -> IDF, ATIRE and BM25L -> IDF(k1+1), BM25+ -> IDF(k1+1+d)
        big = 1e13
        assert oracle_mod.term_score(0, 2.0, big, 50, 60, k1, 0.75, 0.5) == pytest.approx(2.0, rel=1e-9)
        assert oracle_mod.term_score(2, 2.0, big, 50, 60, k1, 0.75, 0.5) == pytest.approx(2 * (k1 + 1), rel=1e-9)
        assert oracle_mod.term_score(3, 2.0, big, 50, 60, k1, 0.75, 0.5) == pytest.approx(2 * (k1 + 1), rel=1e-9)
        assert oracle_mod.term_score(4, 2.0, big, 50, 60, k1, 0.75, 0.5) == pytest.approx(2 * (k1 + 1.5), rel=1e-9)
        # k1 = 0: Lucene scores IDF for any TF > 0
        assert oracle_mod.term_score(0, 2.0, tf, 50, 60, 0.0, 0.75, 0.5) == pytest.approx(2.0, rel=1e-15)


def test_monotone_in_tf_and_length(oracle_mod):
    for v in range(5):
        s = [oracle_mod.term_score(v, 1.0, tf, 60, 60, 1.2, 0.75, 0.5) for tf in range(1, 30)]
        assert all(x < y for x, y in zip(s, s[1:]))
        s = [oracle_mod.term_score(v, 1.0, 3, ln, 60, 1.2, 0.75, 0.5) for ln in range(1, 300, 7)]
        assert all(x > y for x, y in zip(s, s[1:]))


# ------------------------------------------------- brute force, tiny ----

def _brute_tf(corpus):
    out = []
    for dd in range(corpus.n_docs):
        toks = corpus.tokens[corpus.doc_offsets[dd]:corpus.doc_offsets[dd + 1]].tolist()
        out.append(Counter(toks))
    return out


@pytest.mark.parametrize("seed", range(40))
def test_structure_by_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    c = synth.random_tiny_corpus(rng, max_docs=12, max_vocab=9, max_len=10)
    ix = oracle_mod.build(c.tokens, c.doc_offsets, c.vocab, seed % 5, 1.2, 0.75, 0.5)
    tfs = _brute_tf(c)
    assert ix.doc_len.tolist() == [sum(t.values()) for t in tfs]
    assert ix.df.tolist() == [sum(1 for t in tfs if v in t) for v in range(c.vocab)]
    # CSC of the |C| x |V| count matrix, built by scipy
    rows, cols, vals = [], [], []
    for dd, t in enumerate(tfs):
        for v, n in t.items():
            rows.append(dd)
            cols.append(v)
            vals.append(n)
    m = sp.csc_matrix((np.array(vals, np.int64), (rows, cols)), shape=(c.n_docs, c.vocab))
    m.sort_indices()
    assert ix.indptr.tolist() == m.indptr.tolist()
    assert ix.indices.tolist() == m.indices.tolist()
    assert ix.csc_tf.tolist() == m.data.tolist()


@pytest.mark.parametrize("variant", range(5))
def test_shift_identity_brute_force(oracle_mod, variant):
    """Lazy B(Q,D) equals eager sum of S - S0 over stored pairs plus sum S0
    (Sec. 2.1), on 250 random tiny corpora per variant."""
    rng = np.random.default_rng(7 + variant)
    for _ in range(250):
        c = synth.random_tiny_corpus(rng)
        k1, b, d = rng.uniform(0.2, 2.5), rng.uniform(0, 1), rng.uniform(0, 1.5)
        ix = oracle_mod.build(c.tokens, c.doc_offsets, c.vocab, variant, k1, b, d)
        q = rng.integers(0, c.vocab, int(rng.integers(0, 6))).astype(np.int32)
        lazy = oracle_mod.score_all(ix, q)
        eager = np.zeros(c.n_docs)
        for t in q:
            lo, hi = ix.indptr[t], ix.indptr[t + 1]
            np.add.at(eager, ix.indices[lo:hi], ix.csc_delta[lo:hi])
        shift = sum(ix.s0[t] for t in q)
        scale = 1.0 + np.abs(lazy).max(initial=0.0)
        np.testing.assert_allclose(eager + shift, lazy, rtol=0, atol=1e-12 * scale)
        if variant <= 2:
            assert shift == 0.0


def test_rank_matches_lexsort_and_shift_invariance(oracle_mod):
    rng = np.random.default_rng(8)
    for _ in range(100):
        n = int(rng.integers(1, 60))
        sc = np.round(rng.normal(size=n), 1)  # many exact ties
        order = oracle_mod.rank(sc)
        assert order.tolist() == np.lexsort((np.arange(n), -sc)).tolist()
    # -0.0 ties with +0.0 and the lower id wins
    assert oracle_mod.rank(np.array([0.0, -0.0, 0.0, -1.0])).tolist() == [0, 1, 2, 3]
    assert oracle_mod.rank(np.array([-0.0, 0.0])).tolist() == [0, 1]


def test_topk_padding_and_empty_query(oracle_mod):
    c = synth.Corpus(np.array([0, 1, 1, 2], np.int32), np.array([0, 2, 2, 4], np.int64), 3)
    ix = oracle_mod.build(c.tokens, c.doc_offsets, 3, 0)
    ids, sc = oracle_mod.topk(ix, np.zeros(0, np.int32), np.array([0, 0], np.int64), 5)
    assert ids[0].tolist() == [0, 1, 2, -1, -1]
    assert sc[0, :3].tolist() == [0.0, 0.0, 0.0]
    assert np.isneginf(sc[0, 3:]).all()
    # duplicate query tokens count per occurrence
    one = oracle_mod.score_all(ix, [1])
    two = oracle_mod.score_all(ix, [1, 1])
    np.testing.assert_allclose(two, 2 * one, rtol=1e-15)


def test_invalid_corpus_rejected(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.build(np.array([0, 5], np.int32), np.array([0, 2], np.int64), 3)
    with pytest.raises(ValueError):
        oracle_mod.build(np.array([0, 1], np.int32), np.array([0, 3], np.int64), 3)


@pytest.mark.parametrize("variant", range(6))
def test_query_time_parameters_equal_a_build_with_them(oracle_mod, variant):
    """Lazy scoring with k1, b, delta given at query time equals scoring an
    index built with those parameters (the IDF does not depend on them), and
    differs from the build's own parameters where TF or |D| matter."""
    rng = np.random.default_rng(60 + variant)
    for _ in range(40):
        c = synth.random_tiny_corpus(rng, allow_empty=False)
        built = oracle_mod.build(c.tokens, c.doc_offsets, c.vocab, variant, 1.2, 0.75, 0.5)
        k1, b = float(rng.uniform(0.1, 3.0)), float(rng.uniform(0, 1))
        d = float(rng.uniform(0.4, 2.0))
        other = oracle_mod.build(c.tokens, c.doc_offsets, c.vocab, variant, k1, b, d)
        q = rng.integers(0, c.vocab, int(rng.integers(1, 6))).astype(np.int32)
        a = oracle_mod.score_all(built, q, k1=k1, b=b, delta=d)
        assert np.array_equal(a, oracle_mod.score_all(other, q))
        ids, sc = oracle_mod.topk(built, q, np.array([0, q.shape[0]]), 3, k1=k1, b=b, delta=d)
        ids2, sc2 = oracle_mod.topk(other, q, np.array([0, q.shape[0]]), 3)
        assert np.array_equal(ids, ids2) and np.array_equal(sc, sc2)

"""Pins for the oracle's TF_{l o delta o p} x IDF (Sec. 2.1 names it, with
BM25L and BM25+, as a model whose score at TF = 0 is not zero and that the
shift makes sparse; its form is Rousseau and Vazirgiannis 2013's
composition of the pivoted normalisation p, the lower bound delta and the
double logarithm l, times IDF = ln((|C| + 1) / DF)).

Checked against closed forms at parameters where the logarithms come out
exact, the invariants of the three composed steps, and the shift identity
by brute force on tiny corpora.
"""
import math

import numpy as np
import pytest

from paper_2407_03618_gb300 import synth

TFLDP, BM25PLUS = 5, 4
E = math.e


def test_idf_is_bm25plus_idf(oracle_mod):
    for n in (1, 2, 10, 1000, 10**6):
        for df in sorted({1, max(1, n // 2), n}):
            assert oracle_mod.idf(TFLDP, n, df) == oracle_mod.idf(BM25PLUS, n, df)
            assert oracle_mod.idf(TFLDP, n, df) == pytest.approx(math.log((n + 1) / df), rel=1e-14)
        assert oracle_mod.idf(TFLDP, n, 0) == 0.0


def test_closed_forms(oracle_mod):
    rng = np.random.default_rng(21)
    for _ in range(100):
        w = float(rng.uniform(0.1, 5.0))
        k1, ln_, la = float(rng.uniform(0, 3)), float(rng.uniform(1, 100)), float(rng.uniform(1, 100))
        # delta = 1: ln(1) = 0, so S0 = IDF (1 + ln 1) = IDF
        assert oracle_mod.nonoccurrence(TFLDP, w, k1, 0.75, 1.0) == pytest.approx(w, rel=1e-15)
        # delta = e^(1/e - 1): 1 + ln delta = 1/e, ln(1/e) = -1, so S0 = 0 (a sparse case)
        d0 = math.exp(1.0 / E - 1.0)
        assert abs(oracle_mod.nonoccurrence(TFLDP, w, k1, 0.3, d0)) <= 1e-14 * w
        # b = 0, TF = 1, delta = e - 1: ln(1 + delta) = 1, so S = IDF (1 + ln 2), any |D|
        assert oracle_mod.term_score(TFLDP, w, 1, ln_, la, k1, 0.0, E - 1.0) == \
            pytest.approx(w * (1.0 + math.log(2.0)), rel=1e-14)
        # b = 0, TF + delta = e^(e - 1): ln(1 + (e - 1)) = 1, so S = 2 IDF
        assert oracle_mod.term_score(TFLDP, w, E ** (E - 1.0) - 1.0, ln_, la, k1, 0.0, 1.0) == \
            pytest.approx(2.0 * w, rel=1e-14)


def test_pivoted_normalisation_and_k1_unused(oracle_mod):
    rng = np.random.default_rng(22)
    for _ in range(100):
        w, la = float(rng.uniform(0.1, 5.0)), float(rng.uniform(1, 100))
        d = float(rng.uniform(0.4, 2.0))
        tf = int(rng.integers(1, 30))
        # b = 1 and |D| = 2 Lavg halves TF: the same as TF / 2 without normalisation
        a = oracle_mod.term_score(TFLDP, w, 2 * tf, 2 * la, la, 1.2, 1.0, d)
        c = oracle_mod.term_score(TFLDP, w, tf, 7.0, la, 1.2, 0.0, d)
        assert a == pytest.approx(c, rel=1e-14)
        # |D| = Lavg: K_D = 1 for every b
        assert oracle_mod.term_score(TFLDP, w, tf, la, la, 1.2, float(rng.uniform(0, 1)), d) == \
            pytest.approx(oracle_mod.term_score(TFLDP, w, tf, la, la, 1.2, 0.0, d), rel=1e-14)
        # k1 plays no part
        assert oracle_mod.term_score(TFLDP, w, tf, 30.0, la, 0.0, 0.6, d) == \
            oracle_mod.term_score(TFLDP, w, tf, 30.0, la, 2.9, 0.6, d)


def test_monotone_and_free_of_document_at_tf_zero(oracle_mod):
    s = [oracle_mod.term_score(TFLDP, 1.0, tf, 60, 60, 1.2, 0.75, 0.5) for tf in range(0, 40)]
    assert all(x < y for x, y in zip(s, s[1:]))
    s = [oracle_mod.term_score(TFLDP, 1.0, 3, ln, 60, 1.2, 0.75, 0.5) for ln in range(1, 300, 7)]
    assert all(x > y for x, y in zip(s, s[1:]))
    s0 = oracle_mod.nonoccurrence(TFLDP, 1.7, 1.2, 0.75, 0.5)
    assert s0 == pytest.approx(1.7 * (1 + math.log(1 + math.log(0.5))), rel=1e-14)
    assert s0 < 0  # delta = 0.5 < e^(1/e - 1): the non-occurrence score is negative
    for ln in (0, 1, 9, 400):
        assert oracle_mod.term_score(TFLDP, 1.7, 0, ln, 33.0, 1.2, 0.75, 0.5) == \
            pytest.approx(s0, rel=1e-14)


def test_shift_identity_brute_force(oracle_mod):
    """Lazy B(Q,D) = eager sum of S - S0 + sum S0 (Sec. 2.1), 250 tiny corpora."""
    rng = np.random.default_rng(23)
    for _ in range(250):
        c = synth.random_tiny_corpus(rng)
        b, d = rng.uniform(0, 1), rng.uniform(0.38, 2.0)
        ix = oracle_mod.build(c.tokens, c.doc_offsets, c.vocab, TFLDP, 1.2, b, d)
        q = rng.integers(0, c.vocab, int(rng.integers(0, 6))).astype(np.int32)
        lazy = oracle_mod.score_all(ix, q)
        eager = np.zeros(c.n_docs)
        for t in q:
            lo, hi = ix.indptr[t], ix.indptr[t + 1]
            np.add.at(eager, ix.indices[lo:hi], ix.csc_delta[lo:hi])
            assert (ix.csc_delta[lo:hi] > 0).all()  # S grows with TF above S0
        shift = sum(ix.s0[t] for t in q)
        scale = 1.0 + np.abs(lazy).max(initial=0.0)
        np.testing.assert_allclose(eager + shift, lazy, rtol=0, atol=1e-12 * scale)

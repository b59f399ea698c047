"""Query-time scoring (lazy postings: TF and |D| in place of the score;
S computed in the tile kernel with the call's k1, b, delta).

* With the index's own parameters: the same top k as the eager path
  (bm25_retrieve) up to ties within the tolerance, and the oracle's.
* With other parameters: the oracle's lazy scoring at those parameters
  (check_topk), for every variant.
* The unpacked layout (a TF above 65,535) and the argument checks.
"""
import numpy as np
import pytest

import oracle
from oracle.compare import RTOL, check_topk
from paper_2407_03618_gb300 import synth

pytestmark = pytest.mark.gpu

VARIANTS = ["lucene", "robertson", "atire", "bm25l", "bm25+", "tfldp"]


@pytest.fixture(scope="module")
def dev():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _to(dev, a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _check(ids, sc, orc, q, k, params, where):
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for i in range(q.n_queries):
        full, ab = oracle.score_all(orc, q.query(i), with_abs=True, **params)
        check_topk(ids[i], sc[i], full, ab, k, where=f"{where} q{i}")


@pytest.mark.parametrize("variant", VARIANTS)
def test_lazy_parity(dev, variant):
    from paper_2407_03618_gb300 import bm25
    c = synth.make_corpus(30_000, 6_000, 1.1, ("lognormal", 50, 0.6), seed=12)
    q = synth.make_queries(80, 6_000, 1.1, ("uniform", 1, 10), seed=13)
    ix = bm25.Index.build(_to(dev, c.tokens), _to(dev, c.doc_offsets), c.vocab, variant,
                          1.5, 0.75, 0.5)
    ix.enable_lazy()
    ix.enable_lazy()  # idempotent
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.VARIANTS[variant], 1.5, 0.75, 0.5)
    qt, qo = _to(dev, q.tokens), _to(dev, q.offsets)
    for k in (1, 10, 200):
        lid, lsc = ix.retrieve_lazy(qt, qo, k, 1.5, 0.75, 0.5)
        eid, esc = ix.retrieve(qt, qo, k)
        ix.sync_status()
        np.testing.assert_allclose(lsc.cpu().numpy(), esc.cpu().numpy(), rtol=RTOL, atol=RTOL)
        _check(lid, lsc, orc, q, k, {}, f"{variant} own k={k}")
    for (k1, b, d) in ((0.9, 0.4, 0.6), (2.0, 1.0, 1.0), (1.2, 0.0, 0.8)):
        lid, lsc = ix.retrieve_lazy(qt, qo, 10, k1, b, d)
        ix.sync_status()
        _check(lid, lsc, orc, q, 10, {"k1": k1, "b": b, "delta": d},
               f"{variant} k1={k1} b={b} d={d}")
    ix.close()


def test_lazy_unpacked_layout(dev):
    """One document repeats a term 70,000 times: TF does not fit 16 bits, so
    TF is kept in 32 bits and |D| read from the document lengths."""
    from paper_2407_03618_gb300 import bm25
    rng = np.random.default_rng(14)
    lens = rng.integers(1, 40, 3000)
    lens[1234] = 70_000
    off = synth.offsets_from_lengths(lens)
    tok = rng.integers(0, 500, int(off[-1])).astype(np.int32)
    tok[off[1234]:off[1235]] = 7
    c = synth.Corpus(tok, off, 500)
    q = synth.Queries(np.array([7, 7, 3, 9, 7, 11], np.int32), np.array([0, 1, 3, 6], np.int64))
    ix = bm25.Index.build(_to(dev, c.tokens), _to(dev, c.doc_offsets), c.vocab, "bm25+")
    ix.enable_lazy()
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25PLUS, 1.5, 0.75, 0.5)
    for (k1, b, d) in ((1.5, 0.75, 0.5), (0.7, 0.3, 1.1)):
        lid, lsc = ix.retrieve_lazy(_to(dev, q.tokens), _to(dev, q.offsets), 5, k1, b, d)
        ix.sync_status()
        _check(lid, lsc, orc, q, 5, {"k1": k1, "b": b, "delta": d}, f"unpacked {k1} {b} {d}")
    ix.close()


def test_lazy_argument_checks(dev):
    from paper_2407_03618_gb300 import bm25
    c = synth.make_corpus(500, 100, 1.1, ("poisson", 10), seed=15)
    q = synth.make_queries(4, 100, 1.1, ("uniform", 1, 3), seed=16)
    qt, qo = _to(dev, q.tokens), _to(dev, q.offsets)
    ix = bm25.Index.build(_to(dev, c.tokens), _to(dev, c.doc_offsets), c.vocab, "tfldp")
    with pytest.raises(bm25.BM25Error):
        ix.retrieve_lazy(qt, qo, 5, 1.2, 0.75, 0.5)  # not enabled
    ix.enable_lazy()
    for bad in ((-1.0, 0.5, 0.5), (1.2, 1.5, 0.5), (1.2, 0.5, 0.3)):  # k1 < 0, b > 1, delta < 1/e
        with pytest.raises(bm25.BM25Error):
            ix.retrieve_lazy(qt, qo, 5, *bad)
    ix.close()

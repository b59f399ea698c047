"""The device tokenizer (bm25_tokenize_corpus / bm25_tokenize_queries)
against the tokenizer oracle, bit for bit: term ids, per-text offsets and
the vocabulary (ids by first occurrence); and the whole path from text to
top k against the oracle's (its tokenizer, FP64 index, lazy top k)."""
import numpy as np
import pytest

import oracle
from oracle import tokenizer as tk
from oracle.compare import check_topk
from paper_2407_03618_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _to(dev, a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _tokenize(dev, texts, stop):
    from paper_2407_03618_gb300 import bm25
    buf, off = tk.pack(texts)
    ids, toff, vocab = bm25.tokenize_corpus(_to(dev, buf), _to(dev, off), stop)
    return ids.cpu().numpy(), toff.cpu().numpy(), vocab


@pytest.mark.parametrize("seed", [0, 1])
def test_corpus_and_queries_equal_the_oracle(dev, seed):
    from paper_2407_03618_gb300 import bm25
    text, off, lex = synth.make_text_corpus(20_000, 5_000, 1.1, ("poisson", 40), seed=seed)
    docs = synth.split_texts(text, off)
    stop = [w.lower() for w in lex[:25]]
    ids, toff, vocab = _tokenize(dev, docs, stop)
    want_ids, want_off, want_vocab = tk.tokenize_corpus(docs, stop)
    assert np.array_equal(ids, want_ids)
    assert np.array_equal(toff, want_off)
    assert vocab.words() == want_vocab
    qtext, qoff, _ = synth.make_text_corpus(300, 5_000, 1.1, ("poisson", 6), seed=50 + seed)
    qdocs = synth.split_texts(qtext, qoff) + [b"", b"zzzz-unknown qq", b"!!"]
    qbuf, qo = tk.pack(qdocs)
    qid, qof = bm25.tokenize_queries(vocab, _to(dev, qbuf), _to(dev, qo))
    wq, wo = tk.tokenize_queries(qdocs, want_vocab, stop)
    assert np.array_equal(qid.cpu().numpy(), wq)
    assert np.array_equal(qof.cpu().numpy(), wo)
    vocab.close()


def test_edge_texts(dev):
    docs = [b"", b"ab", b"cd", b"x", b"!!!", b"a" * 10_000 + b" bb", "ü".encode() * 3,
            "é".encode(), b"The THE the", b"end"]
    for stop in ([], [b"the", b"BB"]):
        ids, toff, vocab = _tokenize(dev, docs, stop)
        want_ids, want_off, want_vocab = tk.tokenize_corpus(docs, [s.lower() for s in stop])
        assert np.array_equal(ids, want_ids) and np.array_equal(toff, want_off)
        assert vocab.words() == want_vocab
        vocab.close()
    # a corpus without a single token
    ids, toff, vocab = _tokenize(dev, [b"a b", b"", b"."], [])
    assert ids.shape[0] == 0 and toff.tolist() == [0, 0, 0, 0] and vocab.words() == []
    vocab.close()


def test_text_to_top_k(dev):
    """Text -> device tokenizer -> index build -> query tokenizer -> top k,
    against the oracle's tokenizer, index and top k."""
    from paper_2407_03618_gb300 import bm25
    text, off, lex = synth.make_text_corpus(8_000, 3_000, 1.05, ("poisson", 50), seed=7)
    docs = synth.split_texts(text, off)
    stop = [w.lower() for w in lex[:10]]
    tid, toff, vocab = bm25.tokenize_corpus(_to(dev, text), _to(dev, off), stop)
    nv = vocab.info()["n_words"]
    ix = bm25.Index.build(tid, toff, nv, "bm25+")
    qtext, qoff, _ = synth.make_text_corpus(60, 3_000, 1.05, ("poisson", 5), seed=8)
    qid, qof = bm25.tokenize_queries(vocab, _to(dev, qtext), _to(dev, qoff))
    ids, sc = ix.retrieve(qid, qof, 10)
    ix.sync_status()
    w_ids, w_off, w_vocab = tk.tokenize_corpus(docs, stop)
    orc = oracle.build(w_ids, w_off, len(w_vocab), oracle.BM25PLUS, 1.5, 0.75, 0.5)
    wq, wqo = tk.tokenize_queries(synth.split_texts(qtext, qoff), w_vocab, stop)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for i in range(wqo.shape[0] - 1):
        full, ab = oracle.score_all(orc, wq[wqo[i]:wqo[i + 1]], with_abs=True)
        check_topk(ids[i], sc[i], full, ab, 10, where=f"text q{i}")
    ix.close()
    vocab.close()

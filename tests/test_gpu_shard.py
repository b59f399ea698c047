"""Doc-range sharding on one GPU: G = 2 and 3 shards (each its own index over
a contiguous range of documents, rescored with the collection's summed DF,
N and token count) against one index over the whole collection.

* Structure: each shard's CSC is the unsplit CSC restricted to its documents
  (local ids = global - first), TF and DF bit-exact.
* Scores: IDF, S0, Lavg and every stored S - S0 equal the unsplit index's
  bit for bit (the same arithmetic on the same inputs).
* Retrieval: the merge of the shards' top k (bm25_merge_topk) against the
  oracle over the whole collection (check_topk), and equal to the unsplit
  index's result up to ties within the tolerance.
"""
import numpy as np
import pytest

import oracle
from oracle.compare import RTOL, check_topk
from paper_2407_03618_gb300 import shard, synth

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


def _check_shards(loc, full_ex):
    indptr, indices = full_ex["indptr"], full_ex["indices"]
    vocab = indptr.shape[0] - 1
    term = np.repeat(np.arange(vocab), np.diff(indptr))
    for sh, (lo, hi) in zip(loc.shards, loc.ranges):
        ex = sh.export()
        info = sh.shard_info()
        assert info == {"doc_id_offset": lo, "global_n_docs": loc.n_docs,
                        "global_n_tokens": loc.n_tokens}
        m = (indices >= lo) & (indices < hi)
        assert np.array_equal(ex["indices"], indices[m] - lo)
        assert np.array_equal(ex["tf"], full_ex["tf"][m])
        want_ptr = np.concatenate([[0], np.cumsum(np.bincount(term[m], minlength=vocab))])
        assert np.array_equal(ex["indptr"], want_ptr)
        assert np.array_equal(ex["df"], np.diff(want_ptr).astype(np.int32))
        assert np.array_equal(ex["doc_len"], full_ex["doc_len"][lo:hi])
        # the collection's statistics: bit for bit
        assert np.array_equal(ex["idf"], full_ex["idf"])
        assert np.array_equal(ex["s0"], full_ex["s0"])
        assert ex["lavg"] == full_ex["lavg"]
        assert np.array_equal(ex["data"].view(np.uint32), full_ex["data"][m].view(np.uint32))


def _check_retrieval(dev, loc, full_ix, orc, q, k, sample):
    qt, qo = _to(dev, q.tokens), _to(dev, q.offsets)
    ids, sc = loc.retrieve(qt, qo, k)
    for sh in loc.shards:
        sh.sync_status()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    fid, fsc = full_ix.retrieve(qt, qo, k)
    full_ix.sync_status()
    fid, fsc = fid.cpu().numpy(), fsc.cpu().numpy()
    np.testing.assert_allclose(sc, fsc, rtol=RTOL, atol=RTOL)
    for i in sample:
        full, ab = oracle.score_all(orc, q.query(int(i)), with_abs=True)
        check_topk(ids[i], sc[i], full, ab, k, where=f"sharded q{i}")


@pytest.mark.parametrize("variant", ["lucene", "bm25+", "robertson", "tfldp"])
@pytest.mark.parametrize("g", [2, 3])
def test_tiny_shards(dev, variant, g):
    from paper_2407_03618_gb300 import bm25
    w = synth.WORKLOADS["tiny"]
    c, q = w.corpus(), w.queries()
    loc = shard.build_local(shard.GpuEngine(), c.tokens, c.doc_offsets, c.vocab, g, variant,
                            1.5, 0.75, 0.5, to_device=lambda a: _to(dev, a))
    full = bm25.Index.build(_to(dev, c.tokens), _to(dev, c.doc_offsets), c.vocab, variant,
                            1.5, 0.75, 0.5)
    _check_shards(loc, full.export())
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.VARIANTS[variant], 1.5, 0.75, 0.5)
    for k in (1, 10, 700, 2500):  # 700, 2500: wider than a shard's documents
        _check_retrieval(dev, loc, full, orc, q, k, range(q.n_queries))
    loc.close()
    full.close()


@pytest.mark.slow
@pytest.mark.parametrize("g", [2, 3])
def test_1m_shards(dev, g):
    """1M documents of the zipf-1m workload, its 10,000 queries at k = 10;
    the oracle checks a seeded sample of 40 queries."""
    from paper_2407_03618_gb300 import bm25
    w = synth.WORKLOADS["1m"]
    c, q = w.corpus(), w.queries()
    loc = shard.build_local(shard.GpuEngine(), c.tokens, c.doc_offsets, c.vocab, g, "lucene",
                            to_device=lambda a: _to(dev, a))
    full = bm25.Index.build(_to(dev, c.tokens), _to(dev, c.doc_offsets), c.vocab, "lucene")
    _check_shards(loc, full.export())
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.LUCENE, 1.5, 0.75, 0.5)
    sample = np.random.default_rng(31).choice(q.n_queries, 40, replace=False)
    _check_retrieval(dev, loc, full, orc, q, 10, sample)
    loc.close()
    full.close()


def test_merge_topk_padding_and_ties(dev):
    """bm25_merge_topk alone: empty slots (-1) are skipped, equal scores list
    the lower id first, rows shorter than k are padded with -1 / -inf."""
    from paper_2407_03618_gb300 import bm25
    ids = np.array([[[5, 9, -1, -1]], [[2, 7, 11, -1]], [[-1, -1, -1, -1]]], np.int32)
    sc = np.array([[[3.0, 1.0, -np.inf, -np.inf]], [[3.0, 1.0, 0.5, -np.inf]],
                   [[-np.inf] * 4]], np.float32)
    oid, osc = bm25.merge_topk(_to(dev, ids), _to(dev, sc), 4)
    assert oid.cpu().numpy().tolist() == [[2, 5, 7, 9]]
    assert osc.cpu().numpy().tolist() == [[3.0, 3.0, 1.0, 1.0]]
    oid, osc = bm25.merge_topk(_to(dev, ids[:1]), _to(dev, sc[:1]), 4)
    assert oid.cpu().numpy().tolist() == [[5, 9, -1, -1]]
    assert np.isneginf(osc.cpu().numpy()[0, 2:]).all()


def test_rescore_rejects_bad_ranges(dev):
    from paper_2407_03618_gb300 import bm25
    c = synth.make_corpus(100, 50, 1.1, ("poisson", 10), seed=1)
    ix = bm25.Index.build(_to(dev, c.tokens), _to(dev, c.doc_offsets), c.vocab)
    for args in ((None, 99, c.n_tokens, 0), (None, 150, c.n_tokens - 1, 0),
                 (None, 150, c.n_tokens, 51), (None, 150, c.n_tokens, -1)):
        with pytest.raises(bm25.BM25Error):
            ix.rescore(*args)
    ix.rescore(None, 150, c.n_tokens + 10, 50)  # a valid placement
    assert ix.shard_info()["doc_id_offset"] == 50
    ix.close()

"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Structure (|D|, TF, DF, indptr, indices) must be bit-exact; IDF and S0 are
FP64 on both sides; stored scores S - S0 and returned scores are FP32 and
must lie within 1e-5 of the oracle's scale; top-k ids must equal the
oracle's up to ties within that tolerance (oracle/compare.py).
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle.compare import check_topk
from paper_2407_03618_gb300 import synth

pytestmark = pytest.mark.gpu

VARIANTS = ["lucene", "robertson", "atire", "bm25l", "bm25+"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toy_corpus.json")
# accumulator plans every retrieval check runs under: all queries on the
# doc-tiled path, all on the dense path, and a split by postings count
PLANS = {"tiled": (2, 0), "dense": (3, 0), "mixed": (1, 3000)}


def _plan(ix, name):
    acc, dmax = PLANS[name]
    ix.set_plan(acc, 0, 0, dmax)


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def _to(dev, a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _build(dev, corpus, variant, k1=1.5, b=0.75, delta=0.5):
    from paper_2407_03618_gb300 import bm25
    return bm25.Index.build(_to(dev, corpus.tokens), _to(dev, corpus.doc_offsets), corpus.vocab,
                            variant, k1, b, delta)


def _check_structure(ix, orc, k1=1.5, b=0.75, delta=0.5):
    ex = ix.export()
    assert ex["nnz"] == orc.nnz
    assert np.array_equal(ex["doc_len"], orc.doc_len.astype(np.int32))
    assert np.array_equal(ex["df"], orc.df.astype(np.int32))
    assert np.array_equal(ex["indptr"], orc.indptr)
    assert np.array_equal(ex["indices"], orc.indices)
    assert np.array_equal(ex["tf"], orc.csc_tf)
    assert ex["lavg"] == pytest.approx(orc.lavg, rel=1e-15)
    np.testing.assert_allclose(ex["idf"], orc.idf, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ex["s0"], orc.s0, rtol=1e-13, atol=1e-15)
    # stored S - S0 in FP32: within 1e-5 of the term's full score scale
    full = orc.csc_delta + np.repeat(orc.s0, np.diff(orc.indptr))
    scale = np.maximum(np.abs(orc.csc_delta), np.abs(full))
    err = np.abs(ex["data"].astype(np.float64) - orc.csc_delta)
    assert (err <= 1e-5 * scale + 1e-30).all(), f"max rel err {np.max(err / (scale + 1e-300))}"
    return ex


def _check_retrieval(dev, ix, orc, queries, k, sample=None, where=""):
    ids, sc = ix.retrieve(_to(dev, queries.tokens), _to(dev, queries.offsets), k)
    ix.sync_status()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    qs = range(queries.n_queries) if sample is None else sample
    for q in qs:
        full, ab = oracle.score_all(orc, queries.query(q), with_abs=True)
        check_topk(ids[q], sc[q], full, ab, k, where=f"{where} q{q}")
    return ids, sc


# ------------------------------------------------------------- build -----

@pytest.mark.parametrize("variant", VARIANTS)
def test_toy_corpus_build_and_retrieve(torch_dev, variant):
    with open(GOLDEN) as f:
        g = json.load(f)
    docs = g["docs"]
    c = synth.Corpus(np.array([t for d in docs for t in d], np.int32),
                     synth.offsets_from_lengths(np.array([len(d) for d in docs])), g["vocab"])
    ix = _build(torch_dev, c, variant)
    ex = ix.export()
    assert ex["doc_len"].tolist() == g["doc_len"]
    assert ex["df"].tolist() == g["df"]
    assert ex["indptr"].tolist() == g["indptr"]
    assert ex["indices"].tolist() == g["indices"]
    np.testing.assert_allclose(ex["idf"], g["variants"][variant]["idf"], atol=5e-11)
    for case in g["variants"][variant]["queries"]:
        q = synth.Queries(np.array(case["q"], np.int32), np.array([0, len(case["q"])], np.int64))
        ids, sc = ix.retrieve(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), 3)
        ix.sync_status()
        assert ids.cpu().numpy()[0].tolist() == case["order"]
        np.testing.assert_allclose(sc.cpu().numpy()[0], np.array(case["B"])[case["order"]],
                                   rtol=1e-6, atol=1e-6)
    ix.close()


@pytest.mark.parametrize("seed", range(12))
def test_build_parity_random_small(torch_dev, seed):
    rng = np.random.default_rng(1000 + seed)
    c = synth.random_tiny_corpus(rng, max_docs=int(rng.integers(1, 400)),
                                 max_vocab=int(rng.integers(1, 3000)), max_len=40)
    variant = (VARIANTS + ["tfldp"])[seed % 6]
    k1, b, d = float(rng.uniform(0.3, 2.0)), float(rng.uniform(0, 1)), float(rng.uniform(0, 1))
    if variant == "tfldp":
        d = float(rng.uniform(0.38, 2.0))  # delta > 1/e
    ix = _build(torch_dev, c, variant, k1, b, d)
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.VARIANTS[variant], k1, b, d)
    _check_structure(ix, orc, k1, b, d)
    ix.close()


@pytest.mark.parametrize("delta", [0.5, 1.0, 0.5314, 2.0])
def test_tfldp_build_and_retrieve(torch_dev, delta):
    """TF_{l o delta o p} x IDF (Sec. 2.1's third shiftable model) on the tiny
    workload: negative S0 (delta = 0.5), S0 = IDF (delta = 1), S0 near 0
    (delta = e^(1/e - 1) ~ 0.5314), a large lower bound (delta = 2); every
    accumulator plan, k = 1, 10, 100."""
    w = synth.WORKLOADS["tiny"]
    c, q = w.corpus(), w.queries()
    ix = _build(torch_dev, c, "tfldp", 1.5, 0.75, delta)
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.TFLDP, 1.5, 0.75, delta)
    _check_structure(ix, orc, 1.5, 0.75, delta)
    for name in PLANS:
        _plan(ix, name)
        for k in (1, 10, 100):
            _check_retrieval(torch_dev, ix, orc, q, k, where=f"tfldp d={delta} {name} k={k}")
    ix.close()


def test_tfldp_rejects_small_delta(torch_dev):
    from paper_2407_03618_gb300 import bm25
    c = synth.Corpus(np.array([0, 1], np.int32), np.array([0, 2], np.int64), 2)
    with pytest.raises(bm25.BM25Error):
        _build(torch_dev, c, "tfldp", 1.2, 0.75, 0.3)  # 1 + ln 0.3 < 0


@pytest.mark.parametrize("variant", VARIANTS)
def test_tiny_workload_build_and_retrieve(torch_dev, variant):
    """2,000 docs, vocab 5,000, Zipf 1.1, Poisson(60); 100 queries; k=10."""
    w = synth.WORKLOADS["tiny"]
    c, q = w.corpus(), w.queries()
    ix = _build(torch_dev, c, variant)
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.VARIANTS[variant], 1.5, 0.75, 0.5)
    _check_structure(ix, orc)
    for name in PLANS:
        _plan(ix, name)
        for k in (1, 10, 100):
            _check_retrieval(torch_dev, ix, orc, q, k, where=f"{variant} {name} k={k}")
    ix.close()


def test_sort_spans_many_tiles_and_passes(torch_dev):
    """About 5.4M tokens = ~1,300 sort tiles of 4,096: more tiles than one wave
    of sort blocks, so each block walks several tiles in order and its range
    is counted by several upsweep blocks; a 300k vocabulary (19 bits) needing
    three radix passes; a ragged last tile."""
    c = synth.make_corpus(90_001, 300_000, 1.05, ("lognormal", 60, 0.6), seed=5)
    ix = _build(torch_dev, c, "lucene")
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, 0)
    _check_structure(ix, orc)
    ix.close()


# --------------------------------------------------------- retrieval -----

@pytest.mark.parametrize("tile_docs,threads,stage_entries,stages",
                         [(1024, 128, 512, 2), (2048, 256, 128, 8), (16384, 512, 4096, 3),
                          (4096, 512, 512, 2), (49152, 256, 256, 2), (3072, 192, 8192, 2),
                          (10240, 192, 1024, 4), (8192, 256, 2048, 3), (6144, 256, 1536, 2)])
def test_retrieval_across_tiles(torch_dev, tile_docs, threads, stage_entries, stages):
    """Small doc tiles force many (query, tile) items and a ragged last tile;
    staging rings from eight 1 KB buffers (an item spans many) to two 64 KB
    ones (a buffer holds several items' worth)."""
    c = synth.make_corpus(9_999, 3_000, 1.1, ("poisson", 30), seed=2)
    q = synth.make_queries(64, 3_000, 1.1, ("uniform", 0, 12), seed=3)
    ix = _build(torch_dev, c, "bm25+")
    ix.set_plan(2, tile_docs, threads, 0, stage_entries, stages)
    assert ix.get_plan() == {"accumulator": 2, "tile_docs": tile_docs, "block_threads": threads,
                             "dense_max_postings": 4096, "stage_entries": stage_entries,
                             "stages": stages}
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25PLUS)
    for k in (1, 7, 100, 1000, 2500):  # 2500: k' wider than the narrow tiles
        _check_retrieval(torch_dev, ix, orc, q, k, where=f"W={tile_docs} k={k}")
    ix.close()


@pytest.mark.parametrize("variant", ["robertson", "atire"])
def test_negative_and_zero_idf(torch_dev, variant):
    """Robertson IDF < 0 for common terms, so untouched documents (score 0)
    outrank matched ones; ATIRE IDF = 0 when DF = N."""
    rng = np.random.default_rng(11)
    n = 300
    lens = rng.integers(1, 12, n)
    tok = rng.integers(0, 6, int(lens.sum())).astype(np.int32)  # every term very common
    tok[::7] = 0
    c = synth.Corpus(tok, synth.offsets_from_lengths(lens), 6)
    ix = _build(torch_dev, c, variant)
    orc = oracle.build(c.tokens, c.doc_offsets, 6, oracle.VARIANTS[variant])
    if variant == "robertson":
        assert (orc.idf[:6] < 0).any()
    q = synth.random_queries(rng, 6, 40, 5)
    for name in PLANS:
        _plan(ix, name)
        for k in (5, 50, 299, 300):
            _check_retrieval(torch_dev, ix, orc, q, k, where=f"{variant} {name} k={k}")
    ix.close()


def test_edge_cases(torch_dev):
    """k > N, empty queries, duplicate tokens, DF = 0 terms, empty documents,
    a single document and a one-term vocabulary."""
    # empty docs, and terms 3,4 never occur
    c = synth.Corpus(np.array([0, 1, 1, 2, 0], np.int32), np.array([0, 0, 3, 3, 5, 5], np.int64), 5)
    for variant in VARIANTS:
        ix = _build(torch_dev, c, variant)
        orc = oracle.build(c.tokens, c.doc_offsets, 5, oracle.VARIANTS[variant])
        _check_structure(ix, orc)
        q = synth.Queries(np.array([1, 1, 0, 3, 4, 4, 2], np.int32),
                          np.array([0, 0, 3, 5, 7], np.int64))  # empty, dups, DF=0, mixed
        for name in PLANS:
            _plan(ix, name)
            for k in (1, 3, 5, 9):
                _check_retrieval(torch_dev, ix, orc, q, k, where=f"{variant} {name} edge k={k}")
        ix.close()
    one = synth.Corpus(np.array([0, 0, 0], np.int32), np.array([0, 3], np.int64), 1)
    ix = _build(torch_dev, one, "lucene")
    orc = oracle.build(one.tokens, one.doc_offsets, 1, 0)
    q = synth.Queries(np.array([0], np.int32), np.array([0, 1, 1], np.int64))
    _check_retrieval(torch_dev, ix, orc, q, 4, where="single doc")
    ix.close()
    # a corpus of empty documents only
    e = synth.Corpus(np.zeros(0, np.int32), np.zeros(4, np.int64), 3)
    ix = _build(torch_dev, e, "bm25l")
    assert ix.info()["nnz"] == 0
    ids, sc = ix.retrieve(_to(torch_dev, np.array([1], np.int32)),
                          _to(torch_dev, np.array([0, 1], np.int64)), 2)
    ix.sync_status()
    assert ids.cpu().numpy().tolist() == [[0, 1]]
    assert sc.cpu().numpy().tolist() == [[0.0, 0.0]]
    ix.close()


def test_exact_ties_at_the_threshold_across_tiles(torch_dev):
    """30,011 documents in two classes of identical documents ([0, 1], and
    [0, 0, 2] for every fifth): every score ties exactly with its whole class,
    and the classes lie >= 8 % apart.  The top k is then unique — the class
    order, lowest doc ids first — and must come back exactly, across many doc
    tiles (a ragged last one) where the running threshold sits on the tied
    score: the crossing mode (Lucene, BM25+ with its shift) and the list mode
    with untouched documents ranking (Robertson, negative IDF of term 0)."""
    n = 30_011
    toks, offs = [], [0]
    for i in range(n):
        toks += [0, 0, 2] if i % 5 == 3 else [0, 1]
        offs.append(len(toks))
    c = synth.Corpus(np.array(toks, np.int32), np.array(offs, np.int64), 3)
    qlist = [[0], [1], [2], [0, 1], [1, 2], [0, 2], [2, 2, 1]]
    q = synth.Queries(np.array(sum(qlist, []), np.int32),
                      np.concatenate([[0], np.cumsum([len(x) for x in qlist])]).astype(np.int64))
    plans = {"tiled W=1024": (2, 1024, 0), "tiled": (2, 0, 0), "dense": (3, 0, 0),
             "mixed": (1, 0, 20_000)}
    for variant in ("lucene", "bm25+", "robertson"):
        ix = _build(torch_dev, c, variant)
        orc = oracle.build(c.tokens, c.doc_offsets, 3, oracle.VARIANTS[variant], 1.5, 0.75, 0.5)
        want = []
        for i in range(q.n_queries):
            full = oracle.score_all(orc, q.query(i))
            want.append((np.lexsort((np.arange(n), -full)), full))
        for name, (acc, w, dmax) in plans.items():
            ix.set_plan(acc, w, 0, dmax)
            for k in (1, 10, 100, 1000, 4096):
                ids, sc = ix.retrieve(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), k)
                ix.sync_status()
                ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
                for i in range(q.n_queries):
                    order, full = want[i]
                    where = f"{variant} {name} k={k} q{qlist[i]}"
                    assert np.array_equal(ids[i], order[:k]), where
                    np.testing.assert_allclose(sc[i], full[order[:k]], rtol=1e-5, atol=0.0,
                                               err_msg=where)
        ix.close()


def test_out_of_range_tokens_are_reported(torch_dev):
    from paper_2407_03618_gb300 import bm25
    c = synth.Corpus(np.array([0, 1, 2, 1], np.int32), np.array([0, 2, 4], np.int64), 3)
    bad = synth.Corpus(np.array([0, 1, 7, 1], np.int32), c.doc_offsets, 3)
    with pytest.raises(bm25.BM25Error) as e:
        _build(torch_dev, bad, "lucene")
    assert e.value.code == -2
    neg = synth.Corpus(np.array([0, -1, 2, 1], np.int32), c.doc_offsets, 3)
    with pytest.raises(bm25.BM25Error):
        _build(torch_dev, neg, "lucene")
    badoff = synth.Corpus(c.tokens, np.array([0, 3, 2], np.int64), 3)
    with pytest.raises(bm25.BM25Error):
        _build(torch_dev, badoff, "lucene")
    ix = _build(torch_dev, c, "lucene")
    ids, sc = ix.retrieve(_to(torch_dev, np.array([1, 9, -3], np.int32)),
                          _to(torch_dev, np.array([0, 3], np.int64)), 2)
    with pytest.raises(bm25.BM25Error) as e:
        ix.sync_status()
    assert e.value.code == -2
    ix.sync_status()  # the status word was cleared
    # the valid token still scored
    orc = oracle.build(c.tokens, c.doc_offsets, 3, 0)
    full, ab = oracle.score_all(orc, [1], with_abs=True)
    check_topk(ids.cpu().numpy()[0], sc.cpu().numpy()[0], full, ab, 2)
    ix.close()


def test_host_entry_points_and_checkpoint(torch_dev):
    from paper_2407_03618_gb300 import bm25
    w = synth.WORKLOADS["tiny"]
    c, q = w.corpus(), w.queries()
    ix = _build(torch_dev, c, "bm25l")
    ih = bm25.Index.build_host(c.tokens, c.doc_offsets, c.vocab, "bm25l")
    a, b_ = ix.export(), ih.export()
    for key in ("indptr", "indices", "tf", "df", "doc_len", "idf", "s0", "data"):
        assert np.array_equal(a[key], b_[key]), key
    # FP32 atomic accumulation order varies between runs, so each path is
    # held to the oracle rather than to the other bit for bit
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25L)
    im = bm25.Index.load_arrays(a)  # export -> import (checkpoint resume)
    ids_d, sc_d = ix.retrieve(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), 10)
    ids_h, sc_h = ih.retrieve_host(q.tokens, q.offsets, 10)
    ids_i, sc_i = im.retrieve(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), 10)
    im.sync_status()
    results = [(ids_d.cpu().numpy(), sc_d.cpu().numpy()), (ids_h, sc_h),
               (ids_i.cpu().numpy(), sc_i.cpu().numpy())]
    for i in range(q.n_queries):
        full, ab = oracle.score_all(orc, q.query(i), with_abs=True)
        for name, (ids, sc) in zip(("device", "host", "imported"), results):
            check_topk(ids[i], sc[i], full, ab, 10, where=f"{name} q{i}")
    for x in (ix, ih, im):
        x.close()


def test_workspace_and_bad_retrieve_args(torch_dev):
    from paper_2407_03618_gb300 import bm25
    w = synth.WORKLOADS["tiny"]
    c, q = w.corpus(), w.queries()
    ix = _build(torch_dev, c, "lucene")
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, 0)
    ws = bm25.Workspace(ix, q.n_queries, q.tokens.shape[0], 10)
    ids, sc = ix.retrieve(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), 10, workspace=ws,
                          plan={"accumulator": bm25.ACC_SMEM_TILED, "tile_docs": 1024,
                                "block_threads": 128})
    ix.sync_status()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for i in range(q.n_queries):
        full, ab = oracle.score_all(orc, q.query(i), with_abs=True)
        check_topk(ids[i], sc[i], full, ab, 10)
    for k in (0, -3):
        with pytest.raises(bm25.BM25Error):
            ix.retrieve(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), k)
    with pytest.raises(bm25.BM25Error):
        ix.set_plan(0, 1000)
    with pytest.raises(bm25.BM25Error):
        ix.set_plan(0, 0, 96)
    ws.close()
    ix.close()


# ------------------------------------------------ batches and plans -----

def _check_rows(ids, sc, orc, queries, ks, n_docs, where):
    """Row q: the oracle's top min(k_q, N), then -1 / -inf to the row's end."""
    for q in range(queries.n_queries):
        kp = min(int(ks[q]), n_docs)
        full, ab = oracle.score_all(orc, queries.query(q), with_abs=True)
        check_topk(ids[q, :kp], sc[q, :kp], full, ab, kp, where=f"{where} q{q}")
        assert (ids[q, kp:] == -1).all() and np.isneginf(sc[q, kp:]).all(), f"{where} q{q} tail"


@pytest.mark.parametrize("name", list(PLANS))
def test_per_query_k_in_one_call(torch_dev, name):
    """Queries with k in {1, 10, 100, 1000} mixed in one call; rows are
    k_max wide."""
    c = synth.make_corpus(20_000, 8_000, 1.1, ("poisson", 40), seed=21)
    q = synth.make_queries(150, 8_000, 1.1, ("uniform", 0, 20), seed=22)
    ix = _build(torch_dev, c, "bm25l")
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25L)
    _plan(ix, name)
    ks = np.random.default_rng(5).choice([1, 10, 100, 1000], q.n_queries).astype(np.int32)
    ids, sc = ix.retrieve_batch(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), 1000,
                                q_k=_to(torch_dev, ks))
    ix.sync_status()
    _check_rows(ids.cpu().numpy(), sc.cpu().numpy(), orc, q, ks, c.n_docs, f"{name} per-k")
    # an entry outside [1, k_max] is reported through the status word
    from paper_2407_03618_gb300 import bm25
    bad = ks.copy()
    bad[3] = 1001
    ix.retrieve_batch(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), 1000,
                      q_k=_to(torch_dev, bad))
    with pytest.raises(bm25.BM25Error) as e:
        ix.sync_status()
    assert e.value.code == -1
    ix.close()


@pytest.mark.parametrize("name", list(PLANS))
def test_long_queries_span_token_chunks(torch_dev, name):
    """Queries of 60..200 tokens (more than one 64-token chunk)."""
    c = synth.make_corpus(6_000, 4_000, 1.1, ("poisson", 30), seed=31)
    q = synth.make_queries(40, 4_000, 1.1, ("uniform", 60, 200), 50, seed=32)
    ix = _build(torch_dev, c, "lucene")
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.LUCENE)
    _plan(ix, name)
    ix.set_plan(0, 2048, 256)
    for k in (10, 300):
        _check_retrieval(torch_dev, ix, orc, q, k, where=f"{name} long k={k}")
    ix.close()


def test_sub_batches_when_candidates_exceed_the_budget(torch_dev):
    """k = 4096 over 196 doc tiles of 1024 needs 6.4 MB of tile candidates per
    query, so 800 queries run as three sub-batches of at most 2 GiB."""
    c = synth.make_corpus(200_000, 30_000, 1.05, ("poisson", 12), seed=41)
    q = synth.make_queries(800, 30_000, 1.05, ("uniform", 1, 6), 100, seed=42)
    ix = _build(torch_dev, c, "lucene")
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.LUCENE)
    ix.set_plan(2, 1024, 256)
    ids, sc = ix.retrieve(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), 4096)
    ix.sync_status()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for i in [0, 1, 334, 335, 336, 669, 670, 671, 799] + list(range(100, 800, 97)):
        full, ab = oracle.score_all(orc, q.query(i), with_abs=True)
        check_topk(ids[i], sc[i], full, ab, 4096, where=f"sub-batch q{i}")
    ix.close()


@pytest.mark.parametrize("k", [100, 1000, 2500])
def test_merge_tree_for_large_k(torch_dev, k):
    """Six queries over 98 doc tiles of 1024: all their tiles run in the first
    wave with no threshold, so each hands over its k' best, and the merge tree
    cuts groups of tiles to their k' best in place before the final merge
    (groups of 81, 8 and 3 tiles: one, two and five levels, with ragged last
    groups and groups of one tile).  Also per-query k below the row width."""
    c = synth.make_corpus(100_000, 20_000, 1.05, ("poisson", 20), seed=61)
    q = synth.make_queries(6, 20_000, 1.05, ("uniform", 2, 8), seed=62)
    ix = _build(torch_dev, c, "lucene")
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.LUCENE)
    ix.set_plan(2, 1024, 256)
    _check_retrieval(torch_dev, ix, orc, q, k, where=f"tree k={k}")
    ks = np.array([1, k, 7, k // 2, 100, 3], np.int32)
    ids, sc = ix.retrieve_batch(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), k,
                                q_k=_to(torch_dev, ks))
    ix.sync_status()
    _check_rows(ids.cpu().numpy(), sc.cpu().numpy(), orc, q, ks, c.n_docs, f"tree per-k k={k}")
    if k == 2500:  # past the largest k' (BM25_MAX_K = 4096) the call is refused on the host
        from paper_2407_03618_gb300 import bm25
        with pytest.raises(bm25.BM25Error):
            ix.retrieve(_to(torch_dev, q.tokens), _to(torch_dev, q.offsets), 4097)
    ix.close()


@pytest.mark.parametrize("name", ["tiled", "mixed"])
def test_cuda_graph_capture_and_replay(torch_dev, name):
    """A reserved workspace lets a call be captured in a CUDA graph; replays
    on new query contents of the same shape give the oracle's results."""
    import torch
    from paper_2407_03618_gb300 import bm25
    w = synth.WORKLOADS["tiny"]
    c = w.corpus()
    ix = _build(torch_dev, c, "bm25+")
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25PLUS)
    _plan(ix, name)
    qa = synth.make_queries(64, c.vocab, 1.1, ("uniform", 4, 4), seed=51)
    qb = synth.make_queries(64, c.vocab, 1.1, ("uniform", 4, 4), seed=52)
    assert np.array_equal(qa.offsets, qb.offsets)
    qt = _to(torch_dev, qa.tokens)
    qo = _to(torch_dev, qa.offsets)
    ks = torch.full((64,), 10, dtype=torch.int32, device=torch_dev)
    ids = torch.empty((64, 10), dtype=torch.int32, device=torch_dev)
    sc = torch.empty((64, 10), dtype=torch.float32, device=torch_dev)
    ws = bm25.Workspace(ix, 64, qt.numel(), 10)
    s = torch.cuda.Stream()
    ws.reserve(ix, 64, qt.numel(), 10, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        ix.retrieve_batch(qt, qo, 10, q_k=ks, out=(ids, sc), workspace=ws, stream=s)
    for qq in (qa, qb, qa):
        qt.copy_(_to(torch_dev, qq.tokens))
        g.replay()
        torch.cuda.synchronize()
        ix.sync_status()
        _check_rows(ids.cpu().numpy(), sc.cpu().numpy(), orc, qq, np.full(64, 10), c.n_docs,
                    f"graph {name}")
    # capturing a call the workspace is too small for fails instead of allocating
    small = bm25.Workspace(ix, 1, 1, 1)
    g2 = torch.cuda.CUDAGraph()
    with pytest.raises(bm25.BM25Error):
        with torch.cuda.graph(g2, stream=s, capture_error_mode="thread_local"):
            ix.retrieve_batch(qt, qo, 10, out=(ids, sc), workspace=small, stream=s)
    del g, g2
    ws.close()
    small.close()
    ix.close()


def test_default_workspace_reused_across_indexes(torch_dev):
    """A freed index's default workspace serves the next index built on the
    device (one kept per device): indexes of larger, smaller and equal size in
    turn, each through bm25_retrieve and bm25_retrieve_host with dense and
    tiled queries, all give the oracle's results; then the cache is freed."""
    from paper_2407_03618_gb300 import bm25
    shapes = [(3000, 2000, 1.1, ("poisson", 40)), (9000, 4000, 1.05, ("poisson", 30)),
              (1500, 1000, 1.2, ("poisson", 50)), (3000, 2000, 1.1, ("poisson", 40))]
    for i, (n, v, s_, L) in enumerate(shapes):
        c = synth.make_corpus(n, v, s_, L, seed=60 + i)
        q = synth.make_queries(48, v, s_, ("uniform", 1, 10), seed=70 + i)
        orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25PLUS)
        ix = _build(torch_dev, c, "bm25+")
        ix.set_plan(1, 0, 0, 600)  # short queries dense, the rest tiled
        _check_retrieval(torch_dev, ix, orc, q, 10, where=f"index {i} device")
        ids, sc = ix.retrieve_host(q.tokens, q.offsets, 7)
        ix.sync_status()
        for r in range(q.n_queries):
            full, ab = oracle.score_all(orc, q.query(r), with_abs=True)
            check_topk(ids[r], sc[r], full, ab, 7, where=f"index {i} host q{r}")
        ix.close()
    bm25.release_cached()

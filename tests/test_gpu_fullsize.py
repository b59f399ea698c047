"""Full-size parity, in the launch configuration the benchmark times (one
batched call over each workload's whole query batch).

zipf-1m: 1,000,000 documents, vocab 200,000 Zipf(1.05), lognormal(60, 0.6)
lengths; 10,000 queries of 1..16 tokens with the 100 head terms removed;
k = 10 and 100; all five variants.  Structure (|D|, TF, DF, indptr, indices)
is compared in full against the oracle's; scores S - S0 in full within 1e-5
of their scale; the top-k of a seeded sample of queries against the oracle's
lazy exhaustive scores; and, for Lucene at k = 10, every one of the 10,000
queries against the oracle's own top 42 (lazy exhaustive, all host cores).
"""
import os

import numpy as np
import pytest

import oracle
from oracle.compare import check_topk, check_topk_with_list
from paper_2407_03618_gb300 import synth

THREADS = os.cpu_count() or 1

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

VARIANTS = ["lucene", "robertson", "atire", "bm25l", "bm25+"]
N_SAMPLE = 24


@pytest.fixture(scope="module")
def workload():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    w = synth.WORKLOADS["1m"]
    c, q = w.corpus(), w.queries()
    dev = torch.device("cuda:0")
    return {"w": w, "c": c, "q": q, "dev": dev,
            "tok": torch.from_numpy(c.tokens).to(dev),
            "off": torch.from_numpy(c.doc_offsets).to(dev),
            "qt": torch.from_numpy(q.tokens).to(dev),
            "qo": torch.from_numpy(q.offsets).to(dev),
            "sample": np.random.default_rng(123).choice(q.n_queries, N_SAMPLE, replace=False)}


@pytest.mark.parametrize("variant", VARIANTS)
def test_fullsize_parity(workload, variant):
    from paper_2407_03618_gb300 import bm25
    W = workload
    c, q, prm = W["c"], W["q"], W["w"].params
    ix = bm25.Index.build(W["tok"], W["off"], c.vocab, variant, prm["k1"], prm["b"], prm["delta"])
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.VARIANTS[variant], prm["k1"],
                       prm["b"], prm["delta"])
    ex = ix.export()
    assert ex["nnz"] == orc.nnz
    assert np.array_equal(ex["doc_len"], orc.doc_len.astype(np.int32))
    assert np.array_equal(ex["df"], orc.df.astype(np.int32))
    assert np.array_equal(ex["indptr"], orc.indptr)
    assert np.array_equal(ex["indices"], orc.indices)
    assert np.array_equal(ex["tf"], orc.csc_tf)
    np.testing.assert_allclose(ex["idf"], orc.idf, rtol=1e-13, atol=1e-15)
    full_s = orc.csc_delta + np.repeat(orc.s0, np.diff(orc.indptr))
    scale = np.maximum(np.abs(orc.csc_delta), np.abs(full_s))
    assert (np.abs(ex["data"] - orc.csc_delta) <= 1e-5 * scale + 1e-30).all()
    del ex, full_s, scale
    for k in (10, 100):
        ids, sc = ix.retrieve(W["qt"], W["qo"], k)
        ix.sync_status()
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        for i in W["sample"]:
            full, ab = oracle.score_all(orc, q.query(int(i)), with_abs=True)
            check_topk(ids[i], sc[i], full, ab, k, where=f"{variant} k={k} q{i}")
        if variant == "lucene" and k == 10:  # every query of the batch
            top_ids, top_sc = oracle.topk(orc, q.tokens, q.offsets, k + 32, n_threads=THREADS)
            for i in range(q.n_queries):
                check_topk_with_list(ids[i], sc[i], top_ids[i], top_sc[i], k, c.n_docs,
                                     where=f"all {variant} k={k} q{i}")
    ix.close()


# ---- the passage and long-document shapes ------------------------------------
# passage-8.8m at full size: 8.8M documents (lognormal(56, 0.5)), vocab 1M
# Zipf(1.0), ~433M CSC entries, 7,000 queries of geometric length (mean 6, at
# most 32) with head terms, k = 10 / 100 / 1000 in the batched launch the
# bench times; structure bit-exact in full, stored scores on sampled columns,
# the top 10 of a seeded sample of 200 queries against the oracle's top 42
# and the top 100 / 1000 of 8 of them against its exhaustive scores.
# long-5m at full size: 5M documents of lognormal(300, 0.8) lengths, vocab 2M
# Zipf(1.1), ~0.9G CSC entries, 5,000 queries of 20..60 tokens including head
# terms, BM25+ with its shift, k = 100; structure bit-exact in full, the top
# 100 of a seeded sample of 40 queries against the oracle's top 164.

@pytest.mark.parametrize("name", ["passage", "long"])
def test_large_shapes(name):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03618_gb300 import bm25
    w = synth.WORKLOADS[name]
    dev = torch.device("cuda:0")
    c, q = w.corpus(), w.queries()
    if name == "passage":
        variant, ks, n_list, n_full = "lucene", (10, 100, 1000), 200, 8
    else:
        variant, ks, n_list, n_full = "bm25+", (100,), 40, 0
    prm = w.params
    ix = bm25.Index.build(torch.from_numpy(c.tokens).to(dev),
                          torch.from_numpy(c.doc_offsets).to(dev), c.vocab, variant,
                          prm["k1"], prm["b"], prm["delta"])
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.VARIANTS[variant], prm["k1"],
                       prm["b"], prm["delta"])
    info = ix.info()
    assert info["nnz"] == orc.nnz
    # the structure in full (bit-exact), the stored scores on sampled columns
    for key, want in (("df", orc.df.astype(np.int32)), ("indptr", orc.indptr),
                      ("doc_len", orc.doc_len.astype(np.int32)), ("indices", orc.indices),
                      ("tf", orc.csc_tf)):
        got = ix.export([key])[key]
        assert np.array_equal(got, want), key
        del got
    data = ix.export(["data"])["data"]
    rng = np.random.default_rng(5)
    cols = np.unique(np.concatenate([np.arange(20), rng.integers(0, c.vocab, 200)]))
    for t in cols:  # the head terms and a random sample
        a, b = orc.indptr[t], orc.indptr[t + 1]
        full_s = orc.csc_delta[a:b] + orc.s0[t]
        scale = np.maximum(np.abs(orc.csc_delta[a:b]), np.abs(full_s))
        assert (np.abs(data[a:b] - orc.csc_delta[a:b]) <= 1e-5 * scale + 1e-30).all()
    del data
    qt = torch.from_numpy(q.tokens).to(dev)
    qo = torch.from_numpy(q.offsets).to(dev)
    sample = rng.choice(q.n_queries, n_list, replace=False)
    rows = {}
    for k in ks:
        ids, sc = ix.retrieve(qt, qo, k)
        ix.sync_status()
        rows[k] = (ids.cpu().numpy()[sample], sc.cpu().numpy()[sample])
    ix.close()
    sub = q.subset(sample)
    k0 = ks[0]
    top_ids, top_sc = oracle.topk(orc, sub.tokens, sub.offsets, k0 + max(32, k0 * 64 // 100),
                                  n_threads=THREADS)
    for j, i in enumerate(sample):
        check_topk_with_list(rows[k0][0][j], rows[k0][1][j], top_ids[j], top_sc[j], k0,
                             c.n_docs, where=f"{name} k={k0} q{i}")
    for j, i in enumerate(sample[:n_full]):
        full, ab = oracle.score_all(orc, q.query(int(i)), with_abs=True)
        for k in ks[1:]:
            check_topk(rows[k][0][j], rows[k][1][j], full, ab, k, where=f"{name} k={k} q{i}")

"""Full-size parity on the 1M-document workload, in the launch configuration
the benchmark times (one batched call over all 10,000 queries).

1,000,000 documents, vocab 200,000 Zipf(1.05), lognormal(60, 0.6) lengths;
10,000 queries of 1..16 tokens with the 100 head terms removed; k = 10 and
100; all five variants.  Structure (|D|, TF, DF, indptr, indices) is compared
in full against the oracle's; scores S - S0 in full within 1e-5 of their
scale; the top-k of a seeded sample of queries against the oracle's lazy
exhaustive scores (each oracle query scores all 1M documents).
"""
import numpy as np
import pytest

import oracle
from oracle.compare import check_topk
from paper_2407_03618_gb300 import synth

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
    ix.close()

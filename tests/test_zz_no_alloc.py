"""bm25_retrieve_noalloc: retrieval for callers that cannot allocate device
memory (its scratch is a fixed device array inside the library).

Called through the C ABI directly, twice in a row on different batches, and
compared with bm25_retrieve on the same inputs (the same ids up to ties
within the tolerance of the other parity tests, and scores within it) and
with the FP64 oracle (check_topk), so that a mistake both paths shared would
still fail.  Kept in a file of its own that pytest collects last; it passes
alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle.compare import RTOL, check_topk
from paper_2407_03618_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, ix, qt, qo, k, torch):
    nq = qo.numel() - 1
    ids = torch.full((nq, k), -7, dtype=torch.int32, device=qt.device)
    sc = torch.full((nq, k), 7.0, dtype=torch.float32, device=qt.device)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.bm25_retrieve_noalloc(ix.handle, ctypes.c_void_p(qt.data_ptr()), qt.numel(),
                                   ctypes.c_void_p(qo.data_ptr()), nq, k,
                                   ctypes.c_void_p(ids.data_ptr()),
                                   ctypes.c_void_p(sc.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0, lib.bm25_last_error()
    return ids, sc


def _same_result(ids_a, sc_a, ids_b, sc_b):
    """Scores within RTOL of each other; ids equal except where the two sides
    hold equal-within-tolerance scores (FP32 sums in another order)."""
    np.testing.assert_allclose(sc_a, sc_b, rtol=RTOL, atol=RTOL)
    for r in range(ids_a.shape[0]):
        for i in np.nonzero(ids_a[r] != ids_b[r])[0]:
            assert abs(sc_a[r, i] - sc_b[r, i]) <= RTOL * max(1.0, abs(sc_a[r, i]))
        assert set(ids_a[r][sc_a[r] > sc_a[r, -1] + RTOL * max(1.0, abs(sc_a[r, -1]))]) <= \
            set(ids_b[r])


def test_noalloc_matches_retrieve_twice():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03618_gb300 import bm25
    lib = bm25.load()
    dev = torch.device("cuda:0")
    c = synth.make_corpus(30_000, 20_000, 1.05, ("lognormal", 60, 0.6), seed=0)
    ix = bm25.Index.build(torch.from_numpy(c.tokens).to(dev),
                          torch.from_numpy(c.doc_offsets).to(dev), c.vocab, "bm25+")
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25PLUS, 1.5, 0.75, 0.5)
    for call, (seed, k) in enumerate([(1, 10), (2, 100)]):
        q = synth.make_queries(200, 20_000, 1.05, ("uniform", 1, 16), 10, seed=seed)
        qt = torch.from_numpy(q.tokens).to(dev)
        qo = torch.from_numpy(q.offsets).to(dev)
        ids_n, sc_n = _noalloc(lib, ix, qt, qo, k, torch)
        ids_r, sc_r = ix.retrieve(qt, qo, k)
        ix.sync_status()
        ids_n, sc_n = ids_n.cpu().numpy(), sc_n.cpu().numpy()
        _same_result(ids_n, sc_n, ids_r.cpu().numpy(), sc_r.cpu().numpy())
        for i in range(q.n_queries):
            full, ab = oracle.score_all(orc, q.query(i), with_abs=True)
            check_topk(ids_n[i], sc_n[i], full, ab, k, where=f"noalloc call {call} q{i}")
    # a batch beyond the fixed scratch is refused with a clear message
    big = synth.make_queries(20_000, 20_000, 1.05, ("uniform", 8, 16), 10, seed=3)
    qt = torch.from_numpy(big.tokens).to(dev)
    qo = torch.from_numpy(big.offsets).to(dev)
    out = torch.empty((big.n_queries, 100), dtype=torch.int32, device=dev)
    outs = torch.empty((big.n_queries, 100), dtype=torch.float32, device=dev)
    rc = lib.bm25_retrieve_noalloc(ix.handle, ctypes.c_void_p(qt.data_ptr()), qt.numel(),
                                   ctypes.c_void_p(qo.data_ptr()), big.n_queries, 100,
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(outs.data_ptr()), None)
    assert rc == -1
    assert b"scratch" in lib.bm25_last_error()
    ix.close()

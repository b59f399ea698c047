"""Failure paths on the GPU, made to happen without faulting anything.

* A bounded device-side wait that runs out: the producer/consumer waits of
  the doc-tiled retrieval kernel are given a poll limit of 0 (a test hook),
  so each gives up at once.  The kernel must record BM25_E_TIMEOUT in the
  index's status word (seen through bm25_sync_status), wait for its own bulk
  copies and return; the next call with the normal limit must match the
  oracle, so the context, the index and the workspace stay usable.
* A device allocation that fails: a test hook makes the library's next
  allocation report out-of-memory; the build or retrieval that needed it
  must fail with BM25_E_OOM and nothing else, and the same call must succeed
  afterwards.
"""
import numpy as np
import pytest

import oracle
from oracle.compare import check_topk
from paper_2407_03618_gb300 import synth

pytestmark = pytest.mark.gpu

E_OOM, E_TIMEOUT = -3, -5


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03618_gb300 import bm25
    dev = torch.device("cuda:0")
    c = synth.make_corpus(40_000, 8_000, 1.1, ("poisson", 40), seed=3)
    q = synth.make_queries(64, 8_000, 1.1, ("uniform", 1, 8), seed=4)
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.LUCENE, 1.5, 0.75, 0.5)
    t = {"tok": torch.from_numpy(c.tokens).to(dev), "off": torch.from_numpy(c.doc_offsets).to(dev),
         "qt": torch.from_numpy(q.tokens).to(dev), "qo": torch.from_numpy(q.offsets).to(dev)}
    yield {"bm25": bm25, "c": c, "q": q, "orc": orc, "dev": dev, **t}
    bm25.debug_set_handshake_polls(-1)
    bm25.debug_fail_allocs(0)


def _check_all(env, ids, sc, k):
    if hasattr(ids, "cpu"):
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for i in range(env["q"].n_queries):
        full, ab = oracle.score_all(env["orc"], env["q"].query(i), with_abs=True)
        check_topk(ids[i], sc[i], full, ab, k, where=f"q{i}")


def _build(env):
    return env["bm25"].Index.build(env["tok"], env["off"], env["c"].vocab, "lucene", 1.5, 0.75,
                                   0.5)


def test_wait_gives_up_then_library_usable(env):
    bm25 = env["bm25"]
    ix = _build(env)
    ix.set_plan(bm25.ACC_SMEM_TILED, 0, 0, 0)  # every query through the tiled kernel
    for k in (10, 100):
        bm25.debug_set_handshake_polls(0)
        try:
            ix.retrieve(env["qt"], env["qo"], k)
            with pytest.raises(bm25.BM25Error) as e:
                ix.sync_status()
            assert e.value.code == E_TIMEOUT, str(e.value)
        finally:
            bm25.debug_set_handshake_polls(-1)
        ix.sync_status()  # the status was cleared by the read above
        ids, sc = ix.retrieve(env["qt"], env["qo"], k)
        ix.sync_status()
        _check_all(env, ids, sc, k)
    ix.close()


def test_forced_oom_in_build_then_build_works(env):
    bm25 = env["bm25"]
    for n_fail in (1, 3):
        bm25.debug_fail_allocs(n_fail)
        try:
            with pytest.raises(bm25.BM25Error) as e:
                _build(env)
            assert e.value.code == E_OOM, str(e.value)
        finally:
            bm25.debug_fail_allocs(0)
    ix = _build(env)
    ids, sc = ix.retrieve(env["qt"], env["qo"], 10)
    ix.sync_status()
    _check_all(env, ids, sc, 10)
    ix.close()


def test_forced_oom_in_retrieval_then_retrieval_works(env):
    bm25 = env["bm25"]
    bm25.release_cached()  # the next index's workspace must be allocated afresh
    ix = _build(env)
    bm25.debug_fail_allocs(1)
    try:
        with pytest.raises(bm25.BM25Error) as e:
            ix.retrieve(env["qt"], env["qo"], 10)
        assert e.value.code == E_OOM, str(e.value)
    finally:
        bm25.debug_fail_allocs(0)
    ids, sc = ix.retrieve(env["qt"], env["qo"], 10)
    ix.sync_status()
    _check_all(env, ids, sc, 10)
    # the host-buffer path's staging allocation fails the same way
    bm25.release_cached()
    ix2 = _build(env)
    q = env["q"]
    bm25.debug_fail_allocs(1)
    try:
        with pytest.raises(bm25.BM25Error) as e:
            ix2.retrieve_host(q.tokens, q.offsets, 10)
        assert e.value.code == E_OOM, str(e.value)
    finally:
        bm25.debug_fail_allocs(0)
    hid, hsc = ix2.retrieve_host(q.tokens, q.offsets, 10)
    _check_all(env, np.asarray(hid), np.asarray(hsc), 10)
    ix2.close()
    ix.close()

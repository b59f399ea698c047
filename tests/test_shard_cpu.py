"""Doc-range sharding on the CPU: two gloo ranks run the real build and
query path of paper_2407_03618_gb300/shard.py (all-gather of the shards'
sizes, all-reduce of DF, all-gather of the rows, merge) with the FP64 oracle
as the shard engine, and the merged top k must equal the oracle's top k
over the unsplit collection exactly (same FP64 arithmetic on the same
inputs: IDF from the summed DF and N, Lavg from the summed token count).
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2407_03618_gb300 import shard, synth


class OracleEngine:
    """The oracle behind the engine interface shard.py drives.  Rescoring
    replaces the shard's IDF (oracle.idf of the summed DF and N) and Lavg;
    the lazy exhaustive scoring then runs the oracle's own arithmetic."""

    def build(self, tokens, doc_offsets, vocab, variant, k1, b, delta):
        ix = oracle.build(np.asarray(tokens), np.asarray(doc_offsets), vocab,
                          oracle.VARIANTS[variant], k1, b, delta)
        return {"ix": ix, "offset": 0}

    def df(self, sh):
        import torch
        return torch.from_numpy(sh["ix"].df.astype(np.int32))

    def counts(self, sh):
        return sh["ix"].n_docs, int(sh["ix"].doc_len.sum())

    def count_tensor(self, sh):
        import torch
        return torch.tensor(list(self.counts(sh)), dtype=torch.int64)

    def rescore(self, sh, global_df, n_docs, n_tokens, doc_offset):
        ix = sh["ix"]
        ix.idf = np.array([oracle.idf(ix.variant, n_docs, int(d)) for d in global_df.tolist()])
        ix.lavg = n_tokens / n_docs
        sh["offset"] = doc_offset

    def retrieve(self, sh, q_tokens, q_offsets, k):
        import torch
        ids, sc = oracle.topk(sh["ix"], np.asarray(q_tokens), np.asarray(q_offsets), k)
        ids = np.where(ids >= 0, ids + sh["offset"], -1)
        return torch.from_numpy(ids), torch.from_numpy(sc)

    def merge(self, cand_ids, cand_scores, k):
        ci, cs = cand_ids.numpy(), cand_scores.numpy()
        g, nq, _ = ci.shape
        ids = np.full((nq, k), -1, np.int64)
        sc = np.full((nq, k), -np.inf)
        for q in range(nq):
            i, s = ci[:, q, :].ravel(), cs[:, q, :].ravel()
            ok = i >= 0
            i, s = i[ok], s[ok]
            order = np.lexsort((i, -s))[:k]
            ids[q, :order.shape[0]] = i[order]
            sc[q, :order.shape[0]] = s[order]
        return ids, sc


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _corpus():
    return synth.make_corpus(1_001, 300, 1.1, ("poisson", 20), seed=9)


def _queries():
    return synth.make_queries(40, 300, 1.1, ("uniform", 1, 6), seed=10)


def _worker(rank, world, port, variant, k, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c, q = _corpus(), _queries()
        lo, hi = shard.doc_ranges(c.n_docs, world)[rank]
        t, o = shard.slice_corpus(c.tokens, c.doc_offsets, lo, hi)
        coll = shard.TorchCollective()
        eng = OracleEngine()
        sh, first, n_docs, n_tokens = shard.build_shard(eng, coll, t, o, c.vocab, variant,
                                                        1.2, 0.75, 0.5)
        ids, sc = shard.retrieve_sharded(eng, coll, sh, q.tokens, q.offsets, k)
        out[rank] = (first, n_docs, n_tokens, ids.tolist(), sc.tolist())
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("variant,k", [("lucene", 10), ("bm25+", 7), ("robertson", 600),
                                       ("tfldp", 10)])
def test_two_gloo_shards_equal_the_unsplit_collection(variant, k):
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), variant, k, out), nprocs=world, join=True)
        res = dict(out)
    c, q = _corpus(), _queries()
    ranges = shard.doc_ranges(c.n_docs, world)
    assert [res[r][0] for r in range(world)] == [lo for lo, _ in ranges]
    for r in range(world):
        assert res[r][1] == c.n_docs and res[r][2] == c.n_tokens
        assert res[r][3] == res[0][3] and res[r][4] == res[0][4]  # every rank the same rows
    full = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.VARIANTS[variant], 1.2, 0.75, 0.5)
    want_ids, want_sc = oracle.topk(full, q.tokens, q.offsets, k)
    np.testing.assert_array_equal(np.array(res[0][3]), want_ids)
    np.testing.assert_array_equal(np.array(res[0][4]), want_sc)


def test_doc_ranges_cover_and_slice():
    assert shard.doc_ranges(10, 3) == [(0, 3), (3, 6), (6, 10)]
    with pytest.raises(ValueError):
        shard.doc_ranges(2, 3)
    c = _corpus()
    parts = [shard.slice_corpus(c.tokens, c.doc_offsets, lo, hi)
             for lo, hi in shard.doc_ranges(c.n_docs, 4)]
    assert np.array_equal(np.concatenate([t for t, _ in parts]), c.tokens)
    assert all(o[0] == 0 and o[-1] == t.shape[0] for t, o in parts)
    assert sum(o.shape[0] - 1 for _, o in parts) == c.n_docs


def test_local_shards_equal_the_unsplit_collection():
    """build_local (G shards in one process) with the oracle engine."""
    import torch
    c, q = _corpus(), _queries()
    for g in (1, 3, 5):
        loc = shard.build_local(OracleEngine(), c.tokens, c.doc_offsets, c.vocab, g, "bm25l",
                                1.2, 0.75, 0.5)
        rows = [loc.engine.retrieve(sh, q.tokens, q.offsets, 12) for sh in loc.shards]
        ids, sc = loc.engine.merge(torch.stack([r[0] for r in rows]),
                                   torch.stack([r[1] for r in rows]), 12)
        full = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25L, 1.2, 0.75, 0.5)
        want_ids, want_sc = oracle.topk(full, q.tokens, q.offsets, 12)
        np.testing.assert_array_equal(ids, want_ids)
        np.testing.assert_array_equal(sc, want_sc)

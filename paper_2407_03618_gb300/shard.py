"""Doc-range sharding of the eager index: one index per contiguous range of
documents, scored with the whole collection's statistics, queried by merging
every shard's top k.

The paper's index is one sparse |V| x |C| matrix (Sec. 2 "Efficient Matrix
Sparsity"); Sec. 2.1's footnote sizes a dense 2M x 200K one at 1.6 TB.  Split
by documents, every shard keeps the columns' entries of its own documents,
and the method's scores stay exact because IDF, S0 and Lavg are taken from
the collection, not the shard:

  build     each shard indexes its documents; DF[V], N and the token count
            are summed over the shards (one all-reduce); each shard rescores
            its entries with those sums and learns its first global doc id
            (an all-gather of the shards' document counts);
  retrieve  every shard answers the whole query batch (local top k with
            global ids); the rows are gathered (one all-gather) and merged
            by (score desc, doc id asc).

This module only sequences those steps and the collectives; the engine does
the arithmetic.  `GpuEngine` is the CUDA library; the collective is
`torch.distributed` (NCCL between GPUs, gloo on the CPU) through
`TorchCollective`; `build_local` runs the same steps for G shards held by
one process (one GPU standing in for several), the all-reduce becoming a sum
over the shards.  No step here falls back to anything: an engine that is
missing raises.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def doc_ranges(n_docs: int, n_shards: int) -> list[tuple[int, int]]:
    """Contiguous, nearly equal document ranges [lo, hi) covering 0..n_docs."""
    if n_shards < 1 or n_docs < n_shards:
        raise ValueError(f"cannot split {n_docs} documents into {n_shards} non-empty ranges")
    cuts = [n_docs * s // n_shards for s in range(n_shards + 1)]
    return [(cuts[s], cuts[s + 1]) for s in range(n_shards)]


def slice_corpus(tokens: np.ndarray, doc_offsets: np.ndarray, lo: int, hi: int):
    """The tokens of documents [lo, hi) and their offsets rebased to 0."""
    a, b = int(doc_offsets[lo]), int(doc_offsets[hi])
    return tokens[a:b], (doc_offsets[lo:hi + 1] - a).astype(np.int64)


# ------------------------------------------------------------ collectives --

class TorchCollective:
    """Sums and gathers over the ranks of a torch.distributed group (NCCL for
    CUDA tensors, gloo for CPU tensors).  Rank r holds shard r."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def all_reduce_sum(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def all_gather(self, t):
        """[world, *t.shape]: every rank's t, in rank order."""
        import torch
        out = [torch.empty_like(t) for _ in range(self.size)]
        self.dist.all_gather(out, t.contiguous(), group=self.group)
        return torch.stack(out)


# ---------------------------------------------------------------- engines --

class GpuEngine:
    """The CUDA library as the shard engine (bm25.Index per shard)."""

    def __init__(self):
        from . import bm25
        self.bm25 = bm25

    def build(self, tokens, doc_offsets, vocab, variant, k1, b, delta):
        return self.bm25.Index.build(tokens, doc_offsets, vocab, variant, k1, b, delta)

    def df(self, ix):
        return ix.df_device()

    def counts(self, ix):
        inf = ix.info()
        return inf["n_docs"], inf["n_tokens"]

    def count_tensor(self, ix):
        import torch
        n, t = self.counts(ix)
        return torch.tensor([n, t], dtype=torch.int64, device=ix.df_device().device)

    def rescore(self, ix, global_df, n_docs, n_tokens, doc_offset):
        ix.rescore(global_df, n_docs, n_tokens, doc_offset)

    def retrieve(self, ix, q_tokens, q_offsets, k):
        return ix.retrieve(q_tokens, q_offsets, k)

    def merge(self, cand_ids, cand_scores, k):
        return self.bm25.merge_topk(cand_ids, cand_scores, k)


# --------------------------------------------------------- one shard/rank --

def build_shard(engine, coll, tokens, doc_offsets, vocab, variant="lucene", k1=1.5, b=0.75,
                delta=0.5):
    """This rank's shard of a collection split by documents (rank order =
    document order).  tokens / doc_offsets hold this rank's documents only.
    Returns (shard, first global doc id, global N, global token count)."""
    sh = engine.build(tokens, doc_offsets, vocab, variant, k1, b, delta)
    counts = engine.count_tensor(sh)                # [N_r, T_r]
    every = coll.all_gather(counts)                 # [world, 2]
    first = int(every[:coll.rank, 0].sum().item())  # documents of the ranks before this one
    n_docs, n_tokens = (int(x) for x in every.sum(dim=0).tolist())
    df = engine.df(sh).clone()
    coll.all_reduce_sum(df)                         # DF of the whole collection
    engine.rescore(sh, df, n_docs, n_tokens, first)
    return sh, first, n_docs, n_tokens


def retrieve_sharded(engine, coll, shard, q_tokens, q_offsets, k: int):
    """Top k over the whole collection for a query batch every rank holds."""
    ids, scores = engine.retrieve(shard, q_tokens, q_offsets, k)
    return engine.merge(coll.all_gather(ids), coll.all_gather(scores), k)


# ------------------------------------------------- all shards in one process --

@dataclass
class LocalShards:
    """G shards held by one process (one GPU standing in for G of them)."""
    engine: object
    shards: list
    ranges: list
    n_docs: int
    n_tokens: int

    def retrieve(self, q_tokens, q_offsets, k: int):
        import torch
        rows = [self.engine.retrieve(sh, q_tokens, q_offsets, k) for sh in self.shards]
        ids = torch.stack([r[0] for r in rows])
        scores = torch.stack([r[1] for r in rows])
        return self.engine.merge(ids, scores, k)

    def close(self):
        for sh in self.shards:
            sh.close()
        self.shards = []


def build_local(engine, tokens, doc_offsets, vocab, n_shards, variant="lucene", k1=1.5, b=0.75,
                delta=0.5, to_device=None):
    """The same two-step build for G shards in this process: the all-reduce
    becomes a sum over the shards' DF tensors.  tokens / doc_offsets are the
    whole collection (host arrays); to_device moves a shard's slice to where
    the engine wants it."""
    tokens = np.asarray(tokens, np.int32)
    doc_offsets = np.asarray(doc_offsets, np.int64)
    ranges = doc_ranges(doc_offsets.shape[0] - 1, n_shards)
    shards = []
    for lo, hi in ranges:
        t, o = slice_corpus(tokens, doc_offsets, lo, hi)
        if to_device:
            t, o = to_device(t), to_device(o)
        shards.append(engine.build(t, o, vocab, variant, k1, b, delta))
    df = engine.df(shards[0]).clone()
    for sh in shards[1:]:
        df += engine.df(sh)
    n_docs = sum(engine.counts(sh)[0] for sh in shards)
    n_tokens = sum(engine.counts(sh)[1] for sh in shards)
    for sh, (lo, _) in zip(shards, ranges):
        engine.rescore(sh, df, n_docs, n_tokens, lo)
    return LocalShards(engine, shards, ranges, n_docs, n_tokens)

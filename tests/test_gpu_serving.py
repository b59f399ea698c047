"""Serving and plan tuning on the GPU.

The server batches requests as they arrive over several resident indexes;
every result must be the oracle's (same tolerance as the other parity
tests), and a query's result must not depend on what else was in flight:
the same query alone on an idle server and inside a burst of others gives
the same ids (up to ties within tolerance) and scores within tolerance.
"""
import numpy as np
import pytest

import oracle
from oracle.compare import RTOL, check_topk
from paper_2407_03618_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03618_gb300 import bm25
    dev = torch.device("cuda:0")
    corpora = [synth.WORKLOADS["tiny"].corpus(),
               synth.make_corpus(30_000, 20_000, 1.05, ("lognormal", 60, 0.6), seed=7),
               synth.make_corpus(5_000, 3_000, 1.2, ("poisson", 20), seed=8)]
    variants = ["lucene", "bm25+", "robertson"]
    idx, orcs = [], []
    for c, v in zip(corpora, variants):
        idx.append(bm25.Index.build(torch.from_numpy(c.tokens).to(dev),
                                    torch.from_numpy(c.doc_offsets).to(dev), c.vocab, v))
        orcs.append(oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.VARIANTS[v]))
    # one index per plan kind, so batches take both paths
    idx[0].set_plan(bm25.ACC_SMEM_TILED, 1024, 256)
    idx[1].set_plan(bm25.ACC_AUTO, 0, 0, 4096)
    idx[2].set_plan(bm25.ACC_L2_DENSE)
    yield {"bm25": bm25, "idx": idx, "orcs": orcs, "corpora": corpora, "dev": dev}
    for ix in idx:
        ix.close()


def _requests(env, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        i = int(rng.integers(0, len(env["idx"])))
        v = env["corpora"][i].vocab
        L = int(rng.integers(0, 33))
        toks = synth.zipf_sampler(v, 1.1)(rng, L) if L else np.zeros(0, np.int32)
        out.append((i, toks.astype(np.int32), int(rng.choice([1, 10, 100, 1000]))))
    return out


def _check(env, req, res, where):
    i, toks, k = req
    full, ab = oracle.score_all(env["orcs"][i], toks, with_abs=True)
    check_topk(res[0], res[1], full, ab, k, where=where)


def test_burst_of_mixed_requests(env):
    srv = env["bm25"].Server(env["idx"], max_batch_queries=64, max_inflight=3)
    reqs = _requests(env, 400, seed=1)
    tickets = [srv.submit(i, t, k) for i, t, k in reqs]
    for n, (r, tk) in enumerate(zip(reqs, tickets)):
        _check(env, r, srv.poll(tk, r[2]), f"burst r{n}")
    st = srv.stats()
    assert st["completed"] == 400 and st["failed"] == 0
    assert st["batches"] >= 400 // 64
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    srv.close()


def test_result_is_the_same_alone_and_in_the_mix(env):
    srv = env["bm25"].Server(env["idx"], max_batch_queries=128, max_inflight=4)
    probes = _requests(env, 12, seed=2)
    alone = []
    for i, t, k in probes:  # one at a time on an idle server
        alone.append(srv.poll(srv.submit(i, t, k), k))
    others = _requests(env, 600, seed=3)
    tickets = []
    for n, (i, t, k) in enumerate(others):  # probes interleaved with a burst
        tickets.append(srv.submit(i, t, k))
        if n % 50 == 25:
            p = probes[(n // 50) % len(probes)]
            tickets.append(("probe", (n // 50) % len(probes), srv.submit(*p)))
    for tk in tickets:
        if isinstance(tk, tuple):
            _, j, t = tk
            k = probes[j][2]
            ids, sc = srv.poll(t, k)
            a_ids, a_sc = alone[j]
            np.testing.assert_allclose(sc, a_sc, rtol=RTOL, atol=RTOL)
            for pos in np.nonzero(ids != a_ids)[0]:  # only ties may swap
                assert abs(sc[pos] - a_sc[pos]) <= RTOL * max(1.0, abs(a_sc[pos]))
            _check(env, probes[j], (ids, sc), f"probe {j} in mix")
        else:
            srv.poll(tk, 1000, timeout_us=-1)
    for j, p in enumerate(probes):
        _check(env, p, alone[j], f"probe {j} alone")
    srv.close()


def test_memory_budget_admission(env):
    bm25 = env["bm25"]
    # a budget that admits only small batches: everything still completes
    srv = bm25.Server(env["idx"], max_batch_queries=512, max_inflight=3,
                      memory_budget=100 << 20)
    reqs = _requests(env, 200, seed=4)
    tickets = [srv.submit(i, t, k) for i, t, k in reqs]
    for n, (r, tk) in enumerate(zip(reqs, tickets)):
        _check(env, r, srv.poll(tk, r[2]), f"budget r{n}")
    assert srv.stats()["bytes_held"] <= 100 << 20
    srv.close()
    # a budget below one query's scratch fails that query, and only it
    srv = bm25.Server(env["idx"][:1], memory_budget=1 << 10)
    tk = srv.submit(0, np.array([1, 2], np.int32), 10)
    with pytest.raises(bm25.BM25Error) as e:
        srv.poll(tk, 10)
    assert e.value.code == -3
    srv.close()


def test_submit_checks(env):
    bm25 = env["bm25"]
    srv = bm25.Server(env["idx"], k_max=100)
    with pytest.raises(bm25.BM25Error) as e:
        srv.submit(0, np.array([1, 999_999], np.int32), 10)
    assert e.value.code == -2
    for args in [(5, np.array([1], np.int32), 10), (0, np.array([1], np.int32), 0),
                 (0, np.array([1], np.int32), 101)]:
        with pytest.raises(bm25.BM25Error) as e:
            srv.submit(*args)
        assert e.value.code == -1
    tk = srv.submit(0, np.zeros(0, np.int32), 3)  # an empty query: ids 0, 1, 2 at score 0
    ids, sc = srv.poll(tk, 3)
    assert ids.tolist() == [0, 1, 2] and sc.tolist() == [0.0, 0.0, 0.0]
    with pytest.raises(bm25.BM25Error):
        srv.poll(tk, 3)  # the ticket was released
    srv.close()


def test_autotune_picks_a_plan_and_keeps_results(env):
    import torch
    bm25 = env["bm25"]
    c = env["corpora"][1]
    q = synth.make_queries(300, c.vocab, 1.05, ("uniform", 1, 16), 10, seed=9)
    dev = env["dev"]
    ix = bm25.Index.build(torch.from_numpy(c.tokens).to(dev),
                          torch.from_numpy(c.doc_offsets).to(dev), c.vocab, "bm25l")
    qt, qo = torch.from_numpy(q.tokens).to(dev), torch.from_numpy(q.offsets).to(dev)
    best, ms, log = ix.autotune(qt, qo, 10)
    assert ms > 0 and len(log) >= 4
    assert best == ix.get_plan()
    # a later candidate replaces the best only when more than 1 % faster, so
    # the chosen time is one of those logged and within 1 % of the fastest
    assert ms in [m for _, m in log]
    assert ms <= min(m for _, m in log) / 0.99 + 1e-9
    assert best["accumulator"] in (bm25.ACC_SMEM_TILED, bm25.ACC_AUTO)
    orc = oracle.build(c.tokens, c.doc_offsets, c.vocab, oracle.BM25L)
    ids, sc = ix.retrieve(qt, qo, 10)
    ix.sync_status()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for i in range(0, q.n_queries, 7):
        full, ab = oracle.score_all(orc, q.query(i), with_abs=True)
        check_topk(ids[i], sc[i], full, ab, 10, where=f"tuned q{i}")
    ix.close()

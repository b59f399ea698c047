"""The seeded generators: deterministic, and shaped as their recipes say."""
import numpy as np

from paper_2407_03618_gb300 import synth


def test_deterministic_and_shapes():
    w = synth.WORKLOADS["tiny"]
    a, b = w.corpus(), w.corpus()
    assert np.array_equal(a.tokens, b.tokens) and np.array_equal(a.doc_offsets, b.doc_offsets)
    assert a.n_docs == 2000 and a.vocab == 5000
    assert a.tokens.dtype == np.int32 and a.doc_offsets.dtype == np.int64
    assert a.doc_offsets[0] == 0 and a.doc_offsets[-1] == a.n_tokens
    lens = np.diff(a.doc_offsets)
    assert lens.min() >= 1 and abs(lens.mean() - 60) < 1.5
    assert a.tokens.min() >= 0 and a.tokens.max() < 5000
    q = w.queries()
    ql = np.diff(q.offsets)
    assert q.n_queries == 100 and ql.min() >= 2 and ql.max() <= 8


def test_zipf_law_and_head_exclusion():
    rng = np.random.default_rng(0)
    draw = synth.zipf_sampler(1000, 1.0)
    x = draw(rng, 400_000)
    c = np.bincount(x, minlength=1000)
    # P(rank 1) / P(rank 2) = 2**s, P(rank 1)/P(rank 10) = 10**s
    assert abs(c[0] / c[1] - 2.0) < 0.05
    assert abs(c[0] / c[9] - 10.0) < 0.5
    y = synth.zipf_sampler(1000, 1.0, exclude_head=100)(rng, 10_000)
    assert y.min() >= 100 and y.max() < 1000


def test_lognormal_mean_is_arithmetic():
    rng = np.random.default_rng(0)
    x = synth.lengths_lognormal(rng, 200_000, 60, 0.6)
    assert abs(x.mean() - 60) < 0.6
    assert x.min() >= 1


def test_subset():
    q = synth.make_queries(50, 100, 1.1, ("uniform", 0, 5))
    s = q.subset([3, 7, 7])
    assert s.n_queries == 3
    assert np.array_equal(s.query(1), q.query(7))

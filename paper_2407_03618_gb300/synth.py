"""Seeded synthetic corpora and query batches.

Inputs only: token ids and offsets drawn from fixed distributions.  No part of
the scoring method lives here, so the CUDA path and the CPU oracle can both be
fed from this module without sharing any of the method's arithmetic.

The paper measures on BEIR corpora (Sec. 3 "Throughput", Table 1), which are
not available here; these generators stand in for them with the shapes of
those workloads:

* term ids follow a Zipf law truncated to the vocabulary: P(rank r) is
  proportional to r**-s for r = 1..V, and token id = r - 1 (so low ids are
  the frequent terms);
* document lengths are Poisson or lognormal.  A lognormal "mean" is the
  arithmetic mean, so mu = ln(mean) - sigma**2 / 2.  Lengths are rounded to
  the nearest integer and clamped to at least 1;
* query lengths are uniform on [lo, hi] or geometric and clamped;
* stopword removal is imitated by dropping the `exclude_head` most frequent
  ranks from the query distribution.

Corpora use numpy's default_rng(seed=0) and queries default_rng(seed=1)
unless told otherwise.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_CHUNK = 1 << 24


@dataclass
class Corpus:
    tokens: np.ndarray       # int32 [T]
    doc_offsets: np.ndarray  # int64 [N+1]
    vocab: int

    @property
    def n_docs(self) -> int:
        return int(self.doc_offsets.shape[0] - 1)

    @property
    def n_tokens(self) -> int:
        return int(self.tokens.shape[0])


@dataclass
class Queries:
    tokens: np.ndarray       # int32 [sum |Q|]
    offsets: np.ndarray      # int64 [nQ+1]

    @property
    def n_queries(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def query(self, i: int) -> np.ndarray:
        return self.tokens[self.offsets[i]:self.offsets[i + 1]]

    def subset(self, idx) -> "Queries":
        parts = [self.query(int(i)) for i in idx]
        off = np.zeros(len(parts) + 1, np.int64)
        if parts:
            off[1:] = np.cumsum([p.shape[0] for p in parts])
        tok = np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
        return Queries(tok, off)


def zipf_sampler(vocab: int, s: float, exclude_head: int = 0):
    """Return f(rng, n) drawing n int32 ids from the truncated Zipf law over
    ranks exclude_head+1 .. vocab (ids rank-1)."""
    ranks = np.arange(exclude_head + 1, vocab + 1, dtype=np.float64)
    w = ranks ** (-float(s))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]

    def draw(rng: np.random.Generator, n: int) -> np.ndarray:
        out = np.empty(n, np.int32)
        for lo in range(0, n, _CHUNK):
            hi = min(n, lo + _CHUNK)
            u = rng.random(hi - lo)
            idx = np.searchsorted(cdf, u, side="right")
            np.minimum(idx, cdf.shape[0] - 1, out=idx)
            out[lo:hi] = idx + exclude_head
        return out

    return draw


def lengths_poisson(rng, n: int, mean: float, minimum: int = 1) -> np.ndarray:
    return np.maximum(rng.poisson(mean, n), minimum).astype(np.int64)


def lengths_lognormal(rng, n: int, mean: float, sigma: float, minimum: int = 1) -> np.ndarray:
    mu = np.log(mean) - sigma * sigma / 2.0
    x = np.rint(rng.lognormal(mu, sigma, n))
    return np.maximum(x, minimum).astype(np.int64)


def offsets_from_lengths(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(lengths.shape[0] + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def make_corpus(n_docs: int, vocab: int, zipf_s: float, length: tuple, seed: int = 0) -> Corpus:
    """length = ("poisson", mean) or ("lognormal", mean, sigma)."""
    rng = np.random.default_rng(seed)
    if length[0] == "poisson":
        lens = lengths_poisson(rng, n_docs, length[1])
    elif length[0] == "lognormal":
        lens = lengths_lognormal(rng, n_docs, length[1], length[2])
    else:
        raise ValueError(length)
    off = offsets_from_lengths(lens)
    tokens = zipf_sampler(vocab, zipf_s)(rng, int(off[-1]))
    return Corpus(tokens, off, vocab)


def make_queries(n_queries: int, vocab: int, zipf_s: float, length: tuple,
                 exclude_head: int = 0, seed: int = 1) -> Queries:
    """length = ("uniform", lo, hi) or ("geometric", p, max)."""
    rng = np.random.default_rng(seed)
    if length[0] == "uniform":
        lens = rng.integers(length[1], length[2] + 1, n_queries).astype(np.int64)
    elif length[0] == "geometric":
        lens = np.minimum(rng.geometric(length[1], n_queries), length[2]).astype(np.int64)
    else:
        raise ValueError(length)
    off = offsets_from_lengths(lens)
    tok = zipf_sampler(vocab, zipf_s, exclude_head)(rng, int(off[-1]))
    return Queries(tok, off)


@dataclass
class Workload:
    name: str
    n_docs: int
    vocab: int
    zipf_s: float
    doc_length: tuple
    n_queries: int
    query_length: tuple
    query_exclude_head: int
    ks: tuple
    variants: tuple
    params: dict = field(default_factory=lambda: {"k1": 1.5, "b": 0.75, "delta": 0.5})

    def corpus(self, seed: int = 0) -> Corpus:
        return make_corpus(self.n_docs, self.vocab, self.zipf_s, self.doc_length, seed)

    def queries(self, seed: int = 1, n_queries: int | None = None) -> Queries:
        return make_queries(self.n_queries if n_queries is None else n_queries, self.vocab,
                            self.zipf_s, self.query_length, self.query_exclude_head, seed)

    def describe(self) -> dict:
        return {"workload": self.name, "n_docs": self.n_docs, "vocab": self.vocab,
                "zipf_s": self.zipf_s, "doc_length": list(self.doc_length),
                "n_queries": self.n_queries, "query_length": list(self.query_length),
                "query_exclude_head": self.query_exclude_head}


ALL_VARIANTS = ("lucene", "robertson", "atire", "bm25l", "bm25+")

WORKLOADS = {
    # 2,000 docs, vocab 5,000, Zipf s=1.1, Poisson(60) lengths; 100 queries
    # of 2..8 tokens from the same Zipf; k=10; Lucene k1=1.5 b=0.75.
    "tiny": Workload("tiny-2k", 2000, 5000, 1.1, ("poisson", 60), 100, ("uniform", 2, 8),
                     0, (10,), ("lucene",)),
    # 1M docs, vocab 200k, Zipf s=1.05, lognormal(60, 0.6) lengths; 10k
    # queries of 1..16 tokens with the 100 head terms removed; k=10 and 100.
    "1m": Workload("zipf-1m", 1_000_000, 200_000, 1.05, ("lognormal", 60, 0.6), 10_000,
                   ("uniform", 1, 16), 100, (10, 100), ALL_VARIANTS),
    # passage scale: 8.8M docs, vocab 1M, Zipf s=1.0, lognormal(56, 0.5);
    # 7k queries, geometric lengths (mean 6) clamped to 32; k=10/100/1000.
    "passage": Workload("passage-8.8m", 8_800_000, 1_000_000, 1.0, ("lognormal", 56, 0.5),
                        7_000, ("geometric", 1.0 / 6.0, 32), 0, (10, 100, 1000), ("lucene",)),
    # long documents: 5M docs, vocab 2M, Zipf s=1.1, lognormal(300, 0.8);
    # 5k queries of 20..60 tokens incl. head terms; k=100; BM25+.
    "long": Workload("long-5m", 5_000_000, 2_000_000, 1.1, ("lognormal", 300, 0.8), 5_000,
                     ("uniform", 20, 60), 0, (100,), ("bm25+",)),
}


def random_tiny_corpus(rng: np.random.Generator, max_docs: int = 8, max_vocab: int = 6,
                       max_len: int = 6, allow_empty: bool = True) -> Corpus:
    """Small uniform corpora for brute-force checks (empty docs allowed)."""
    n = int(rng.integers(1, max_docs + 1))
    v = int(rng.integers(1, max_vocab + 1))
    lens = rng.integers(0 if allow_empty else 1, max_len + 1, n).astype(np.int64)
    off = offsets_from_lengths(lens)
    tok = rng.integers(0, v, int(off[-1])).astype(np.int32)
    return Corpus(tok, off, v)


def random_queries(rng: np.random.Generator, vocab: int, n_queries: int, max_len: int,
                   min_len: int = 0) -> Queries:
    lens = rng.integers(min_len, max_len + 1, n_queries).astype(np.int64)
    off = offsets_from_lengths(lens)
    tok = rng.integers(0, vocab, int(off[-1])).astype(np.int32)
    return Queries(tok, off)


# ---- text (for the tokenizer) ----------------------------------------------

_ASCII_WORD = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz", np.uint8)
_ASCII_MIXED = np.frombuffer(b"ABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789_", np.uint8)
_NON_ASCII = ["é", "ü", "ß", "ñ", "ø", "中", "文", "ж",
              "λ", "\U0001f600"]
_SEPARATORS = [b" ", b" ", b" ", b" ", b" ", b", ", b". ", b"\n", b" - ", b"'", b" (", b") ",
               b"; ", b"\t", b"!", b"\"", b"/", b" ... "]


def make_lexicon(n_words: int, seed: int = 0) -> list:
    """n_words synthetic word forms (bytes): 1-12 characters, mostly lowercase
    ASCII letters, some upper case, digits, '_' and non-ASCII characters;
    about a tenth are one character long.  Forms may repeat or differ only by
    case."""
    rng = np.random.default_rng(seed)
    lens = np.where(rng.random(n_words) < 0.1, 1, rng.integers(2, 13, n_words))
    out = []
    for L in lens.tolist():
        chars = []
        for _ in range(L):
            u = rng.random()
            if u < 0.85:
                chars.append(bytes([int(rng.choice(_ASCII_WORD))]))
            elif u < 0.95:
                chars.append(bytes([int(rng.choice(_ASCII_MIXED))]))
            else:
                chars.append(_NON_ASCII[int(rng.integers(0, len(_NON_ASCII)))].encode())
        out.append(b"".join(chars))
    return out


def make_text_corpus(n_docs: int, n_words: int, zipf_s: float, length: tuple, seed: int = 0,
                     lexicon_seed: int = 1000):
    """UTF-8 texts: words of a synthetic lexicon drawn Zipf(zipf_s), joined by
    ASCII separators (spaces, punctuation, newlines, apostrophes).  Returns
    (text uint8 [bytes], offsets int64 [n_docs + 1], lexicon)."""
    rng = np.random.default_rng(seed)
    lex = make_lexicon(n_words, lexicon_seed)
    if length[0] == "poisson":
        lens = lengths_poisson(rng, n_docs, length[1], minimum=0)
    else:
        lens = lengths_lognormal(rng, n_docs, length[1], length[2], minimum=0)
    words = zipf_sampler(n_words, zipf_s)(rng, int(lens.sum()))
    seps = rng.integers(0, len(_SEPARATORS), int(lens.sum()))
    pieces = lex + _SEPARATORS
    plen = np.array([len(p) for p in pieces], np.int64)
    pbuf = np.frombuffer(b"".join(pieces), np.uint8)
    pstart = np.concatenate([[0], np.cumsum(plen)[:-1]])
    # piece sequence: word, separator, word, separator, ... per document
    seq = np.empty(2 * words.shape[0], np.int64)
    seq[0::2] = words
    seq[1::2] = len(lex) + seps
    seq_len = plen[seq]
    ends = np.cumsum(seq_len)
    total = int(ends[-1]) if ends.shape[0] else 0
    owner = np.repeat(np.arange(seq.shape[0]), seq_len)
    within = np.arange(total) - np.repeat(ends - seq_len, seq_len)
    text = pbuf[pstart[seq][owner] + within] if total else np.zeros(0, np.uint8)
    tok_off = np.concatenate([[0], np.cumsum(lens)]) * 2  # piece index of each doc's start
    byte_off = np.concatenate([[0], ends])[tok_off]
    return np.ascontiguousarray(text, np.uint8), byte_off.astype(np.int64), lex


def split_texts(text: np.ndarray, offsets: np.ndarray) -> list:
    """The texts as a list of bytes."""
    raw = text.tobytes()
    return [raw[offsets[i]:offsets[i + 1]] for i in range(offsets.shape[0] - 1)]

"""Tokenizer oracle (Sec. 2 "Tokenization").

TEST INFRASTRUCTURE ONLY (used by tests/ and bench.py's oracle leg); the
CUDA tokenizer never imports it and shares no code with it.

The paper splits text with scikit-learn's pattern r"(?u)\\b\\w\\w+\\b"
(words of at least two word characters), removes stopwords, and maps each
distinct word to an integer id.  Read here, on UTF-8 bytes:

* word characters: ASCII letters, digits and '_', and every non-ASCII
  character (its UTF-8 bytes 0x80-0xFF); on ASCII text this is exactly
  Python's \\w, which the pins check against the re module;
* ASCII letters are lowercased first (scikit-learn lowercases by default);
* a token is a maximal run of word bytes holding at least two characters
  (bytes that are not UTF-8 continuation bytes 0x80-0xBF);
* a token equal to one of the given stopwords (lowercase bytes) is dropped;
* corpus ids are given in order of first occurrence over the corpus
  (document order, then position); a query keeps only tokens that are in
  the vocabulary, with their corpus ids.
"""
from __future__ import annotations

import re

import numpy as np

_RUN = re.compile(rb"[A-Za-z0-9_\x80-\xff]+")


def lower_ascii(text: bytes) -> bytes:
    return text.lower()  # bytes.lower() changes ASCII letters only


def split(text: bytes) -> list[bytes]:
    """The tokens of one text, in order (before stopwords)."""
    out = []
    for m in _RUN.finditer(lower_ascii(text)):
        tok = m.group()
        chars = sum(1 for c in tok if not 0x80 <= c <= 0xBF)
        if chars >= 2:
            out.append(tok)
    return out


def tokenize_corpus(docs: list[bytes], stopwords=()):
    """(ids int32 [T], offsets int64 [N+1], vocab list[bytes] in id order)."""
    stop = set(stopwords)
    vocab: dict[bytes, int] = {}
    ids, offs = [], [0]
    for d in docs:
        for tok in split(d):
            if tok in stop:
                continue
            ids.append(vocab.setdefault(tok, len(vocab)))
        offs.append(len(ids))
    words = [None] * len(vocab)
    for w, i in vocab.items():
        words[i] = w
    return np.array(ids, np.int32), np.array(offs, np.int64), words


def tokenize_queries(queries: list[bytes], vocab_words: list[bytes], stopwords=()):
    """(ids int32, offsets int64 [Q+1]): known tokens only, corpus ids."""
    stop = set(stopwords)
    index = {w: i for i, w in enumerate(vocab_words)}
    ids, offs = [], [0]
    for qtext in queries:
        for tok in split(qtext):
            if tok in stop or tok not in index:
                continue
            ids.append(index[tok])
        offs.append(len(ids))
    return np.array(ids, np.int32), np.array(offs, np.int64)


def pack(texts: list[bytes]):
    """Concatenated bytes (uint8) and byte offsets (int64 [n+1])."""
    offs = np.zeros(len(texts) + 1, np.int64)
    offs[1:] = np.cumsum([len(t) for t in texts])
    buf = np.frombuffer(b"".join(texts), np.uint8) if texts else np.zeros(0, np.uint8)
    return buf.copy(), offs

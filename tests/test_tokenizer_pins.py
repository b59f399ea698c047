"""Pins of the tokenizer oracle (oracle/tokenizer.py, Sec. 2 "Tokenization").

* On ASCII text, and on text whose non-ASCII characters are all letters, its
  split equals Python's re engine running the paper's pattern
  r"(?u)\\b\\w\\w+\\b" on the lowercased text.
* Hand-worked cases: one-character words, multi-byte characters counted as
  one character, a character outside \\w (an emoji; the reading counts every
  non-ASCII character as a word character), text boundaries, stopwords, ids
  by first occurrence, unknown query words.
"""
import re

import numpy as np

from oracle import tokenizer as tk
from paper_2407_03618_gb300 import synth

PAPER = re.compile(r"(?u)\b\w\w+\b")


def _paper(text: bytes):
    return [w.encode() for w in PAPER.findall(text.decode("utf-8").lower())]


def test_ascii_equals_the_papers_pattern():
    rng = np.random.default_rng(5)
    alphabet = b"abcXYZ019_ .,;:'-\n\t!?()[]/\\\"@#$%&*+=<>|~`^{}"
    for _ in range(500):
        n = int(rng.integers(0, 60))
        s = bytes(rng.choice(np.frombuffer(alphabet, np.uint8), n).tolist())
        assert tk.split(s) == _paper(s), s


def test_letters_only_text_equals_the_papers_pattern():
    text, off, lex = synth.make_text_corpus(300, 400, 1.1, ("poisson", 20), seed=6)
    emoji = "\U0001f600".encode()
    for d in synth.split_texts(text, off):
        if emoji in d:
            continue  # outside \w: the reading differs there (next test)
        assert tk.split(d) == _paper(d)


def test_hand_cases():
    assert tk.split(b"a bc d ef_ g") == [b"bc", b"ef_"]
    assert tk.split("café é 中文 中 a中 Ünï".encode()) == \
        ["café".encode(), "中文".encode(), "a中".encode(), "Ünï".encode()]  # non-ASCII keeps its case
    assert tk.split(b"Don't STOP, it's 42") == [b"don", b"stop", b"it", b"42"]
    # an emoji is not \w for re, but a word character here
    assert tk.split("ab\U0001f600cd".encode()) == ["ab\U0001f600cd".encode()]
    assert _paper("ab\U0001f600cd".encode()) == [b"ab", b"cd"]


def test_corpus_ids_offsets_and_stopwords():
    docs = [b"The cat sat", b"", b"the dog, THE cat!", b"a b c"]
    ids, off, vocab = tk.tokenize_corpus(docs, stopwords=[b"the"])
    assert vocab == [b"cat", b"sat", b"dog"]
    assert ids.tolist() == [0, 1, 2, 0]
    assert off.tolist() == [0, 2, 2, 4, 4]
    qids, qoff = tk.tokenize_queries([b"Cat unknown DOG the", b"zz"], vocab, stopwords=[b"the"])
    assert qids.tolist() == [0, 2] and qoff.tolist() == [0, 2, 2]


def test_text_boundaries_split_words():
    ids, off, vocab = tk.tokenize_corpus([b"ab", b"cd", b"abcd"])
    assert vocab == [b"ab", b"cd", b"abcd"] and off.tolist() == [0, 1, 2, 3]

"""FP64 CPU oracle for BM25S eager sparse scoring (arXiv 2407.03618).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path (the CUDA
library and its binding) never imports it and shares no code with it.

The arithmetic lives in ``bm25_oracle.c`` (plain C, FP64); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

* ``build``      -- |D|, Lavg, TF, DF, IDF, S0 and the term-major CSC of
                    S - S0 (Sec. 2 "Calculation of BM25", "Eager index-time
                    scoring", "Efficient Matrix Sparsity"; Sec. 2.1)
* ``score_all``  -- lazy exhaustive B(Q,D) for every document (Sec. 2)
* ``rank``/``topk`` -- full sort by (score desc, doc id asc) (Sec. 2
                    "Top-k selection", with the tie rule written out)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

LUCENE, ROBERTSON, ATIRE, BM25L, BM25PLUS, TFLDP = 0, 1, 2, 3, 4, 5
VARIANTS = {"lucene": LUCENE, "robertson": ROBERTSON, "atire": ATIRE,
            "bm25l": BM25L, "bm25+": BM25PLUS, "tfldp": TFLDP}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bm25_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def compile_oracle(force: bool = False) -> str:
    """Compile bm25_oracle.c into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(compile_oracle())
            P = ctypes.c_void_p
            i64, i32, f64, cint = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
            lib.oracle_idf.restype = f64
            lib.oracle_idf.argtypes = [cint, f64, f64]
            lib.oracle_term_score.restype = f64
            lib.oracle_term_score.argtypes = [cint, f64, f64, f64, f64, f64, f64, f64]
            lib.oracle_nonoccurrence.restype = f64
            lib.oracle_nonoccurrence.argtypes = [cint, f64, f64, f64, f64]
            lib.oracle_build.restype = i64
            lib.oracle_build.argtypes = [P, i64, P, i64, i32, cint, f64, f64, f64,
                                         P, P, P, P, P, P, P, P, P, P, P, P]
            lib.oracle_score_all.restype = None
            lib.oracle_score_all.argtypes = [P, i64, i64, i32, cint, f64, f64, f64,
                                             P, f64, P, P, P, P, P, P]
            lib.oracle_rank.restype = None
            lib.oracle_rank.argtypes = [P, i64, P]
            lib.oracle_topk.restype = None
            lib.oracle_topk.argtypes = [P, P, i64, i64, i64, i32, cint, f64, f64, f64,
                                        P, f64, P, P, P, P, cint, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def idf(variant: int, n_docs: float, df: float) -> float:
    return _load().oracle_idf(variant, float(n_docs), float(df))


def term_score(variant: int, idf_t: float, tf: float, doc_len: float, lavg: float,
               k1: float, b: float, delta: float) -> float:
    return _load().oracle_term_score(variant, idf_t, float(tf), float(doc_len), lavg,
                                     k1, b, delta)


def nonoccurrence(variant: int, idf_t: float, k1: float, b: float, delta: float) -> float:
    return _load().oracle_nonoccurrence(variant, idf_t, k1, b, delta)


@dataclass
class OracleIndex:
    n_docs: int
    vocab: int
    variant: int
    k1: float
    b: float
    delta: float
    doc_len: np.ndarray      # int64 [N]
    lavg: float
    pair_start: np.ndarray   # int64 [N+1]   doc-major pair offsets
    pair_term: np.ndarray    # int32 [nnz]
    pair_tf: np.ndarray      # int32 [nnz]
    df: np.ndarray           # int64 [V]
    idf: np.ndarray          # f64 [V]
    s0: np.ndarray           # f64 [V]
    indptr: np.ndarray       # int64 [V+1]   term-major CSC
    indices: np.ndarray      # int32 [nnz]   doc ids ascending per term
    csc_tf: np.ndarray       # int32 [nnz]
    csc_delta: np.ndarray    # f64 [nnz]     S - S0

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])


def build(tokens, doc_offsets, vocab: int, variant: int = LUCENE, k1: float = 1.5,
          b: float = 0.75, delta: float = 0.5) -> OracleIndex:
    """Index a corpus: tokens[int32], doc_offsets[int64, N+1]."""
    tok = np.ascontiguousarray(tokens, dtype=np.int32)
    off = np.ascontiguousarray(doc_offsets, dtype=np.int64)
    n = off.shape[0] - 1
    t = tok.shape[0]
    cap = max(t, 1)
    doc_len = np.zeros(max(n, 1), np.int64)
    lavg = ctypes.c_double(0.0)
    pair_start = np.zeros(n + 1, np.int64)
    pair_term = np.zeros(cap, np.int32)
    pair_tf = np.zeros(cap, np.int32)
    df = np.zeros(vocab, np.int64)
    idf_ = np.zeros(vocab, np.float64)
    s0 = np.zeros(vocab, np.float64)
    indptr = np.zeros(vocab + 1, np.int64)
    indices = np.zeros(cap, np.int32)
    csc_tf = np.zeros(cap, np.int32)
    csc_delta = np.zeros(cap, np.float64)
    nnz = _load().oracle_build(_p(tok), t, _p(off), n, vocab, variant, k1, b, delta,
                               _p(doc_len), ctypes.byref(lavg), _p(pair_start),
                               _p(pair_term), _p(pair_tf), _p(df), _p(idf_), _p(s0),
                               _p(indptr), _p(indices), _p(csc_tf), _p(csc_delta))
    if nnz < 0:
        raise ValueError("oracle_build: invalid corpus (token outside [0, vocab) or bad offsets)")
    return OracleIndex(n, vocab, variant, k1, b, delta, doc_len[:n], lavg.value, pair_start,
                       pair_term[:nnz], pair_tf[:nnz], df, idf_, s0, indptr,
                       indices[:nnz], csc_tf[:nnz], csc_delta[:nnz])


def _params(ix: OracleIndex, k1, b, delta):
    """The index's k1, b, delta, or the ones a query passes (query-time
    scoring: the lazy oracle evaluates S from TF anyway)."""
    return (ix.k1 if k1 is None else float(k1), ix.b if b is None else float(b),
            ix.delta if delta is None else float(delta))


def score_all(ix: OracleIndex, query, with_abs: bool = False, k1=None, b=None, delta=None):
    """Lazy B(Q,D) for every document, FP64.  With with_abs, also returns
    sum_i |S(q_i, D)| per document.  k1 / b / delta override the index's."""
    q = np.ascontiguousarray(query, dtype=np.int32)
    out = np.zeros(ix.n_docs, np.float64)
    ab = np.zeros(ix.n_docs, np.float64) if with_abs else None
    pk1, pb, pd = _params(ix, k1, b, delta)
    _load().oracle_score_all(_p(q), q.shape[0], ix.n_docs, ix.vocab, ix.variant, pk1,
                             pb, pd, _p(ix.doc_len), ix.lavg, _p(ix.pair_start),
                             _p(ix.pair_term), _p(ix.pair_tf), _p(ix.idf), _p(out),
                             _p(ab) if with_abs else None)
    return (out, ab) if with_abs else out


def rank(scores: np.ndarray) -> np.ndarray:
    """All document ids ordered by (score desc, id asc)."""
    sc = np.ascontiguousarray(scores, dtype=np.float64)
    order = np.zeros(sc.shape[0], np.int64)
    _load().oracle_rank(_p(sc), sc.shape[0], _p(order))
    return order


def topk(ix: OracleIndex, q_tokens, q_offsets, k: int, n_threads: int = 1, k1=None, b=None,
         delta=None):
    """Top-k (ids int64, scores f64) for a batch of queries, lazy + full sort.
    k1 / b / delta override the index's."""
    qt = np.ascontiguousarray(q_tokens, dtype=np.int32)
    qo = np.ascontiguousarray(q_offsets, dtype=np.int64)
    nq = qo.shape[0] - 1
    ids = np.zeros((max(nq, 1), k), np.int64)
    sc = np.zeros((max(nq, 1), k), np.float64)
    if qt.shape[0] == 0:
        qt = np.zeros(1, np.int32)
    pk1, pb, pd = _params(ix, k1, b, delta)
    _load().oracle_topk(_p(qt), _p(qo), nq, k, ix.n_docs, ix.vocab, ix.variant, pk1,
                        pb, pd, _p(ix.doc_len), ix.lavg, _p(ix.pair_start),
                        _p(ix.pair_term), _p(ix.pair_tf), _p(ix.idf), n_threads,
                        _p(ids), _p(sc))
    return ids[:nq], sc[:nq]

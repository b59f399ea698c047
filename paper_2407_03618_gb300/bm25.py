"""Python binding of libbm25gpu: argument marshalling only.

Every step of index build and retrieval runs in the library's CUDA kernels;
this module converts torch tensors / numpy arrays to pointers, passes the
current torch CUDA stream, and raises on a non-zero status.  PyTorch is used
for device memory and streams, nothing else.  If the library has not been
built the module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build_ext

VARIANTS = {"lucene": 0, "robertson": 1, "atire": 2, "bm25l": 3, "bm25+": 4, "tfldp": 5}
ACC_UNSET, ACC_AUTO, ACC_SMEM_TILED, ACC_L2_DENSE = 0, 1, 2, 3
STATUS = {0: "BM25_OK", -1: "BM25_E_INVALID", -2: "BM25_E_TOKEN_RANGE", -3: "BM25_E_OOM",
          -4: "BM25_E_CUDA", -5: "BM25_E_TIMEOUT", 1: "BM25_PENDING"}
PENDING = 1
MAX_K = 4096


class Plan(ctypes.Structure):
    """bm25_plan: how retrieval runs (zero fields = library defaults)."""
    _fields_ = [("accumulator", ctypes.c_int32), ("tile_docs", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("dense_max_postings", ctypes.c_int32),
                ("stage_entries", ctypes.c_int32), ("stages", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"accumulator": self.accumulator, "tile_docs": self.tile_docs,
                "block_threads": self.block_threads,
                "dense_max_postings": self.dense_max_postings,
                "stage_entries": self.stage_entries, "stages": self.stages}


class ServerConfig(ctypes.Structure):
    """bm25_server_config (zero fields = defaults)."""
    _fields_ = [("max_batch_queries", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("k_max", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("batched_queries", ctypes.c_int64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("bytes_held", ctypes.c_int64),
                ("span_us", ctypes.c_double)]


class BM25Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/bm25.h."""
    with open(os.path.join(build_ext.INCLUDE, "bm25.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"\b(bm25_\w+)\s*\(", text)


def load(path: str | None = None):
    """Load libbm25gpu.so (built by build_ext.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or build_ext.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libbm25gpu.so is not built ({path}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, i32, i64, f64, cint = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                              ctypes.c_int)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "bm25_index_build": (cint, [P, i64, P, i64, i32, cint, f64, f64, f64, P, PP]),
        "bm25_index_build_host": (cint, [P, i64, P, i64, i32, cint, f64, f64, f64, P, PP]),
        "bm25_index_info": (cint, [P, P, P, P, P, P, P, P, P, P]),
        "bm25_index_export": (cint, [P, P, P, P, P, P, P, P, P]),
        "bm25_index_import": (cint, [i64, i64, i64, i32, cint, f64, f64, f64, f64,
                                     P, P, P, P, P, P, P, P, PP]),
        "bm25_sync_status": (cint, [P, P]),
        "bm25_index_free": (None, [P]),
        "bm25_release_cached": (None, []),
        "bm25_retrieve": (cint, [P, P, i64, P, i32, i32, P, P, P]),
        "bm25_retrieve_host": (cint, [P, P, P, i32, i32, P, P, P]),
        "bm25_retrieve_noalloc": (cint, [P, P, i64, P, i32, i32, P, P, P]),
        "bm25_workspace_create": (cint, [P, i32, i64, i32, PP]),
        "bm25_workspace_free": (None, [P]),
        "bm25_retrieve_ws": (cint, [P, P, P, i64, P, i32, i32, P, P, P, P]),
        "bm25_retrieve_batch": (cint, [P, P, P, i64, P, i32, P, i32, P, P, P, P]),
        "bm25_workspace_reserve": (cint, [P, P, i32, i64, i32, P, P]),
        "bm25_autotune": (cint, [P, P, i64, P, i32, i32, P, P, P, P, P, i32, P]),
        "bm25_server_create": (cint, [P, i32, P, PP]),
        "bm25_server_submit": (cint, [P, i32, P, i32, i32, P]),
        "bm25_server_poll": (cint, [P, i64, P, P, i32]),
        "bm25_server_stats_get": (cint, [P, cint, P]),
        "bm25_server_replay": (cint, [P, i32, P, P, P, P, P, P]),
        "bm25_replay_plain": (cint, [P, i32, i32, P, P, P, P, P, P, P]),
        "bm25_server_destroy": (None, [P]),
        "bm25_index_set_plan": (cint, [P, P]),
        "bm25_index_get_plan": (cint, [P, P]),
        "bm25_last_error": (ctypes.c_char_p, []),
        "bm25_launch_count": (i64, []),
        "bm25_version": (ctypes.c_char_p, []),
        "bm25_profile_begin": (cint, []),
        "bm25_profile_end": (cint, []),
        "bm25_profile_count": (cint, []),
        "bm25_profile_get": (cint, [cint, ctypes.c_char_p, cint, P, P]),
        "bm25_tokenize_corpus": (cint, [P, i64, P, i64, P, P, i32, P, i64, P, P, PP, P]),
        "bm25_tokenize_queries": (cint, [P, P, i64, P, i64, P, i64, P, P, P]),
        "bm25_vocab_info": (cint, [P, P, P]),
        "bm25_vocab_export": (cint, [P, P, P]),
        "bm25_vocab_free": (None, [P]),
        "bm25_index_enable_lazy": (cint, [P, P]),
        "bm25_retrieve_lazy": (cint, [P, P, i64, P, i32, i32, f64, f64, f64, P, P, P]),
        "bm25_index_df_device": (cint, [P, P, P]),
        "bm25_index_rescore": (cint, [P, P, i64, i64, i64, P]),
        "bm25_index_shard_info": (cint, [P, P, P, P]),
        "bm25_merge_topk": (cint, [P, P, i32, i32, i32, P, P, P]),
        "bm25_debug_set_handshake_polls": (cint, [i32]),
        "bm25_debug_fail_allocs": (cint, [i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise BM25Error(rc, load().bm25_last_error().decode())


def debug_set_handshake_polls(polls: int):
    """Test hook: polls after which a wait of the tiled kernel gives up (< 0: default)."""
    _check(load().bm25_debug_set_handshake_polls(polls))


def debug_fail_allocs(n: int):
    """Test hook: the next n device allocations of the library fail with BM25_E_OOM."""
    _check(load().bm25_debug_fail_allocs(n))


def merge_topk(cand_ids, cand_scores, k: int, out=None, stream=None):
    """Merge shard rows: cand_ids int32 / cand_scores float32 CUDA tensors
    [n_shards, n_queries, k] -> (ids, scores) [n_queries, k]."""
    import torch
    ci = _dev_tensor(cand_ids, torch.int32)
    cs = _dev_tensor(cand_scores, torch.float32)
    g, nq = int(ci.shape[0]), int(ci.shape[1])
    if out is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=ci.device)
        sc = torch.empty((nq, k), dtype=torch.float32, device=ci.device)
    else:
        ids, sc = out
    _check(load().bm25_merge_topk(ci.data_ptr(), cs.data_ptr(), g, nq, k, ids.data_ptr(),
                                  sc.data_ptr(), _stream(stream)))
    return ids, sc


class Vocab:
    """A vocabulary built on the device by tokenize_corpus."""

    def __init__(self, handle):
        self.handle = handle

    def info(self) -> dict:
        n, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().bm25_vocab_info(self.handle, ctypes.byref(n), ctypes.byref(b)))
        return {"n_words": n.value, "n_bytes": b.value}

    def words(self) -> list:
        """The words (lowercased bytes) in id order."""
        inf = self.info()
        buf = np.zeros(max(inf["n_bytes"], 1), np.uint8)
        off = np.zeros(inf["n_words"] + 1, np.int64)
        _check(load().bm25_vocab_export(self.handle, _ptr(buf), _ptr(off)))
        raw = buf.tobytes()
        return [raw[off[i]:off[i + 1]] for i in range(inf["n_words"])]

    def close(self):
        if self.handle:
            load().bm25_vocab_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stopword_arrays(stopwords):
    words = [bytes(w) for w in stopwords]
    off = np.zeros(len(words) + 1, np.int64)
    off[1:] = np.cumsum([len(w) for w in words])
    buf = np.frombuffer(b"".join(words) or b"\0", np.uint8).copy()
    return buf, off


def tokenize_corpus(text, doc_offsets, stopwords=(), stream=None):
    """Term ids of a corpus of UTF-8 texts on the device: text CUDA uint8,
    doc_offsets CUDA int64 [N+1].  Returns (token_ids CUDA int32 [T],
    token_offsets CUDA int64 [N+1], Vocab)."""
    import torch
    tx = _dev_tensor(text, torch.uint8)
    do = _dev_tensor(doc_offsets, torch.int64)
    n = do.numel() - 1
    cap = tx.numel() // 2 + 1
    ids = torch.empty(cap, dtype=torch.int32, device=tx.device)
    offs = torch.empty(n + 1, dtype=torch.int64, device=tx.device)
    sb, so = _stopword_arrays(stopwords)
    nt = ctypes.c_int64()
    h = ctypes.c_void_p()
    _check(load().bm25_tokenize_corpus(tx.data_ptr(), tx.numel(), do.data_ptr(), n, _ptr(sb),
                                       _ptr(so), len(so) - 1, ids.data_ptr(), cap, offs.data_ptr(),
                                       ctypes.byref(nt), ctypes.byref(h), _stream(stream)))
    return ids[:nt.value], offs, Vocab(h.value)


def tokenize_queries(vocab: Vocab, text, offsets, stream=None):
    """Term ids of query texts with a corpus vocabulary (unknown words
    dropped).  Returns (token_ids CUDA int32, token_offsets CUDA int64)."""
    import torch
    tx = _dev_tensor(text, torch.uint8)
    qo = _dev_tensor(offsets, torch.int64)
    n = qo.numel() - 1
    cap = tx.numel() // 2 + 1
    ids = torch.empty(cap, dtype=torch.int32, device=tx.device)
    offs = torch.empty(n + 1, dtype=torch.int64, device=tx.device)
    nt = ctypes.c_int64()
    _check(load().bm25_tokenize_queries(vocab.handle, tx.data_ptr(), tx.numel(), qo.data_ptr(), n,
                                        ids.data_ptr(), cap, offs.data_ptr(), ctypes.byref(nt),
                                        _stream(stream)))
    return ids[:nt.value], offs


def replay_plain(indexes: list, index_ids, queries: list, ks, arrival_s, stream=None):
    """The same requests through the one-query-per-call host path, served
    in order natively; returns each request's latency in microseconds."""
    n = len(queries)
    arr_ix = (ctypes.c_void_p * len(indexes))(*[ix.handle.value for ix in indexes])
    ids_a = np.ascontiguousarray(index_ids, np.int32)
    ks_a = np.ascontiguousarray(ks, np.int32)
    arr = np.ascontiguousarray(arrival_s, np.float64)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in queries])
    tok = (np.concatenate([np.asarray(x, np.int32) for x in queries]) if off[-1]
           else np.zeros(1, np.int32))
    lat = np.zeros(max(n, 1), np.float64)
    _check(load().bm25_replay_plain(arr_ix, len(indexes), n, _ptr(ids_a), _ptr(tok), _ptr(off),
                                    _ptr(ks_a), _ptr(arr), _ptr(lat), _stream(stream)))
    return lat[:n]


def release_cached():
    """Free the retrieval scratch kept from freed indexes (all devices)."""
    load().bm25_release_cached()


def launch_count() -> int:
    return int(load().bm25_launch_count())


def profile_begin():
    """Start bracketing every library kernel launch with CUDA events."""
    _check(load().bm25_profile_begin())


def profile_end() -> dict:
    """Stop; returns {kernel name: (launches, total milliseconds)}."""
    lib = load()
    _check(lib.bm25_profile_end())
    out = {}
    buf = ctypes.create_string_buffer(128)
    for i in range(lib.bm25_profile_count()):
        n, ms = ctypes.c_int64(), ctypes.c_double()
        _check(lib.bm25_profile_get(i, buf, 128, ctypes.byref(n), ctypes.byref(ms)))
        out[buf.value.decode()] = (n.value, ms.value)
    return out


def _stream(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_tensor(x, dtype):
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if x.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {x.dtype}")
    return x.contiguous()


def _np(x, dtype):
    return np.ascontiguousarray(x, dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Workspace:
    """Scratch memory for retrieval, sized once (no allocation inside calls
    that stay within its limits)."""

    def __init__(self, index: "Index", max_queries: int, max_query_tokens: int, max_k: int):
        h = ctypes.c_void_p()
        _check(load().bm25_workspace_create(index.handle, max_queries, max_query_tokens, max_k,
                                            ctypes.byref(h)))
        self.handle = h

    def reserve(self, index: "Index", n_queries: int, n_query_tokens: int, k_max: int,
                plan: dict | None = None, stream=None):
        """Grow to what one such call needs (do this before graph capture)."""
        p = Plan(**(plan or {}))
        _check(load().bm25_workspace_reserve(self.handle, index.handle, n_queries,
                                             n_query_tokens, k_max, ctypes.byref(p),
                                             _stream(stream)))

    def close(self):
        if self.handle:
            load().bm25_workspace_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Index:
    """A BM25 index resident on one GPU (term-major CSC of S - S0)."""

    def __init__(self, handle):
        self.handle = handle
        self._refs = []

    # ---- construction ----
    @classmethod
    def build(cls, tokens, doc_offsets, vocab: int, variant="lucene", k1: float = 1.5,
              b: float = 0.75, delta: float = 0.5, stream=None) -> "Index":
        """tokens: CUDA int32 [T]; doc_offsets: CUDA int64 [N+1]."""
        import torch
        tok = _dev_tensor(tokens, torch.int32)
        off = _dev_tensor(doc_offsets, torch.int64)
        h = ctypes.c_void_p()
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        _check(load().bm25_index_build(tok.data_ptr(), tok.numel(), off.data_ptr(),
                                       off.numel() - 1, vocab, v, k1, b, delta,
                                       _stream(stream), ctypes.byref(h)))
        return cls(h)

    @classmethod
    def build_host(cls, tokens, doc_offsets, vocab: int, variant="lucene", k1: float = 1.5,
                   b: float = 0.75, delta: float = 0.5, stream=None) -> "Index":
        """tokens / doc_offsets in host memory (numpy or pinned CPU tensors)."""
        tok = _host_array(tokens, np.int32)
        off = _host_array(doc_offsets, np.int64)
        h = ctypes.c_void_p()
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        _check(load().bm25_index_build_host(_hptr(tok), _hlen(tok), _hptr(off), _hlen(off) - 1,
                                            vocab, v, k1, b, delta, _stream(stream),
                                            ctypes.byref(h)))
        return cls(h)

    @classmethod
    def load_arrays(cls, arrays: dict) -> "Index":
        """Rebuild an index from export() output (checkpoint resume)."""
        a = arrays
        h = ctypes.c_void_p()
        keep = {k: _np(a[k], dt) for k, dt in (("indptr", np.int64), ("indices", np.int32),
                                               ("data", np.float32), ("tf", np.int32),
                                               ("df", np.int32), ("doc_len", np.int32),
                                               ("idf", np.float64), ("s0", np.float64))}
        _check(load().bm25_index_import(int(a["n_docs"]), int(a["n_tokens"]), int(a["nnz"]),
                                        int(a["vocab"]), int(a["variant"]), float(a["k1"]),
                                        float(a["b"]), float(a["delta"]), float(a["lavg"]),
                                        *[_ptr(keep[k]) for k in ("indptr", "indices", "data",
                                                                  "tf", "df", "doc_len", "idf",
                                                                  "s0")],
                                        ctypes.byref(h)))
        return cls(h)

    # ---- queries ----
    def info(self) -> dict:
        n, t, z = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        v, var = ctypes.c_int32(), ctypes.c_int()
        k1, b, d, la = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().bm25_index_info(self.handle, *[ctypes.byref(x) for x in
                                                     (n, t, z, v, var, k1, b, d, la)]))
        return {"n_docs": n.value, "n_tokens": t.value, "nnz": z.value, "vocab": v.value,
                "variant": var.value, "k1": k1.value, "b": b.value, "delta": d.value,
                "lavg": la.value}

    def export(self, fields=None) -> dict:
        """The index's arrays in host memory (all of them, or the named ones)."""
        inf = self.info()
        V, N, Z = inf["vocab"], inf["n_docs"], inf["nnz"]
        shapes = {"indptr": (V + 1, np.int64), "indices": (Z, np.int32), "data": (Z, np.float32),
                  "tf": (Z, np.int32), "df": (V, np.int32), "doc_len": (N, np.int32),
                  "idf": (V, np.float64), "s0": (V, np.float64)}
        names = list(shapes) if fields is None else list(fields)
        out = {k: np.zeros(shapes[k][0], shapes[k][1]) for k in names}
        _check(load().bm25_index_export(self.handle, *[_ptr(out[k]) if k in out else None
                                                       for k in shapes]))
        out.update(inf)
        return out

    def set_plan(self, accumulator: int = ACC_UNSET, tile_docs: int = 0, block_threads: int = 0,
                 dense_max_postings: int = 0, stage_entries: int = 0, stages: int = 0):
        p = Plan(accumulator, tile_docs, block_threads, dense_max_postings, stage_entries, stages)
        _check(load().bm25_index_set_plan(self.handle, ctypes.byref(p)))

    def autotune(self, q_tokens, q_offsets, k: int, stream=None):
        """Time candidate plans on a sample batch (CUDA tensors) and keep the
        fastest.  Returns (best plan dict, best ms, [(plan dict, ms), ...])."""
        import torch
        qt = _dev_tensor(q_tokens, torch.int32)
        qo = _dev_tensor(q_offsets, torch.int64)
        best, best_ms = Plan(), ctypes.c_double()
        cap = 32
        tried = (Plan * cap)()
        tried_ms = (ctypes.c_double * cap)()
        n = ctypes.c_int32()
        _check(load().bm25_autotune(self.handle, qt.data_ptr(), qt.numel(), qo.data_ptr(),
                                    qo.numel() - 1, k, _stream(stream), ctypes.byref(best),
                                    ctypes.byref(best_ms), tried, tried_ms, cap,
                                    ctypes.byref(n)))
        log = [(tried[i].as_dict(), tried_ms[i]) for i in range(min(n.value, cap))]
        return best.as_dict(), best_ms.value, log

    def get_plan(self) -> dict:
        p = Plan()
        _check(load().bm25_index_get_plan(self.handle, ctypes.byref(p)))
        return p.as_dict()

    def enable_lazy(self, stream=None):
        """Add the lazy postings (doc id with TF and |D|) that query-time
        scoring reads."""
        _check(load().bm25_index_enable_lazy(self.handle, _stream(stream)))

    def retrieve_lazy(self, q_tokens, q_offsets, k: int, k1: float, b: float, delta: float = 0.5,
                      out=None, stream=None):
        """Top k with S(t,D) computed at query time with k1, b, delta (CUDA
        tensors as in retrieve)."""
        import torch
        qt = _dev_tensor(q_tokens, torch.int32)
        qo = _dev_tensor(q_offsets, torch.int64)
        nq = qo.numel() - 1
        if out is None:
            ids = torch.empty((nq, max(k, 0)), dtype=torch.int32, device=qo.device)
            sc = torch.empty((nq, max(k, 0)), dtype=torch.float32, device=qo.device)
        else:
            ids, sc = out
        _check(load().bm25_retrieve_lazy(self.handle, qt.data_ptr(), qt.numel(), qo.data_ptr(),
                                         nq, k, float(k1), float(b), float(delta), ids.data_ptr(),
                                         sc.data_ptr(), _stream(stream)))
        return ids, sc

    def df_device(self, out=None, stream=None):
        """The index's DF as a CUDA int32 tensor [vocab]."""
        import torch
        v = self.info()["vocab"]
        if out is None:
            out = torch.empty(v, dtype=torch.int32, device=torch.device("cuda",
                                                                          torch.cuda.current_device()))
        _check(load().bm25_index_df_device(self.handle, out.data_ptr(), _stream(stream)))
        return out

    def rescore(self, global_df, global_n_docs: int, global_n_tokens: int, doc_id_offset: int,
                stream=None):
        """Apply a collection's statistics to this doc-range shard (global_df:
        CUDA int32 [vocab] or None) and set its global doc-id offset."""
        import torch
        p = None
        if global_df is not None:
            global_df = _dev_tensor(global_df, torch.int32)
            p = global_df.data_ptr()
        _check(load().bm25_index_rescore(self.handle, p, int(global_n_docs), int(global_n_tokens),
                                         int(doc_id_offset), _stream(stream)))

    def shard_info(self) -> dict:
        off, nd, nt = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().bm25_index_shard_info(self.handle, ctypes.byref(off), ctypes.byref(nd),
                                            ctypes.byref(nt)))
        return {"doc_id_offset": off.value, "global_n_docs": nd.value,
                "global_n_tokens": nt.value}

    def sync_status(self, stream=None):
        _check(load().bm25_sync_status(self.handle, _stream(stream)))

    def retrieve(self, q_tokens, q_offsets, k: int, out=None, stream=None,
                 workspace: Workspace | None = None, plan: dict | None = None):
        """Device path.  q_tokens CUDA int32, q_offsets CUDA int64 [nQ+1].
        Returns (ids int32 [nQ, k], scores float32 [nQ, k]) CUDA tensors."""
        import torch
        qt = _dev_tensor(q_tokens, torch.int32)
        qo = _dev_tensor(q_offsets, torch.int64)
        nq = qo.numel() - 1
        if out is None:  # k < 1 reaches the library, which rejects it
            ids = torch.empty((nq, max(k, 0)), dtype=torch.int32, device=qo.device)
            sc = torch.empty((nq, max(k, 0)), dtype=torch.float32, device=qo.device)
        else:
            ids, sc = out
        if workspace is None and plan is None:
            _check(load().bm25_retrieve(self.handle, qt.data_ptr(), qt.numel(), qo.data_ptr(), nq,
                                        k, ids.data_ptr(), sc.data_ptr(), _stream(stream)))
        else:
            if workspace is None:
                workspace = self._default_workspace(nq, qt.numel(), k)
            p = Plan(**(plan or {}))
            _check(load().bm25_retrieve_ws(self.handle, workspace.handle, qt.data_ptr(),
                                           qt.numel(), qo.data_ptr(), nq, k, ids.data_ptr(),
                                           sc.data_ptr(), ctypes.byref(p), _stream(stream)))
        return ids, sc

    def retrieve_batch(self, q_tokens, q_offsets, k_max: int, q_k=None, out=None, stream=None,
                       workspace: Workspace | None = None, plan: dict | None = None):
        """Queries with different k in one call: q_k CUDA int32 [nQ] (None =
        k_max for all).  Returns (ids, scores) [nQ, k_max]; row q holds
        min(q_k[q], N) results, then -1 / -inf."""
        import torch
        qt = _dev_tensor(q_tokens, torch.int32)
        qo = _dev_tensor(q_offsets, torch.int64)
        nq = qo.numel() - 1
        qk = _dev_tensor(q_k, torch.int32) if q_k is not None else None
        if out is None:
            ids = torch.empty((nq, max(k_max, 0)), dtype=torch.int32, device=qo.device)
            sc = torch.empty((nq, max(k_max, 0)), dtype=torch.float32, device=qo.device)
        else:
            ids, sc = out
        p = Plan(**(plan or {}))
        _check(load().bm25_retrieve_batch(self.handle, workspace.handle if workspace else None,
                                          qt.data_ptr(), qt.numel(), qo.data_ptr(), nq,
                                          qk.data_ptr() if qk is not None else None, k_max,
                                          ids.data_ptr(), sc.data_ptr(), ctypes.byref(p),
                                          _stream(stream)))
        return ids, sc

    def _default_workspace(self, nq, ntok, k):
        ws = Workspace(self, max(nq, 1), ntok, k)
        self._refs.append(ws)
        return ws

    def retrieve_host(self, q_tokens, q_offsets, k: int, out=None, stream=None):
        """Host path: inputs and outputs in host memory (numpy or pinned CPU
        tensors).  Returns (ids, scores) as given in `out` or new numpy arrays."""
        qt = _host_array(q_tokens, np.int32)
        qo = _host_array(q_offsets, np.int64)
        nq = _hlen(qo) - 1
        if out is None:
            ids = np.zeros((nq, max(k, 0)), np.int32)
            sc = np.zeros((nq, max(k, 0)), np.float32)
        else:
            ids, sc = out
        _check(load().bm25_retrieve_host(self.handle, _hptr(qt), _hptr(qo), nq, k, _hptr(ids),
                                         _hptr(sc), _stream(stream)))
        return ids, sc

    def close(self):
        if self.handle:
            for ws in self._refs:
                ws.close()
            self._refs = []
            load().bm25_index_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_array(x, dtype):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.is_cuda:
                raise TypeError("expected host memory")
            return x.contiguous()
    except ImportError:
        pass
    return _np(x, dtype)


def _hptr(x):
    if isinstance(x, np.ndarray):
        return _ptr(x)
    return ctypes.c_void_p(x.data_ptr())


def _hlen(x) -> int:
    return int(x.shape[0]) if isinstance(x, np.ndarray) else int(x.numel())


class Server:
    """Continuous-batching request loop over resident indexes (a worker
    thread inside the library; queries and results in host memory)."""

    def __init__(self, indexes: list, max_batch_queries: int = 0, max_inflight: int = 0,
                 k_max: int = 0, memory_budget: int = 0):
        self._indexes = list(indexes)  # kept alive while the server runs
        arr = (ctypes.c_void_p * len(indexes))(*[ix.handle.value for ix in indexes])
        cfg = ServerConfig(max_batch_queries, max_inflight, k_max, 0, memory_budget)
        h = ctypes.c_void_p()
        _check(load().bm25_server_create(arr, len(indexes), ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h

    def submit(self, index_id: int, tokens, k: int) -> int:
        t = _np(tokens, np.int32)
        ticket = ctypes.c_int64()
        _check(load().bm25_server_submit(self.handle, index_id, _ptr(t), int(t.shape[0]), k,
                                         ctypes.byref(ticket)))
        return ticket.value

    def poll(self, ticket: int, k: int, timeout_us: int = -1):
        """(ids, scores) numpy arrays of length k, or None while pending."""
        ids = np.zeros(k, np.int32)
        sc = np.zeros(k, np.float32)
        rc = load().bm25_server_poll(self.handle, ticket, _ptr(ids), _ptr(sc), timeout_us)
        if rc == PENDING:
            return None
        _check(rc)
        return ids, sc

    def replay(self, index_ids, queries: list, ks, arrival_s) -> list:
        """Submit request i (queries[i] on index_ids[i] at k = ks[i]) at
        arrival_s[i] seconds from now, natively; returns the tickets."""
        n = len(queries)
        ids_a = np.ascontiguousarray(index_ids, np.int32)
        ks_a = np.ascontiguousarray(ks, np.int32)
        arr = np.ascontiguousarray(arrival_s, np.float64)
        off = np.zeros(n + 1, np.int64)
        off[1:] = np.cumsum([len(x) for x in queries])
        tok = (np.concatenate([np.asarray(x, np.int32) for x in queries]) if off[-1]
               else np.zeros(1, np.int32))
        tickets = np.zeros(max(n, 1), np.int64)
        _check(load().bm25_server_replay(self.handle, n, _ptr(ids_a), _ptr(tok), _ptr(off),
                                         _ptr(ks_a), _ptr(arr), _ptr(tickets)))
        return tickets[:n].tolist()

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _check(load().bm25_server_stats_get(self.handle, int(reset), ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            load().bm25_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

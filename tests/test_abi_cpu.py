"""The C-ABI library builds, loads without a GPU, exports every function
include/bm25.h declares, and rejects bad arguments on the host before any
CUDA call."""
import ctypes
import os

import pytest

from paper_2407_03618_gb300 import bm25, build_ext


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return bm25.load()


def test_exports_every_declared_function(lib):
    names = bm25.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), f"{name} declared in bm25.h but not exported"


def test_version_and_launch_counter(lib):
    assert b"sm_103a" in lib.bm25_version()
    assert lib.bm25_launch_count() >= 0


@pytest.mark.parametrize("args, msg", [
    (dict(variant=7), b"variant"),
    (dict(k1=-1.0), b"k1"),
    (dict(b=1.5), b"b <= 1"),
    (dict(delta=-0.1), b"delta"),
    (dict(n_docs=0), b"n_docs"),
    (dict(vocab=0), b"vocab"),
    (dict(n_tokens=-1), b"n_tokens"),
    (dict(variant=3, k1=0.0, delta=0.0), b"BM25L"),
])
def test_build_rejects_bad_arguments_on_host(lib, args, msg):
    a = dict(n_tokens=4, n_docs=2, vocab=3, variant=0, k1=1.5, b=0.75, delta=0.5)
    a.update(args)
    h = ctypes.c_void_p(1)
    rc = lib.bm25_index_build(None, a["n_tokens"], None, a["n_docs"], a["vocab"], a["variant"],
                              a["k1"], a["b"], a["delta"], None, ctypes.byref(h))
    assert rc == -1
    assert h.value is None
    assert msg in lib.bm25_last_error()


def test_null_handles_are_rejected(lib):
    assert lib.bm25_index_info(None, *([None] * 9)) == -1
    assert lib.bm25_sync_status(None, None) == -1
    lib.bm25_index_free(None)
    lib.bm25_workspace_free(None)
    assert lib.bm25_index_set_plan(None, None) == -1
    assert lib.bm25_index_get_plan(None, None) == -1


def test_missing_library_fails_loudly(monkeypatch):
    # no fallback of any kind: without the built library the binding raises
    monkeypatch.setattr(bm25, "_lib", None)
    missing = os.path.join(build_ext.PKG, "_missing", "libbm25gpu.so")
    assert not os.path.exists(missing)
    with pytest.raises(RuntimeError, match="not built"):
        bm25.load(missing)
    monkeypatch.setattr(build_ext, "LIB_PATH", missing)
    with pytest.raises(RuntimeError, match="not built"):
        bm25.load()

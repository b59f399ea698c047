"""bench.py's roofline `traffic`: read from a profile's "key: value" lines only
for the code, workload and plan the counters were taken on; the code stamp
ignores comments, whitespace and where the repository lives."""
import os

import bench
from paper_2407_03618_gb300 import build_ext


def _profile(**kv):
    body = "# k — DRAM traffic\n\nCommand: ncu ... (a prose line with a colon)\n\n"
    return body + "".join(f"{k}: {v}\n" for k, v in kv.items())


def test_plan_key_order():
    plan = {"dense_max_postings": 4096, "block_threads": 192, "tile_docs": 10240,
            "accumulator": 1}
    assert bench.plan_key(plan) == "1,10240,192,4096"


def test_matching_stamp_workload_and_plan():
    t = _profile(code_stamp="abc", workload="zipf-1m", plan="1,10240,192,4096",
                 traffic_bytes_per_launch=300100000)
    assert bench.parse_traffic(t, "abc", "zipf-1m", "1,10240,192,4096") == 300100000


def test_any_mismatch_gives_none():
    t = _profile(code_stamp="abc", workload="zipf-1m", plan="1,10240,192,4096",
                 traffic_bytes_per_launch=300100000)
    assert bench.parse_traffic(t, "abd", "zipf-1m", "1,10240,192,4096") is None
    assert bench.parse_traffic(t, "abc", "tiny-2k", "1,10240,192,4096") is None
    assert bench.parse_traffic(t, "abc", "zipf-1m", "1,10240,192,2048") is None


def test_profile_without_a_plan_holds_for_any_plan():
    t = _profile(code_stamp="abc", workload="zipf-1m", traffic_bytes_per_launch=7)
    assert bench.parse_traffic(t, "abc", "zipf-1m", "2,7168,256,0") == 7


def test_missing_or_malformed_gives_none():
    assert bench.read_traffic(os.path.join(bench.ROOT, "profiles", "absent.md"), "abc",
                              "zipf-1m", "x") is None
    t = _profile(code_stamp="abc", workload="zipf-1m", traffic_bytes_per_launch="n/a")
    assert bench.parse_traffic(t, "abc", "zipf-1m", "x") is None


def test_committed_profiles_are_readable():
    """Every committed traffic profile carries the four keys; bench.py uses its
    figure only while the code still hashes to the recorded stamp."""
    import glob
    paths = glob.glob(os.path.join(bench.ROOT, "profiles", "*_traffic.md"))
    assert paths
    keys = ("code_stamp", "plan", "workload", "traffic_bytes_per_launch")
    for path in paths:
        kv = {}
        for line in open(path).read().splitlines():
            key, sep, val = line.partition(":")
            if sep and key in keys:
                kv[key] = val.strip()
        assert set(kv) == set(keys), path
        got = bench.read_traffic(path, build_ext.code_stamp(), kv["workload"], kv["plan"])
        if kv["code_stamp"] == build_ext.code_stamp():
            assert got == int(kv["traffic_bytes_per_launch"])
        else:
            assert got is None


def test_strip_c_comments():
    src = ('int a = 1; // c\'mon "x"\n'
           'const char* p = "// not a comment"; /* block\n comment */ char q = \'\\\'\';\n'
           "char r = '\"';   int  b=2;\n")
    assert build_ext.strip_c_comments(src) == \
        "int a = 1; const char* p = \"// not a comment\"; char q = '\\''; char r = '\"'; int b=2;"
    assert build_ext.strip_c_comments("x /* a */ y\n\n  // b\nz") == "x y z"


def test_code_stamp_ignores_include_paths(monkeypatch):
    s0 = build_ext.code_stamp()
    flags = [f if not f.startswith("-I") else "-I/elsewhere" + f[2:] for f in build_ext.NVCC_FLAGS]
    monkeypatch.setattr(build_ext, "NVCC_FLAGS", flags)
    assert build_ext.code_stamp() == s0
    monkeypatch.setattr(build_ext, "NVCC_FLAGS", flags + ["-DX=1"])
    assert build_ext.code_stamp() != s0


def test_kernel_bytes_per_launch_of_a_split_call():
    """A retrieval call split into sub-batches launches the tile and dense
    kernels once per sub-batch: each launch moves its share of the batch's
    algorithmic bytes.  The sort's passes each move all tokens."""
    ctx = {"tile_bytes": 1000, "dense_bytes": 300, "n_tokens": 10, "nnz": 7}
    assert bench.kernel_bytes("k_tile_staged", ctx) == 1000
    assert bench.kernel_bytes("k_tile_staged", ctx, 2.0) == 500
    assert bench.kernel_bytes("k_dense_topk", ctx, 3.0) == 100
    assert bench.kernel_bytes("k_radix_downsweep", ctx, 3.0) == 160
    assert bench.kernel_bytes("k_score", ctx, 1.0) == 140
    assert bench.kernel_bytes("k_merge", ctx) is None

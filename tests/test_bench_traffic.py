"""bench.py's roofline `traffic`: read from a profile's "key: value" lines only
for the sources, workload and plan the counters were taken on."""
import bench


def _write(tmp_path, **kv):
    p = tmp_path / "k_traffic.md"
    body = "# k — DRAM traffic\n\nCommand: ncu ... (a prose line with a colon)\n\n"
    body += "".join(f"{k}: {v}\n" for k, v in kv.items())
    p.write_text(body)
    return str(p)


def test_plan_key_order():
    plan = {"dense_max_postings": 4096, "block_threads": 192, "tile_docs": 10240,
            "accumulator": 1}
    assert bench.plan_key(plan) == "1,10240,192,4096"


def test_matching_stamp_workload_and_plan(tmp_path):
    p = _write(tmp_path, build_stamp="abc", workload="zipf-1m", plan="1,10240,192,4096",
               traffic_bytes_per_launch=300100000)
    assert bench.read_traffic(p, "abc", "zipf-1m", "1,10240,192,4096") == 300100000


def test_any_mismatch_gives_none(tmp_path):
    p = _write(tmp_path, build_stamp="abc", workload="zipf-1m", plan="1,10240,192,4096",
               traffic_bytes_per_launch=300100000)
    assert bench.read_traffic(p, "abd", "zipf-1m", "1,10240,192,4096") is None
    assert bench.read_traffic(p, "abc", "tiny-2k", "1,10240,192,4096") is None
    assert bench.read_traffic(p, "abc", "zipf-1m", "1,10240,192,2048") is None


def test_file_without_a_plan_holds_for_any_plan(tmp_path):
    p = _write(tmp_path, build_stamp="abc", workload="zipf-1m", traffic_bytes_per_launch=7)
    assert bench.read_traffic(p, "abc", "zipf-1m", "2,7168,256,0") == 7


def test_missing_or_malformed_gives_none(tmp_path):
    assert bench.read_traffic(str(tmp_path / "absent.md"), "abc", "zipf-1m", "x") is None
    p = _write(tmp_path, build_stamp="abc", workload="zipf-1m", traffic_bytes_per_launch="n/a")
    assert bench.read_traffic(p, "abc", "zipf-1m", "x") is None


def test_committed_profile_parses():
    # the committed file names a stamp, the bench workload and a plan
    import os
    path = os.path.join(bench.ROOT, "profiles", "k_tile_staged_zipf1m_traffic.md")
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, _, v = line.partition(":")
            kv[k.strip()] = v.strip()
    assert kv["workload"] == "zipf-1m" and len(kv["build_stamp"]) == 64
    assert bench.read_traffic(path, kv["build_stamp"], "zipf-1m", kv["plan"]) == \
        int(kv["traffic_bytes_per_launch"])

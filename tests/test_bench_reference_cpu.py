"""bench.py --impl reference (the oracle timed on the host cores): one JSON
line from rank 0 with the keys the measurement contract names; under a
multi-rank launch the other ranks exit 0 without work."""
import json
import os
import subprocess
import sys

import bench


def _run(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    cmd = [sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
           "--workload", "tiny", "--steps", "2", "--warmup", "1", "--ref-sample-queries", "4"]
    return subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=300,
                          cwd=bench.ROOT)


def test_rank0_prints_the_reference_line():
    r = _run(0, 2)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "queries/s @k=10" and d["unit"] == "queries/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["config"]["workload"] == "tiny-2k"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    # the same config dict the GPU arm prints (bench_config), so the two lines compare
    import argparse
    from paper_2407_03618_gb300 import synth
    args = argparse.Namespace(variant="lucene", k=10)
    w = synth.WORKLOADS["tiny"]
    assert d["config"] == json.loads(json.dumps(bench.bench_config(args, w, w.n_queries, 2)))
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_other_ranks_exit_without_work():
    r = _run(1, 2)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]

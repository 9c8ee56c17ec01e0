"""The benchmark's JSON contract, checked on the CPU: the reference arm (the
FP64 oracle timed on the host cores) prints one JSON line with the keys a
driver reads, and the DRAM traffic figure of the dominant kernel is reported
only for the configuration and kernel sources it was measured on."""
import argparse
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "pairs matched/s" and d["unit"] == "pairs/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "grid5000"


def _args(**kw):
    a = dict(grid=None, workload="grid5000", rerank="bf16", K=8)
    a.update(kw)
    return argparse.Namespace(**a)


def test_traffic_is_reported_only_where_it_was_measured():
    t = bench.KMATCH_TRAFFIC
    same_sources = bench.kmatch_sources_sha256() == t["sources_sha256"] and t["bytes_per_pair"] is not None
    # after a change of the kernel's sources the recorded figure no longer applies
    got = bench.kmatch_traffic(_args(), 4500.0)
    assert got == (t["bytes_per_pair"] * 4500.0 if same_sources else None)
    for kw in (dict(workload="grid500"), dict(rerank="fp8"), dict(K=16)):
        assert bench.kmatch_traffic(_args(**kw), 4500.0) is None, kw


def test_oracle_sample_covers_its_share_and_the_pairs_among_its_images():
    import numpy as np
    import synth
    wl = synth.grid500(gx=10, gy=8)
    sel, imgs, elig = bench.pick_sample(wl.pairs, 0.02, 50)
    assert len(sel) == max(50, int(np.ceil(0.02 * len(wl.pairs)))) and len(set(sel.tolist())) == len(sel)
    assert set(sel.tolist()) <= set(elig.tolist())
    assert set(np.unique(wl.pairs[sel]).tolist()) == set(imgs.tolist())
    both = [k for k, (i, j) in enumerate(wl.pairs) if i in imgs and j in imgs]
    assert both == elig.tolist()
    # the same seed gives the same sample; all pairs when the share covers them
    assert np.array_equal(bench.pick_sample(wl.pairs, 0.02, 50)[0], sel)
    assert len(bench.pick_sample(wl.pairs, 1.0, 1)[0]) == len(wl.pairs)

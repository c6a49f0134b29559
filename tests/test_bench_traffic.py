"""bench.profiled_traffic: the DRAM traffic of a roofline family is taken from a committed ncu summary only
when the summary covers the same family, workload and (for the batch) schedule, and the kernel sources
hashed in it are unchanged. Both forms of a summary (bytes per launch over a step, or the DRAM /
algorithmic ratio of one captured launch) are checked on synthetic summaries; the committed summaries are
checked to name existing sources and to match them."""
import glob
import hashlib
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _summary(tmp, name, fields, sources):
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(tmp, rel), "rb") as f:
            h.update(f.read())
    lines = ["# synthetic summary", ""] + ["%s: %s" % kv for kv in fields.items()]
    lines += ["traffic_sources: " + " ".join(sources), "traffic_sources_sha256: " + h.hexdigest(), ""]
    with open(os.path.join(tmp, "profiles", name), "w") as f:
        f.write("\n".join(lines))


@pytest.fixture
def tree(tmp_path, monkeypatch):
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / "src")
    (tmp_path / "src" / "a.cuh").write_text("kernel a\n")
    (tmp_path / "src" / "b.cuh").write_text("kernel b\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_bytes_per_launch_form(tree):
    _summary(str(tree), "k_a_1m.md", {"traffic_bytes_per_launch": "123456", "traffic_kernel": "refine"},
             ["src/a.cuh", "src/b.cuh"])
    b, src, how = bench.profiled_traffic("refine", "1m")
    assert b == 123456.0 and src == os.path.join("profiles", "k_a_1m.md") and "every launch" in how
    assert bench.profiled_traffic("refine", "16m") is None      # another workload
    assert bench.profiled_traffic("contract_merge", "1m") is None  # another family


def test_ratio_form_scales_the_run(tree):
    _summary(str(tree), "k_b_16m.md", {"traffic_ratio": "1.25", "traffic_workload": "16m",
                                       "traffic_kernel": "contract_merge"}, ["src/a.cuh"])
    b, _, how = bench.profiled_traffic("contract_merge", "16m", 800.0)
    assert b == pytest.approx(1000.0) and "1.25" in how
    assert bench.profiled_traffic("contract_merge", "16m", None) is None  # nothing to scale


def test_schedule_must_match(tree):
    _summary(str(tree), "k_c_batch.md", {"traffic_ratio": "1.1", "traffic_workload": "batch4096",
                                         "traffic_schedule": "s1", "traffic_kernel": "batch"}, ["src/b.cuh"])
    assert bench.profiled_traffic("batch", "batch4096", 100.0, "s1")[0] == pytest.approx(110.0)
    assert bench.profiled_traffic("batch", "batch4096", 100.0, "s2") is None


def test_changed_source_disables_the_summary(tree):
    _summary(str(tree), "k_a_1m.md", {"traffic_bytes_per_launch": "7", "traffic_kernel": "refine"}, ["src/a.cuh"])
    assert bench.profiled_traffic("refine", "1m") is not None
    (tree / "src" / "a.cuh").write_text("kernel a, changed\n")
    assert bench.profiled_traffic("refine", "1m") is None


def test_committed_summaries_name_existing_sources_and_match_them():
    found = 0
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        kv = {}
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_"):
                    k, _, v = line.partition(":")
                    kv[k.strip()] = v.strip()
        if not kv:
            continue
        found += 1
        assert kv.get("traffic_kernel"), path
        assert ("traffic_bytes_per_launch" in kv) != ("traffic_ratio" in kv), path
        assert re.fullmatch(r"[0-9a-f]{64}", kv.get("traffic_sources_sha256", "")), path
        h = hashlib.sha256()
        for rel in kv["traffic_sources"].split():
            assert os.path.isfile(os.path.join(ROOT, rel)), (path, rel)
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        assert h.hexdigest() == kv["traffic_sources_sha256"], "%s: sources changed since the capture" % path
    assert found >= 3

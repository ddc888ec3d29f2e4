"""Host-side pieces of bench.py (no GPU): the reference arm's JSON line and
the comment-insensitive source hash that guards the stored DRAM counters."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_strip_comments_keeps_code_and_literals():
    src = ('a = "http://x" /* c1 */ + b; // tail\n'
           "char q = '/'; int z = 1; /* multi\nline */ w = \"\\\"//\"; // x\n"
           "s = \"/* not a comment */\";")
    out = bench._strip_comments(src)
    assert out == ('a = "http://x" + b; char q = \'/\'; int z = 1; w = "\\"//"; '
                   's = "/* not a comment */";')


def test_strip_comments_ignores_comment_and_spacing_edits_only():
    a = "int f(int x) {  // one\n  return x + 1; /* two */\n}\n"
    b = "int f(int x) {\n  // other words\n  return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench._strip_comments(a) == bench._strip_comments(b)
    assert bench._strip_comments(a) != bench._strip_comments(c)


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` times the oracle on the host and prints the
    contract's line with impl, cpu_baseline and e2e."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "20000",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "strings/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_scatter_bytes_follow_the_step_layout():
    """The scatter's algorithmic bytes are the redistribution's own: a u16
    bucket id read, a u32 index and a u64 key read and written (26 bytes per
    string); the offsets this implementation carries beside them are
    reported apart, never inside the roofline's bytes."""
    assert bench.BYTES_PER_UNIT["scatter"] == 26
    assert bench.CARRIED_BYTES_PER_UNIT["scatter"] == 16
    assert bench.BYTES_PER_UNIT["classify"] == 10
    assert bench.BYTES_PER_UNIT["merge_round"] == 16


def test_dram_traffic_needs_matching_sources_and_workload(tmp_path, monkeypatch):
    """roofline.traffic scales a small-case capture's bytes per unit to a full
    launch only while the sources hash to the capture's and the workload kind
    matches; otherwise it is null."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    tj = {"source_hash": bench._source_hash(),
          "kernels": {"url_like": {"scatter": {"workload_kind": "url_like", "dram_bytes_per_unit": 50.0}}}}
    (prof / "traffic.json").write_text(json.dumps(tj))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_source_hash", lambda: tj["source_hash"])
    assert bench.dram_traffic("scatter", "url_like", 1000) == 50000.0
    assert bench.dram_traffic("scatter", "no_lcp", 1000) is None
    assert bench.dram_traffic("classify", "url_like", 1000) is None
    monkeypatch.setattr(bench, "_source_hash", lambda: "other")
    assert bench.dram_traffic("scatter", "url_like", 1000) is None


def test_committed_traffic_file_has_every_workload_kind(monkeypatch):
    """profiles/traffic.json holds DRAM bytes per unit for every workload kind
    the bench can run, in the layout dram_traffic reads (checked as if the
    sources still hashed to the capture's)."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        tj = json.load(f)
    monkeypatch.setattr(bench, "_source_hash", lambda: tj["source_hash"])
    for kind in bench.WORKLOADS:
        assert bench.dram_traffic("scatter", kind, 1000) is not None, kind

"""The committed ncu traffic record (CPU): every entry names a benchmark
workload, sources and a summary that exist, and a positive byte count; the
bench reports an entry only while the hash of its sources matches."""
import json
import os

from paper_1801_10187_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_entries():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    assert rec
    for key, ent in rec.items():
        kernel, workload = key.split("/", 1)
        assert kernel.startswith("k_"), key
        assert workload in inputs.WORKLOADS, key
        for src in ent["sources"]:
            assert os.path.exists(os.path.join(ROOT, src)), (key, src)
        assert os.path.exists(os.path.join(ROOT, ent["summary"])), key
        assert ent["dram_bytes_per_launch"] > 0
        assert ent.get("scale_to_workload", 1.0) >= 1.0
        assert len(ent["sources_sha256_16"]) == 16
        assert "ncu" in ent["from"] or "scaled" in ent["from"]


def test_profile_summaries_give_their_commands():
    pdir = os.path.join(ROOT, "profiles")
    for name in os.listdir(pdir):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(pdir, name)) as f:
            text = f.read()
        assert "ncu " in text and "--clock-control none" in text, name
        assert "python bench.py" in text, name


def test_sources_hash_follows_code_not_comments(tmp_path, monkeypatch):
    """The record's hash changes with the code and not with comments or blank
    lines (the counters depend on the compiled code only)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "k.cu"
    src.write_text("// a kernel\n__global__ void k(int* x) {\n  x[0] = 1;  /* one */\n}\n")
    h0 = bench.sources_hash(["k.cu"])
    src.write_text("/* another\n   comment */\n__global__ void k(int* x) {\n\n  x[0] = 1;  // one\n}\n")
    assert bench.sources_hash(["k.cu"]) == h0
    src.write_text("__global__ void k(int* x) {\n  x[0] = 2;\n}\n")
    assert bench.sources_hash(["k.cu"]) != h0


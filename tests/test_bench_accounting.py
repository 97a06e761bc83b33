"""The bench line's roofline bookkeeping (host code, no GPU): the shift tests' operation counts
and the committed DRAM traffic record, which counts only while it was taken on the current
kernel sources."""
import importlib.util
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_shift_test_ops():
    b = load_bench()
    n = 1000
    # every test settled by the binary32 pass: one binary64 subtraction and 16 binary32 ops per term
    o64, o32 = b.shift_test_ops(n, {"shift_binary32": n - 1})
    assert o64 == (n - 1) * (n - 1) * b.SHIFT32_B64_OPS_PER_TERM
    assert o32 == (n - 1) * (n - 1) * b.SHIFT32_OPS_PER_TERM
    # none settled: the binary32 pass and then the 5-op binary64 pass for every test
    o64, o32 = b.shift_test_ops(n, {"shift_binary32": 0})
    assert o64 == (n - 1) * (n - 1) * (b.OPS_PER_TERM + b.SHIFT32_B64_OPS_PER_TERM)
    assert o32 == (n - 1) * (n - 1) * b.SHIFT32_OPS_PER_TERM
    # with the screens off only the binary64 pass runs
    o64, o32 = b.shift_test_ops(n, {"shift_binary32": 0}, screen=False)
    assert o64 == (n - 1) * (n - 1) * b.OPS_PER_TERM and o32 == 0


def test_committed_traffic_follows_the_sources(tmp_path, monkeypatch):
    b = load_bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_solve_traffic.json")))
    # the committed record was taken on the committed kernel sources
    assert rec["source_hash"] == b.kernel_source_hash(rec["source_files"])
    n = rec["bisection"]["n"]
    assert b.committed_traffic(n, 0) == rec["bisection"]["dram_bytes_per_launch"]
    assert b.committed_traffic(n, 1) == rec["accelerated"]["dram_bytes_per_launch"]
    assert b.committed_traffic(n + 1, 0) is None           # another order: no figure
    # a record whose hash does not match the sources gives no figure
    stale = dict(rec, source_hash="0" * 16)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_solve_traffic.json").write_text(json.dumps(stale))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "kernel_source_hash", lambda files: rec["source_hash"])
    assert b.committed_traffic(n, 0) is None

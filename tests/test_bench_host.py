"""Host-side logic of bench.py that needs no GPU: the kernel-source hash
that decides whether a committed ncu traffic figure still describes the
code (comments and whitespace do not count, code does)."""
import bench


def test_code_only_drops_comments_and_whitespace():
    a = "int f(int x) {  // doubles x\n    return 2 * x; /* no\n overflow check */\n}\n"
    b = "int f(int x) {\n  return 2 * x;\n}"
    assert bench._code_only(a) == bench._code_only(b)


def test_code_only_keeps_code_changes():
    a = "int f(int x) { return 2 * x; }"
    b = "int f(int x) { return 3 * x; }"
    assert bench._code_only(a) != bench._code_only(b)


def test_profiled_traffic_reads_matching_summary(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sssp_source_hash", lambda: "abc123")
    (prof / "sssp_w.md").write_text("sssp_source_hash: abc123\ntraffic_bytes_per_launch: 42\n")
    assert bench.profiled_traffic("w") == 42
    (prof / "sssp_w.md").write_text("sssp_source_hash: def456\ntraffic_bytes_per_launch: 42\n")
    assert bench.profiled_traffic("w") is None          # captured on other code
    assert bench.profiled_traffic("absent") is None

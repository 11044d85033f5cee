"""Host-side logic of bench.py that decides what the bench line may claim."""
import bench


def test_code_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    """The recorded DRAM traffic stays valid across comment edits of the flooding
    sources and becomes stale (null in the bench line) on any code edit."""
    src = "// header\nint f(int x) {  /* block\n comment */ return x + 1; }  // tail\n"
    (tmp_path / "a.cu").write_text(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.sources_hash(["a.cu"])
    (tmp_path / "a.cu").write_text("// another header\n\nint f(int x) { return x + 1; }\n/* more */\n")
    assert bench.sources_hash(["a.cu"]) == h0
    (tmp_path / "a.cu").write_text("int f(int x) { return x + 2; }\n")
    assert bench.sources_hash(["a.cu"]) != h0
    assert bench.code_text(src) == "int f(int x) { return x + 1; }"


def test_recorded_traffic_matches_a_known_kernel_or_is_dropped():
    """The bench reports the recorded JFA traffic only for the code it was measured on."""
    rec = bench.JFA_ROOM_TRAFFIC
    assert len(rec["sources_sha256_16"]) == 16
    assert 0 < rec["bytes_per_frame"] < 4 * 2.56e9
    current = bench.sources_hash(bench.JFA_SOURCES)
    assert isinstance(current, str) and len(current) == 16

"""The DRAM traffic that bench.py reports beside its roofline comes from one
ncu capture and holds only for the kernel code it was captured from: the
record is keyed by a digest of the CUDA sources with comments and blank
lines removed."""
import bench


def test_code_only_drops_comments_and_blank_lines_only():
    src = (b"// header\n"
           b"int a = 1;  // trailing\n"
           b"\n"
           b"/* block\n   comment */ int b = 2;\n"
           b"x = y / z;\n")
    assert bench._code_only(src) == b"int a = 1;\n int b = 2;\nx = y / z;"


def test_a_code_change_changes_the_key_and_a_comment_does_not():
    src = b"constexpr int kTile = 8;   // rows per block\n"
    assert bench._code_only(src) == bench._code_only(b"constexpr int kTile = 8;   // rows of a block\n\n")
    assert bench._code_only(src) != bench._code_only(b"constexpr int kTile = 4;   // rows per block\n")


def test_recorded_traffic_only_for_the_captured_sources(monkeypatch):
    monkeypatch.setattr(bench, "_TRAFFIC", {"k_demo": 123.0})
    monkeypatch.setattr(bench, "_TRAFFIC_SRC", bench._csrc_digest())
    assert bench._recorded_traffic("k_demo") == 123.0
    assert bench._recorded_traffic("k_other") is None
    monkeypatch.setattr(bench, "_TRAFFIC_SRC", "0" * 64)
    assert bench._recorded_traffic("k_demo") is None

"""Host logic of bench.py that needs no GPU: replica aggregation is covered by
test_multirank_cpu.py; here, the roofline traffic is taken from the committed ncu summary only
while the kernel code it was captured from is unchanged."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench as b
    finally:
        sys.argv = argv
    return b


def test_code_hash_ignores_comments_and_spacing(bench):
    a = "int f(int x) {  // twice\n    return 2 * x; /* no overflow here */\n}\n"
    b = "int f(int x) {\n\treturn 2*x;\n}  // a different comment\n"
    c = "int f(int x) {\n    return 3 * x;\n}\n"
    assert bench.code_sha1(a) == bench.code_sha1(b)
    assert bench.code_sha1(a) != bench.code_sha1(c)


def test_traffic_follows_the_recorded_code_hash(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k(float* a) { a[0] = 1.f; }\n")
    md = tmp_path / "summary.md"
    md.write_text(f"code_sha1: {bench.code_sha1(src.read_text())}\ntraffic_bytes_per_step: 12345\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.TRAFFIC_SOURCES, ("particles", 2), ("summary.md", "k.cu"))
    assert bench.captured_traffic("particles", 2) == 12345.0
    src.write_text("// edited comment\n__global__ void k(float* a) { a[0] = 1.f; }\n")
    assert bench.captured_traffic("particles", 2) == 12345.0
    src.write_text("__global__ void k(float* a) { a[0] = 2.f; }\n")
    assert bench.captured_traffic("particles", 2) is None
    assert bench.captured_traffic("fields", 2) is None


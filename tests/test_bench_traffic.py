"""Host logic of bench.py's stored ncu traffic: a capture applies only while
the kernel's code (not its comments or layout), the batch and the mesh match."""
import json

import bench


def test_normalize_source_ignores_comments_and_layout_only():
    a = 'int f(int x) {\n  // doubled\n  return 2 * x; /* plain */\n}\n'
    b = 'int f(int x)\n{\n    /* a longer\n       comment */ return 2 * x;\n}'
    c = 'int f(int x) { return 3 * x; }'
    assert bench.normalize_source(a) == bench.normalize_source(b)
    assert bench.normalize_source(a) != bench.normalize_source(c)


def test_normalize_source_keeps_string_literals():
    s = 'asm volatile("mov.u64 %0, %%globaltimer; // not a comment" : "=l"(t)); char q = \'/\'; // gone'
    out = bench.normalize_source(s)
    assert "// not a comment" in out and "gone" not in out and "'/'" in out


def test_stored_traffic_matches_hash_batch_and_mesh(tmp_path):
    rec = {"kernel": "k_fim", "kernel_hash": bench.kernel_hash("k_fim"), "batch": 16, "n": 72,
           "bytes_per_launch": 123456789}
    path = tmp_path / "t.txt"
    path.write_text(json.dumps(rec))
    assert bench.stored_traffic(16, 72, str(path)) == 123456789
    assert bench.stored_traffic(8, 72, str(path)) is None
    assert bench.stored_traffic(16, 40, str(path)) is None
    rec["kernel_hash"] = "0" * 12
    path.write_text(json.dumps(rec))
    assert bench.stored_traffic(16, 72, str(path)) is None
    assert bench.stored_traffic(16, 72, str(tmp_path / "missing.txt")) is None


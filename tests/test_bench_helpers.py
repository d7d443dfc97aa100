"""Host helpers of bench.py (no GPU): the comment-free source hash that ties
a stored ncu capture to the kernel code, and the capture's scaling."""
import json
import os

import bench


def test_strip_comments_keeps_code_and_literals():
    src = ('int a = 1; // note\n/* block\n   comment */ const char *s = "// kept /* kept */";\n'
           "char c = '\"';\n\n   x /= 2; /**/ y = a / b;\n")
    out = bench.strip_comments(src)
    assert out == ('int a = 1;\n const char *s = "// kept /* kept */";\nchar c = \'"\';\n   x /= 2;  y = a / b;')
    # editing or adding comments leaves the stripped text unchanged
    edited = src.replace("// note", "// another note").replace("\n\n", "\n// a new comment line\n\n")
    assert bench.strip_comments(edited) == out
    # a code change does not
    assert bench.strip_comments(src.replace("x /= 2", "x /= 3")) != out


def test_stored_traffic_is_scaled_or_withheld():
    """The committed capture's DRAM bytes are scaled by the algorithmic bytes
    of a launch while it belongs to the current kernel code, and withheld
    (None) once the code has changed."""
    with open(os.path.join(bench.ROOT, "profiles", "k_liquid_traffic.json")) as fh:
        rec = json.load(fh)
    r = rec["f32"]
    t = bench.stored_traffic("f32", 2.0 * r["algorithmic_bytes"])
    if rec["kernel_source_sha256"] == bench.kernel_source_hash():
        assert abs(t - 2.0 * r["dram_bytes"]) <= 1e-9 * t
    else:
        assert t is None
    assert bench.stored_traffic("bf16", 1.0) is None  # no capture of that storage


def test_stored_fp64_ops_follow_the_capture():
    """The double path's operations per liquid cell come from the committed
    capture while it belongs to the current kernel code."""
    with open(os.path.join(bench.ROOT, "profiles", "k_liquid_traffic.json")) as fh:
        rec = json.load(fh)
    ops = bench.stored_fp64_ops()
    if rec["kernel_source_sha256"] == bench.kernel_source_hash():
        r = rec["f64"]
        assert ops == r["dp_ops_per_liquid_cell"]
        assert abs(r["dp_ops"] / r["liquid_cells"] - ops) < 0.01
    else:
        assert ops is None

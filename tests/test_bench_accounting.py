"""The benchmark's byte accounting (host arithmetic, no GPU): the
algorithmic bytes of the staging + clip launch and of the whole path per
Jungfrau-4M frame, against the terms written out by hand."""
import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(HERE, "..", "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


N, NNZ, B, F = 2164 * 2068, 5_996_800, 1000, 512


def test_clip_launch_bytes():
    b = _bench()
    raw = 2 * N * F                        # every raw word once
    cal = 2 * 3 * 4 * N                    # pedestal and gain, three levels, float32
    mat = 4 * NNZ + 4 * (B + 1)            # packed entries and row pointers
    outs = 4 * 4 * B * F                   # mean, sigma, count, threshold
    assert b.algorithmic_bytes_clip(F, N, 0, NNZ, B) == raw + cal + mat + outs


def test_whole_path_bytes_per_frame():
    b = _bench()
    kept, peaks = 5000.0, 120.0
    got = b.algorithmic_bytes_path(F, N, NNZ, B, kept, peaks)
    want = 2 * N + (24 * N + 4 * NNZ + 4 * (B + 1) + 4 * N) / F + 12 * B + 8 * kept + 24 * peaks + 8
    assert abs(got - want) < 1e-6
    # about 9.2-9.4 MB per frame at 512 frames: the raw frame dominates
    assert 9.2e6 < got < 9.4e6


def test_traffic_record_follows_the_code_not_the_comments():
    b = _bench()
    code = 'int f(int x) { // twice\n  /* the "input" */ return x * 2; }\nconst char* s = "// kept /* too */";\n'
    assert b.strip_comments(code) == 'int f(int x) { return x * 2; } const char* s = "// kept /* too */";'
    # a comment or a blank line changes nothing, an operator does
    assert b.strip_comments(code.replace("// twice", "// three times\n\n")) == b.strip_comments(code)
    assert b.strip_comments(code.replace("x * 2", "x * 3")) != b.strip_comments(code)
    assert b.strip_comments("a = '\\'' ; /* c */ b") == "a = '\\'' ; b"
    # the recorded capture scales with the frames while its fingerprint is the code's
    import json
    with open(os.path.join(HERE, "..", "profiles", "roofline_traffic.json")) as f:
        rec = json.load(f)
    got = b.measured_traffic(512)
    if rec["sources_sha256"] == b.source_fingerprint():
        assert got == int(rec["bytes_per_frame"] * 512)
    else:
        assert got is None

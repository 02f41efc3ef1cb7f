"""Host-side pieces of the benchmark that need no GPU: the code digest that keys the committed DRAM
traffic figures to the kernel sources."""
import importlib.util
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


SRC = """// header comment
__global__ void k(float* a) {  // trailing comment
    /* block
       comment */ a[0] = 1.0f;
}
"""


def test_code_digest_ignores_comments_and_blank_lines():
    b = _bench()
    base = b.code_digest([SRC])
    assert b.code_digest([SRC.replace("// header comment", "// reworded header")]) == base
    assert b.code_digest([SRC + "\n\n// a note\n/* another */\n"]) == base
    assert b.code_digest([SRC.replace("trailing comment", "other words")]) == base


def test_code_digest_tracks_code():
    b = _bench()
    base = b.code_digest([SRC])
    assert b.code_digest([SRC.replace("1.0f", "2.0f")]) != base
    assert b.code_digest([SRC + "\nint x;\n"]) != base
    assert b.code_digest([SRC, ""]) == base  # an empty file adds no code
    assert b.code_digest(["int a;", "int b;"]) != b.code_digest(["int b;", "int a;"])


def test_traffic_record_names_its_kernel():
    with open(os.path.join(ROOT, "profiles", "g2p2g_traffic.json")) as f:
        rec = json.load(f)
    assert rec["kernel"] == "k_g2p2g" and len(rec["kernel_source_hash"]) == 16
    assert rec["dram_bytes_per_launch_full_size"] == rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]


def test_flag_names_match_the_header():
    b = _bench()
    from paper_2302_04659_gb300 import _native as mpm
    assert b.flag_names(0) == []
    assert b.flag_names(mpm.MPM_FLAG_CLAMPED)[0].startswith("clamped")
    every = (mpm.MPM_FLAG_CLAMPED | mpm.MPM_FLAG_NONFINITE | mpm.MPM_FLAG_SV_CLAMPED | mpm.MPM_FLAG_FAR_MOVE
             | mpm.MPM_FLAG_INTERNAL)
    assert len(b.flag_names(every)) == 5


def test_oracle_replicas_on_all_cores(monkeypatch):
    """The CPU baseline runs the oracle as independent spawned replicas, one per core; its value is the
    replicas' particle-substeps over the slowest replica's time."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as b  # importable by name, so that spawned replicas can unpickle its functions
    monkeypatch.setattr(b.os, "cpu_count", lambda: 2)
    value, cores, secs = b.oracle_on_all_cores(1000, 4000, 300, 1, 2)
    assert cores == 2 and secs > 0.0
    assert abs(value - 2 * 300 * 2 / secs) <= 1e-9 * value


def test_every_bench_section_is_selectable():
    """Each profiling section of the bench (--only) is offered on its command line."""
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                         timeout=300).stdout
    for section in ("batched", "serving", "surrogate", "contact", "render", "conv", "train"):
        assert section in out, section

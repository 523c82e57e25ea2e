"""Host-side helpers of bench.py: the recorded-traffic check keys on the kernels'
code, not on their comments (a changed kernel reports no traffic until re-measured)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_source_hash_ignores_comments_and_whitespace_only():
    files = ["k_pass.cu", "mpsm_internal.cuh"]
    d = os.path.join(ROOT, "paper_1207_0145_gb300", "csrc")
    texts = {fn: open(os.path.join(d, fn)).read() for fn in files}
    base = bench.kernel_source_hash(files, texts)
    assert bench.kernel_source_hash(files) == base
    commented = dict(texts)
    commented["k_pass.cu"] = "// a new comment\n/* and a block\n comment */\n" + texts["k_pass.cu"].replace("\n", "\n  ")
    assert bench.kernel_source_hash(files, commented) == base
    changed = dict(texts)
    changed["k_pass.cu"] = texts["k_pass.cu"].replace("RX_TILE = 5120", "RX_TILE = 4096", 1)
    assert changed["k_pass.cu"] != texts["k_pass.cu"]
    assert bench.kernel_source_hash(files, changed) != base

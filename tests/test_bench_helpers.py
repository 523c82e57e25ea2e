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


def test_step_traffic_record_is_read_only_for_unchanged_sources(tmp_path, monkeypatch):
    files = ["k_pass.cu", "k_split.cu"]
    h = bench.kernel_source_hash(files)
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = prof / "step_traffic_cfgx.txt"
    rec.write_text(f"# note\nsources: {' '.join(files)}\nsource_hash: {h}\ndram_bytes_per_tuple: 110.5\n"
                   "measured_on: plain-25M-100M\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # kernel_source_hash reads csrc under ROOT: point it at the real sources
    real = os.path.join(ROOT, "paper_1207_0145_gb300")
    os.symlink(real, tmp_path / "paper_1207_0145_gb300")
    assert bench.traffic_per_tuple("cfgx") == (110.5, "plain-25M-100M")
    rec.write_text(f"sources: {' '.join(files)}\nsource_hash: 0000\ndram_bytes_per_tuple: 110.5\n")
    assert bench.traffic_per_tuple("cfgx") is None
    assert bench.traffic_per_tuple("missing") is None


def test_host_numa_of_reads_numa_maps():
    import numpy as np

    a = np.ones(1 << 20, dtype=np.uint8)
    got = bench.host_numa_of(a.ctypes.data)
    assert got is None or all(p.startswith("N") for p in got.split())


def test_host_huge_bytes_of_reads_smaps():
    import numpy as np

    a = np.ones(1 << 20, dtype=np.uint8)
    v = bench.host_huge_bytes_of(a.ctypes.data, a.nbytes)
    assert v is None or (isinstance(v, int) and 0 <= v <= (4 << 30))

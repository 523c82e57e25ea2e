"""The C ABI library loads without a GPU, exports every function include/mpsm.h
declares, and the binding's ctypes structures match the header's layout."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1207_0145_gb300 import mpsm as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpsm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpsm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("mpsm_plan_create", "mpsm_join", "mpsm_plan_destroy", "mpsm_join_batch", "mpsm_sort_runs",
                 "mpsm_splitters", "mpsm_scatter", "mpsm_sort_partitions", "mpsm_search", "mpsm_merge_join"):
        assert want in names


def test_library_exports_every_declared_function():
    lib = ctypes.CDLL(M.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", M.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mpsm_\w+)", out))
    assert set(declared_functions()) <= exported


def test_strerror_and_defaults_without_gpu():
    assert M.strerror(0) == "ok"
    assert "capacity" in M.strerror(M.ERR_CAPACITY) or "small" in M.strerror(M.ERR_CAPACITY)
    o = M.make_options()
    assert o.splitter_mode == M.SPLIT_HIST and o.search_mode == M.SEARCH_BINARY and o.runs_r == 0


LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "mpsm.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("mpsm_options_t %zu\n", sizeof(mpsm_options_t));
  printf("mpsm_stats_t %zu\n", sizeof(mpsm_stats_t));
  printf("mpsm_view_t %zu\n", sizeof(mpsm_view_t));
  printf("mpsm_job_t %zu\n", sizeof(mpsm_job_t));
  printf("mpsm_pairs_t %zu\n", sizeof(mpsm_pairs_t));
  F(mpsm_options_t, seed); F(mpsm_options_t, flags); F(mpsm_options_t, learn_steps);
  F(mpsm_options_t, run_len); F(mpsm_options_t, partition_side); F(mpsm_options_t, run_buckets);
  F(mpsm_options_t, reserved);
  printf("mpsm_rmi_info_t %zu\n", sizeof(mpsm_rmi_info_t));
  F(mpsm_stats_t, loss_s0); F(mpsm_stats_t, part_probes); F(mpsm_stats_t, search_err);
  F(mpsm_stats_t, s_kept); F(mpsm_stats_t, imbalance); F(mpsm_stats_t, tiles); F(mpsm_stats_t, segments_s);
  F(mpsm_stats_t, launches);
  printf("mpsm_kernel_time_t %zu\n", sizeof(mpsm_kernel_time_t));
  F(mpsm_view_t, key_min); F(mpsm_view_t, fine_s); F(mpsm_view_t, s_chunks); F(mpsm_view_t, windows);
  F(mpsm_view_t, join_tile); F(mpsm_view_t, s_kept); F(mpsm_view_t, segments); F(mpsm_view_t, n_segments);
  F(mpsm_view_t, window_stride); F(mpsm_view_t, seg_windows);
  printf("mpsm_segment_t %zu\n", sizeof(mpsm_segment_t));
  return 0;
}
"""


def test_ctypes_structs_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert int(got["mpsm_options_t"]) == ctypes.sizeof(M.Options)
    assert int(got["mpsm_stats_t"]) == ctypes.sizeof(M.Stats)
    assert int(got["mpsm_view_t"]) == ctypes.sizeof(M.View)
    assert int(got["mpsm_job_t"]) == ctypes.sizeof(M.JobDesc)
    assert int(got["mpsm_pairs_t"]) == ctypes.sizeof(M.Pairs)
    assert int(got["mpsm_kernel_time_t"]) == ctypes.sizeof(M.KernelTime)
    assert int(got["mpsm_rmi_info_t"]) == ctypes.sizeof(M.RmiInfo)
    assert int(got["mpsm_segment_t"]) == 40
    for key, val in got.items():
        if "." not in key:
            continue
        struct, member = key.split(".")
        cls = {"mpsm_options_t": M.Options, "mpsm_stats_t": M.Stats, "mpsm_view_t": M.View}[struct]
        assert getattr(cls, member).offset == int(val), key


def test_plan_create_without_gpu_fails_cleanly():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = M.lib().mpsm_plan_create(ctypes.byref(h), 1000, 1000, 1, None, None)
    assert rc in (M.ERR_CUDA, M.ERR_OOM)
    assert not h.value

"""mpsm_join_host with the partitioned side copied and joined in pieces.

Above 2^28 partitioned-side tuples the host-buffer join copies that side in
equal pieces (a quarter of the run side, between 2^26 and 2^27 tuples) and joins
each piece against the sorted runs while the next one is in flight.  The join
sums over pairs, so any split gives the same count and checksum; these cases
check that against the generator's closed form, with a split that leaves the
last piece a few tuples short, and skewed keys whose hot keys fall into every
piece.  The inputs sit in the library's own host buffers (mpsm_host_alloc); two
cases use torch's pinned memory and pageable memory instead.
"""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import Plan  # noqa: E402
from paper_1207_0145_gb300 import mpsm as M  # noqa: E402

PIECE = 1 << 27


def pinned_inputs(w):
    R = torch.empty((w.n_r, 2), dtype=torch.int64, device="cuda")
    S = torch.empty((w.n_s, 2), dtype=torch.int64, device="cuda")
    w.fill_r_device(R.data_ptr(), torch.cuda.current_stream().cuda_stream)
    w.fill_s_device(S.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    # the library's page-locked huge-page buffers: released when the test drops them,
    # not kept by the process's pinned-memory pool
    Rh = torch.from_numpy(M.host_tuples(w.n_r).view(np.int64))
    Rh.copy_(R)
    Sh = torch.from_numpy(M.host_tuples(w.n_s).view(np.int64))
    Sh.copy_(S)
    assert Rh.is_pinned() and Sh.is_pinned()
    return R, S, Rh, Sh


@pytest.mark.parametrize("w", [gen.plain((5 * PIECE) // 8, 5 * PIECE // 2 + 12345, seed=61),
                               gen.zipf(1 << 24, 2 * PIECE + 7, 0.9, seed=62)])
def test_host_join_in_pieces_matches_closed_form(w):
    want = oracle.closed_form(w)
    R, S, Rh, Sh = pinned_inputs(w)
    with Plan(w.n_r, w.n_s) as p:
        assert p.join_host(Rh, Sh) == want
        assert p.join_host(Rh, Sh) == want  # staging buffers and events reused
        assert p.join(R, S) == want         # the device-buffer join on the same plan
        assert p.device_errors() == 0


def test_host_join_in_pieces_reversed_roles():
    # the larger input partitioned in pieces while the smaller one is cut into runs
    w = gen.plain(2 * PIECE + 99, PIECE // 2, seed=63)
    want = oracle.closed_form(w)
    _, _, Rh, Sh = pinned_inputs(w)
    with Plan(w.n_r, w.n_s, partition_side=M.PART_R) as p:
        assert p.join_host(Rh, Sh) == want


@pytest.mark.parametrize("kind", ["torch_pinned", "pageable"])
def test_host_join_from_other_host_memory(kind):
    # buffers from torch's pinned pool and plain pageable numpy memory take the same path
    w = gen.plain(1 << 20, 3_000_017, seed=64)
    R, S = w.r_host(), w.s_host()
    if kind == "torch_pinned":
        Rh = torch.from_numpy(R.view(np.int64)).pin_memory()
        Sh = torch.from_numpy(S.view(np.int64)).pin_memory()
    else:
        Rh, Sh = R, S
    with Plan(w.n_r, w.n_s) as p:
        assert p.join_host(Rh, Sh) == oracle.closed_form(w)
        assert p.device_errors() == 0


def test_library_host_buffers_start_zeroed_and_pinned():
    h = M.host_tuples(1 << 20)
    assert h.shape == (1 << 20, 2) and not h.any()
    assert torch.from_numpy(h.view(np.int64)).is_pinned()


def test_host_alloc_rejects_bad_arguments():
    import ctypes

    out = ctypes.c_void_p()
    assert M.lib().mpsm_host_alloc(0, ctypes.byref(out)) == M.ERR_INVALID_ARG
    assert M.lib().mpsm_host_alloc(16, None) == M.ERR_INVALID_ARG
    assert M.lib().mpsm_host_free(None, 0) == M.OK

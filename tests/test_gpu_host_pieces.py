"""mpsm_join_host with the partitioned side copied and joined in pieces.

Above 2^28 partitioned-side tuples the host-buffer join copies that side in
equal pieces (a quarter of the run side, between 2^26 and 2^27 tuples) and joins
each piece against the sorted runs while the next one is in flight.  The join
sums over pairs, so any split gives the same count and checksum; these cases
check that against the generator's closed form, with a split that leaves the
last piece a few tuples short, and skewed keys whose hot keys fall into every
piece.
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
    Rh = torch.empty(R.shape, dtype=torch.int64, pin_memory=True)
    Sh = torch.empty(S.shape, dtype=torch.int64, pin_memory=True)
    Rh.copy_(R)
    Sh.copy_(S)
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

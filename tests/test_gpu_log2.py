"""The splitter kernel's Q16 logarithm against the oracle's, value by value.

Sec. 4.3 charges a partition of n tuples n log n for its sort; both sides
evaluate it as n * floor(2^16 log2 n) in integers, so they pick the same
splitters bit for bit.  The values include every n below 2^16, random n over
the whole 64-bit range, and the integers at the steps of the floor, where a
finite-precision method is most likely to slip.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle import boundary_n

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import mpsm as M  # noqa: E402

U64 = (1 << 64) - 1


def values():
    rng = np.random.default_rng(51)
    ns = list(range(0, 1 << 16))
    ns += [int(x) for x in rng.integers(2, U64, 20000, dtype=np.uint64, endpoint=True)]
    ns += [int(x) >> int(s) for x, s in zip(rng.integers(2, U64, 20000, dtype=np.uint64), rng.integers(0, 62, 20000))]
    for L in [int(x) for x in rng.integers(65536, 64 * 65536, 3000)]:
        n = boundary_n(L)
        ns += [m for m in (n - 1, n, n + 1) if m <= U64]
    return np.array(ns, dtype=np.uint64)


@pytest.mark.parametrize("wide", [False, True])
def test_kernel_log2_equals_oracle(wide):
    n = values()
    want = np.array([oracle.log2_q16(int(v)) for v in n.tolist()], dtype=np.uint64)
    dn = torch.from_numpy(n.view(np.int64)).cuda()
    out = torch.full_like(dn, -1)
    M.selftest_log2_q16(dn, out, wide=wide)
    got = out.cpu().numpy().view(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, [(int(n[i]), int(got[i]), int(want[i])) for i in bad[:5]]

"""The multithreaded CPU P-MPSM baseline (pmpsm_cpu/) against the oracle: every
workload shape, several thread counts, the degenerate cases."""
import numpy as np
import pytest

import gen
import oracle
import pmpsm_cpu


@pytest.mark.parametrize("w", [gen.plain(100_000, 400_000, seed=1), gen.zipf(50_000, 300_000, 0.9, seed=2),
                               gen.sparse(60_000, 90_000, seed=3), gen.negcorr(70_000, 280_000, seed=4),
                               gen.locskew(70_000, 210_000, seed=5)])
def test_pmpsm_matches_oracle(w):
    R, S = w.r_host(), w.s_host()
    want = oracle.join(R, S)
    for T in (1, 2, 7, 16):
        for B in (4, 10, 14):
            assert pmpsm_cpu.join(R, S, threads=T, fine_bits=B)[:2] == want


def test_pmpsm_degenerate_inputs():
    rng = np.random.default_rng(3)
    R = np.zeros((500, 2), dtype=np.uint64)
    S = np.zeros((700, 2), dtype=np.uint64)
    R[:, 0] = rng.integers(0, 4, 500, dtype=np.uint64)  # few distinct keys, many duplicates
    S[:, 0] = rng.integers(0, 6, 700, dtype=np.uint64)
    R[:, 1] = rng.integers(0, 2**64 - 1, 500, dtype=np.uint64)
    S[:, 1] = rng.integers(0, 2**64 - 1, 700, dtype=np.uint64)
    assert pmpsm_cpu.join(R, S, threads=8)[:2] == oracle.join(R, S)
    R[:, 0] = 2**64 - 1  # one key at the top of the domain
    S[::3, 0] = 2**64 - 1
    assert pmpsm_cpu.join(R, S, threads=4)[:2] == oracle.join(R, S)
    one = R[:1].copy()
    assert pmpsm_cpu.join(one, S, threads=16)[:2] == oracle.join(one, S)  # more threads than R tuples
    empty = np.zeros((0, 2), dtype=np.uint64)
    assert pmpsm_cpu.join(empty, S)[:2] == (0, 0)
    assert pmpsm_cpu.join(R, empty)[:2] == (0, 0)

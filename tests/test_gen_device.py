"""The device fill of the generator writes the same bytes as the host fill."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w", [gen.plain(70_000, 300_000, seed=1), gen.zipf(50_000, 200_000, 0.9, seed=2),
                               gen.sparse(60_000, 90_000, seed=3), gen.zipf(3, 1000, 0.8, seed=4),
                               gen.negcorr(70_001, 280_000, seed=5), gen.locskew(70_001, 200_000, seed=6)])
def test_device_generation_matches_host(w):
    R = torch.empty((w.n_r, 2), dtype=torch.int64, device="cuda")
    S = torch.empty((w.n_s, 2), dtype=torch.int64, device="cuda")
    w.fill_r_device(R.data_ptr())
    w.fill_s_device(S.data_ptr())
    torch.cuda.synchronize()
    assert (R.cpu().numpy().view(np.uint64) == w.r_host()).all()
    assert (S.cpu().numpy().view(np.uint64) == w.s_host()).all()

"""The library's device memory pool: scratch freed by a call stays reserved
for later calls, gs_trim_memory hands it back, and calls after a trim are
correct."""
import numpy as np
import pytest

from helpers import rel_err
from oracle import exhaustive as oracle_ex
from workloads import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    from paper_1206_6857_gb300 import build, gs as _gs
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _gs.load()
    return _gs


def test_pool_keeps_and_trims(gs):
    import torch
    q, _, w = synth.small_random(61, 20000, 3)
    h = np.array([0.01, 0.1])
    tq = torch.from_numpy(q).cuda()
    tw = torch.from_numpy(w).cuda()
    exact = oracle_ex.gauss_sum(q, q, w, h)
    W = float(w.astype(np.float64).sum())
    torch.cuda.synchronize()
    _, used0 = gs.gs_pool_bytes()        # earlier calls of this process may hold pool memory (trees)
    a = gs.gs_sum(tq, tq, tw, h, 1e-2).cpu().numpy()
    torch.cuda.synchronize()
    reserved, used = gs.gs_pool_bytes()
    assert used == used0                 # every scratch buffer of the call went back to the pool
    assert reserved > used               # ... and the pool kept it
    gs.gs_trim_memory(0)
    reserved2, used2 = gs.gs_pool_bytes()
    assert used2 == used0 and reserved2 < reserved
    b = gs.gs_sum(tq, tq, tw, h, 1e-2).cpu().numpy()
    assert np.allclose(a, b, rtol=1e-9, atol=0)
    assert rel_err(b, exact, W).max() <= 1e-2

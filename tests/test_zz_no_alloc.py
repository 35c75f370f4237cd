"""The allocation-free exhaustive entry point (scratch in a fixed device
array inside the library) agrees with gs_sum's exhaustive mode, on two
calls in a row with different inputs.  Collected last on purpose."""
import numpy as np
import pytest

from workloads import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def gs():
    import torch
    from paper_1206_6857_gb300 import build, gs as _gs
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _gs.load()
    return _gs


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_gs_sum_on_consecutive_calls(gs):
    cases = [synth.small_random(301, 20000, 3, m=3000), synth.small_random(302, 7777, 5)]
    hs = [np.array([0.01, 0.05, 0.3]), synth.log_bandwidths(1.0, 9, 1e-3, 1.0)]
    for (q, r, w), h in zip(cases, hs):
        tq, tr, tw = _dev(q), _dev(r), _dev(w)
        got = gs.gs_sum_exhaustive_noalloc(tq, tr, tw, h).cpu().numpy()
        want = gs.gs_sum(tq, tr, tw, h, 0.0).cpu().numpy()
        assert np.max(np.abs(got - want) / want) <= TOL


def test_noalloc_fp64_input_and_size_limit(gs):
    wl = synth.config1(0.3)
    tq, tw = _dev(wl.queries), _dev(wl.weights)
    got = gs.gs_sum_exhaustive_noalloc(tq, tq, tw, wl.h).cpu().numpy()
    want = gs.gs_sum(tq, tq, tw, wl.h, 0.0).cpu().numpy()
    assert np.max(np.abs(got - want) / want) <= TOL
    big = _dev(np.zeros((2_000_000, 3), np.float32))
    rc, _ = gs.gs_sum_exhaustive_noalloc(big[:10], big, _dev(np.ones(2_000_000, np.float32)), [0.1],
                                         raise_on_error=False)
    assert rc == gs.GS_ERR_ARG and "16 MiB" in gs.gs_last_error()

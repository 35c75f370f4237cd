"""The allocation-free exhaustive entry point (scratch in a fixed device
array inside the library, for callers that cannot let a library allocate
device memory) against the FP64 oracle and against gs_sum's exhaustive mode,
on two calls in a row with different inputs; and a call after the warm-up
leaves the library's pool and the device's free memory unchanged.  Collected
last on purpose, so that a run stopping at the first failure has run every
other test before it."""
import numpy as np
import pytest

from oracle import exhaustive as oracle_ex
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


def test_noalloc_matches_oracle_and_gs_sum_on_consecutive_calls(gs):
    cases = [synth.small_random(301, 20000, 3, m=3000), synth.small_random(302, 7777, 5)]
    hs = [np.array([0.01, 0.05, 0.3]), synth.log_bandwidths(1.0, 9, 1e-3, 1.0)]
    for (q, r, w), h in zip(cases, hs):
        tq, tr, tw = _dev(q), _dev(r), _dev(w)
        got = gs.gs_sum_exhaustive_noalloc(tq, tr, tw, h).cpu().numpy()
        want = gs.gs_sum(tq, tr, tw, h, 0.0).cpu().numpy()
        assert np.max(np.abs(got - want) / want) <= TOL
        # the FP64 oracle on a seeded sample of the queries (the whole set for the smaller case)
        idx = np.arange(q.shape[0]) if q.shape[0] <= 3000 else \
            np.sort(np.random.default_rng(5).choice(q.shape[0], 500, replace=False))
        exact = oracle_ex.gauss_sum(q[idx], r, w, h)
        assert np.max(np.abs(got[idx] - exact) / exact) <= TOL


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


def test_noalloc_call_allocates_nothing(gs):
    """After one warm-up call with the same shapes (which loads the device
    code), a call on new inputs changes neither what the library's memory
    pool holds or uses nor the device's free memory."""
    import torch
    q1, r1, w1 = synth.small_random(303, 9000, 4, m=1500)
    q2, r2, w2 = synth.small_random(304, 9000, 4, m=1500)
    h = np.array([0.02, 0.1, 0.5])
    a = [_dev(v) for v in (q1, r1, w1)]
    b = [_dev(v) for v in (q2, r2, w2)]
    out = torch.empty((1500, 3), dtype=torch.float64, device="cuda")
    gs.gs_sum_exhaustive_noalloc(*a, h, out=out)
    torch.cuda.synchronize()
    pool0 = gs.gs_pool_bytes()
    free0 = torch.cuda.mem_get_info()[0]
    gs.gs_sum_exhaustive_noalloc(*b, h, out=out)
    torch.cuda.synchronize()
    pool1 = gs.gs_pool_bytes()
    free1 = torch.cuda.mem_get_info()[0]
    assert pool1 == pool0
    assert free0 - free1 < (1 << 20), (free0, free1)
    exact = oracle_ex.gauss_sum(q2[:300], r2, w2, h)
    assert np.max(np.abs(out.cpu().numpy()[:300] - exact) / exact) <= TOL

"""Failures made on the host, none on the GPU: an injected allocation failure
at several points of a call surfaces as GS_ERR_OOM and the next call is
correct; invalid inputs are refused with their own codes."""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_injected_allocation_failures(gs):
    q, _, w = synth.small_random(51, 4000, 3)
    h = np.array([0.01, 0.1, 0.5])
    tq, tw = _dev(q), _dev(w)
    exact = oracle_ex.gauss_sum(q, q, w, h)
    W = float(w.astype(np.float64).sum())
    import torch
    lib = gs.load()
    failed = 0
    torch.cuda.synchronize()
    _, used0 = gs.gs_pool_bytes()
    leaks = {}
    try:
        for n in (0, 1, 2, 5, 9, 17, 33, 65, 129):
            lib.gs_debug_fail_alloc(n)
            try:
                gs.gs_sum(tq, tq, tw, h, 1e-2)
            except gs.GSError as e:
                assert e.code == gs.GS_ERR_OOM, e
                failed += 1
            lib.gs_debug_fail_alloc(-1)
            torch.cuda.synchronize()
            leaks[n] = gs.gs_pool_bytes()[1] - used0        # scratch the failed call did not return
            out = gs.gs_sum(tq, tq, tw, h, 1e-2).cpu().numpy()      # the library is still usable
            assert rel_err(out, exact, W).max() <= 1e-2
    finally:
        lib.gs_debug_fail_alloc(-1)
    assert failed >= 4
    assert all(v == 0 for v in leaks.values()), leaks


def test_invalid_inputs_are_refused(gs):
    q, _, w = synth.small_random(52, 500, 2)
    tq = _dev(q)
    bad = q.copy()
    bad[7, 0] = np.inf
    with pytest.raises(gs.GSError) as ei:
        gs.gs_sum(_dev(bad), _dev(bad), _dev(w), [0.1], 1e-2)
    assert ei.value.code == gs.GS_ERR_NONFINITE
    w0 = w.copy()
    w0[3] = -1.0
    with pytest.raises(gs.GSError) as ei:
        gs.gs_sum(tq, tq, _dev(w0), [0.1], 1e-2)
    assert ei.value.code == gs.GS_ERR_WEIGHT
    for h, eps in (([0.0], 1e-2), ([0.1], 1.5), ([np.nan], 1e-2)):
        with pytest.raises(gs.GSError) as ei:
            gs.gs_sum(tq, tq, _dev(w), h, eps)
        assert ei.value.code == gs.GS_ERR_ARG
    with pytest.raises(gs.GSError) as ei:          # eps below what the FP32 base-case charge leaves
        gs.gs_sum(tq, tq, _dev(w), [0.1], 1e-7)
    assert ei.value.code == gs.GS_ERR_ARG

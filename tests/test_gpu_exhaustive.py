"""GPU exhaustive mode (eps = 0) against the FP64 oracle, element by element.

Tolerance: 1e-5 relative per (query, bandwidth), measured against
max(G, 2^-40 W) (the library's relative floor; it only matters for
bichromatic queries far from every reference).
"""
import numpy as np
import pytest

from helpers import rel_err
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


def _run(gs, q, r, w, h, mono, **kw):
    tq = _dev(q)
    tr = tq if mono else _dev(r)
    return gs.gs_sum(tq, tr, _dev(w), h, 0.0, **kw).cpu().numpy()


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 7, 8, 11, 16, 23, 32])
def test_exhaustive_matches_oracle_across_dimensions(gs, D):
    q, r, w = synth.small_random(100 + D, 1537, D, m=611)
    h = np.array([0.02, 0.1, 0.5]) * np.sqrt(D)
    got = _run(gs, q, r, w, h, mono=False)
    want = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(got, want, w.sum()).max() <= TOL


@pytest.mark.parametrize("nh", [1, 2, 3, 5, 8, 9, 16, 33, 64])
def test_exhaustive_all_bandwidth_counts(gs, nh):
    q, r, w = synth.small_random(7, 2049, 3)
    h = synth.log_bandwidths(1.0, nh, 1e-3, 1.0)
    got = _run(gs, q, r, w, h, mono=True)
    want = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(got, want).max() <= TOL


def test_exhaustive_fp64_input_config1(gs):
    wl = synth.config1()
    got = _run(gs, wl.queries, wl.refs, wl.weights, wl.h, mono=True)
    want = oracle_ex.gauss_sum(wl.queries, wl.refs, wl.weights, wl.h)
    assert rel_err(got, want).max() <= TOL


@pytest.mark.parametrize("M,N", [(1, 1), (1, 1000), (1000, 1), (33, 129), (257, 255), (5000, 7)])
def test_exhaustive_ragged_and_tiny_sizes(gs, M, N):
    q, r, w = synth.small_random(M * 7 + N, N, 4, m=M)
    h = np.array([0.05, 0.4])
    got = _run(gs, q, r, w, h, mono=False)
    want = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(got, want, w.sum()).max() <= TOL


def test_exhaustive_limits(gs):
    q, r, w = synth.small_random(3, 3000, 3)
    got = _run(gs, q, r, w, [1e-7, 1e7], mono=True)
    assert np.allclose(got[:, 0], w, rtol=TOL)                    # only the self term
    assert np.allclose(got[:, 1], w.astype(np.float64).sum(), rtol=TOL)


def test_exhaustive_config4_shape_sample(gs):
    """D=16 bichromatic data of the high-dimensional workload, reduced size."""
    wl = synth.config4(0.01)
    got = _run(gs, wl.queries, wl.refs, wl.weights, wl.h, mono=False)
    want = oracle_ex.gauss_sum(wl.queries, wl.refs, wl.weights, wl.h)
    assert rel_err(got, want, wl.weights.astype(np.float64).sum()).max() <= TOL


def test_exhaustive_bad_inputs_report_codes(gs):
    import torch
    q, r, w = synth.small_random(5, 500, 2)
    h = [0.1]
    w_bad = w.copy()
    w_bad[17] = 0.0
    rc, _ = gs.gs_sum(_dev(q), _dev(r), _dev(w_bad), h, 0.0, raise_on_error=False)
    assert rc == gs.GS_ERR_WEIGHT
    q_bad = q.copy()
    q_bad[3, 1] = np.nan
    rc, _ = gs.gs_sum(_dev(q_bad), _dev(r), _dev(w), h, 0.0, raise_on_error=False)
    assert rc == gs.GS_ERR_NONFINITE
    torch.cuda.synchronize()       # context still healthy
    got = _run(gs, q, r, w, h, mono=False)
    assert np.isfinite(got).all()


def test_exhaustive_host_entry_point(gs):
    q, r, w = synth.small_random(9, 1200, 3, m=300)
    h = np.array([0.03, 0.3])
    got = gs.gs_sum_host(q, r, w, h, 0.0)
    want = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(got, want, w.sum()).max() <= TOL


def test_exhaustive_full_size_config2_sampled(gs):
    """Full-size D=3 sweep (1e6 points, 16 bandwidths) on the GPU; the oracle
    checks a seeded sample of 64 queries one by one."""
    import torch
    wl = synth.config2()
    tq = _dev(wl.queries)
    got = gs.gs_sum(tq, tq, _dev(wl.weights), wl.h, 0.0)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(wl.M, 64, replace=False))
    sub = got[torch.from_numpy(idx).cuda()].cpu().numpy()
    want = oracle_ex.gauss_sum(wl.queries[idx], wl.refs, wl.weights, wl.h)
    assert rel_err(sub, want).max() <= TOL


def test_probe_rates(gs):
    ex2, ffma = gs.gs_probe_rates()
    assert 4 <= ex2 <= 256 and 32 <= ffma <= 512

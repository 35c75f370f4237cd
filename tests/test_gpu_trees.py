"""Built trees reused across sums (gs_build_tree / gs_sum_trees / gs_tree_free):
the same results as gs_sum on the same data, every query within eps of the
FP64 oracle, several sums per tree, and the argument checks."""
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


def test_monochromatic_tree_matches_gs_sum(gs):
    q, _, w = synth.small_random(41, 5000, 3)
    tq, tw = _dev(q), _dev(w)
    tree = gs.Tree(tq, tw)
    W = float(w.astype(np.float64).sum())
    for h, eps in (([0.005, 0.05, 0.4], 1e-2), ([0.02, 0.2], 1e-3)):
        a = gs.gs_sum_trees(tree, tree, h, eps).cpu().numpy()
        b = gs.gs_sum(tq, tq, tw, h, eps).cpu().numpy()
        assert np.allclose(a, b, rtol=1e-12, atol=0)
        exact = oracle_ex.gauss_sum(q, q, w, np.asarray(h))
        assert rel_err(a, exact, W).max() <= eps
    tree.close()


def test_bichromatic_trees_and_fp64_points(gs):
    q, r, w = synth.small_random(42, 4000, 4, m=1500, dtype=np.float64)
    o = gs.gs_opts_default()
    o.leaf_size = 16
    qtree = gs.Tree(_dev(q), None, opts=o)
    rtree = gs.Tree(_dev(r), _dev(w), opts=o)
    h = np.array([0.03, 0.3])
    st = gs.gs_stats()
    out = gs.gs_sum_trees(qtree, rtree, h, 1e-2, opts=o, stats=st).cpu().numpy()
    exact = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(out, exact, float(w.astype(np.float64).sum())).max() <= 1e-2
    assert st.pairs_fd + st.pairs_base > 0 and st.ms_phase[gs.GS_PH_TREE] == 0.0   # no tree was built


def test_tree_argument_checks(gs):
    q, r, w = synth.small_random(43, 600, 3, m=200)
    qtree = gs.Tree(_dev(q))
    rtree = gs.Tree(_dev(r), _dev(w))
    with pytest.raises(gs.GSError) as ei:                       # references need weights
        gs.gs_sum_trees(rtree, qtree, [0.1], 1e-2)
    assert ei.value.code == gs.GS_ERR_ARG
    with pytest.raises(gs.GSError) as ei:                       # eps 0 belongs to gs_sum
        gs.gs_sum_trees(qtree, rtree, [0.1], 0.0)
    assert ei.value.code == gs.GS_ERR_ARG
    other = gs.Tree(_dev(synth.small_random(44, 300, 2)[0]))
    with pytest.raises(gs.GSError) as ei:                       # dimensions differ
        gs.gs_sum_trees(other, rtree, [0.1], 1e-2)
    assert ei.value.code == gs.GS_ERR_ARG
    bad = r.copy()
    bad[5, 1] = np.nan
    with pytest.raises(gs.GSError) as ei:
        gs.Tree(_dev(bad), _dev(w))
    assert ei.value.code == gs.GS_ERR_NONFINITE
    wneg = w.copy()
    wneg[0] = 0.0
    with pytest.raises(gs.GSError) as ei:
        gs.Tree(_dev(r), _dev(wneg))
    assert ei.value.code == gs.GS_ERR_WEIGHT
    for t in (qtree, rtree, other):
        t.close()


@pytest.mark.parametrize("n,D,m,dtype,leaf", [(40000, 3, None, np.float32, 32), (70000, 2, 20000, np.float64, 64)])
def test_tree_levels_across_the_per_node_threshold(gs, n, D, m, dtype, leaf):
    """Trees whose upper levels hold nodes of more than 16384 points (built by
    the device-wide level kernels) and whose lower levels are built one CTA
    per node: the permutations equal the CPU tree's bit for bit."""
    from oracle import dualtree as T
    q, r, w = synth.small_random(60 + D, n, D, m=m, dtype=dtype)
    mono = m is None
    tr = _dev(r)
    tq = tr if mono else _dev(q)
    o = gs.gs_opts_default()
    o.leaf_size = leaf
    h = np.array([4.0 * synth.bbox_diagonal(r)])       # everything pruned near the root
    _, _, qperm, rperm = gs.gs_sum_trace(tq, tr, _dev(w), h, 1e-2, opts=o, trace_cap=1 << 16)
    rt = T.build_tree(r, w, leaf)
    assert np.array_equal(rperm.cpu().numpy(), rt.perm)
    if not mono:
        qt = T.build_tree(q, np.ones(q.shape[0], np.float32), leaf)
        assert np.array_equal(qperm.cpu().numpy(), qt.perm)

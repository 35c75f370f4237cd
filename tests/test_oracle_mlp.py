"""Pins of the pair-selector network oracle (oracle/mlp.py) against closed forms,
finite differences and independent compositions."""
import math

import numpy as np
import pytest

from oracle import mlp


def _data(n=64, seed=1):
    g = np.random.default_rng(seed)
    return g.normal(0, 1, (n, mlp.NIN)), g.integers(0, mlp.NOUT, n)


def test_blob_layout():
    assert mlp.NPARAM == 24 + 12 * 64 + 64 + 64 * 64 + 64 + 64 * 5 + 5 == 5341
    blob = np.arange(mlp.NPARAM, dtype=np.float64)
    p = mlp.unpack(blob)
    assert p["mu"][0] == 0 and p["sc"][0] == 12 and p["W1"][0, 1] == 25 and p["W1"][1, 0] == 24 + 64
    assert p["b3"][-1] == mlp.NPARAM - 1
    assert np.array_equal(mlp.pack(p, np.float64), blob)


def test_zero_network_is_uniform():
    # all weights zero: every logit is b3, the loss is log(5) at b3 = 0
    x, y = _data()
    blob = np.zeros(mlp.NPARAM)
    mlp.unpack(blob)["sc"][:] = 1
    assert mlp.loss(blob, x, y) == pytest.approx(math.log(5.0), rel=1e-15)
    b3 = np.array([0.5, -1.0, 2.0, 0.0, 1.0])
    mlp.unpack(blob)["b3"][:] = b3
    lse = math.log(sum(math.exp(v) for v in b3))
    want = np.mean([lse - b3[k] for k in y])
    assert mlp.loss(blob, x, y) == pytest.approx(want, rel=1e-14)
    # the logit gradient of softmax cross entropy is softmax - onehot
    g = mlp.unpack(mlp.grad(blob, x, y))
    pr = np.exp(b3) / np.exp(b3).sum()
    onehot = np.bincount(y, minlength=5) / len(y)
    assert np.allclose(g["b3"], pr - onehot, rtol=0, atol=1e-15)
    assert not g["W1"].any() and not g["W2"].any()


def test_linear_regime_equals_matrix_product():
    # positive inputs, weights and biases keep every unit active, so the
    # network is the affine map z (W1 W2 W3) + (b1 W2 W3 + b2 W3 + b3)
    g = np.random.default_rng(3)
    p = {"mu": g.normal(0, 1, 12), "sc": g.uniform(0.5, 2, 12), "W1": g.uniform(0, 1, (12, 64)),
         "b1": g.uniform(0, 1, 64), "W2": g.uniform(0, 1, (64, 64)), "b2": g.uniform(0, 1, 64),
         "W3": g.normal(0, 1, (64, 5)), "b3": g.normal(0, 1, 5)}
    blob = mlp.pack(p, np.float64)
    x = p["mu"] + g.uniform(0, 1, (20, 12))
    z = (x - p["mu"]) * p["sc"]
    M = p["W1"] @ p["W2"] @ p["W3"]
    c = p["b1"] @ p["W2"] @ p["W3"] + p["b2"] @ p["W3"] + p["b3"]
    o, _ = mlp.forward(blob, x)
    assert np.allclose(o, z @ M + c, rtol=1e-12, atol=1e-9)


def test_gradient_matches_finite_differences():
    x, y = _data(48, seed=5)
    s = np.random.default_rng(6).uniform(0.5, 2.0, len(y))
    blob = mlp.init(seed=7).astype(np.float64)
    p = mlp.unpack(blob)
    p["mu"][:] = 0.1
    p["sc"][:] = 0.9
    p["b1"][:] = np.random.default_rng(8).normal(0, 0.1, 64)
    g = mlp.grad(blob, x, y, s)
    rng = np.random.default_rng(9)
    off = 0
    for name, shp in mlp.SHAPES:
        n = int(np.prod(shp))
        if name in mlp.TRAINED:
            for i in rng.choice(n, size=min(n, 12), replace=False):
                k = off + int(i)
                hstep = 1e-6
                bp = blob.copy(); bp[k] += hstep
                bm = blob.copy(); bm[k] -= hstep
                fd = (mlp.loss(bp, x, y, s) - mlp.loss(bm, x, y, s)) / (2 * hstep)
                assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (name, i, fd, g[k])
        else:
            assert not g[off:off + n].any()
        off += n


def test_adam_first_step_is_signed_lr():
    g = np.random.default_rng(2).normal(0, 1e-2, mlp.NPARAM)
    blob = np.zeros(mlp.NPARAM)
    nb, m, v = mlp.adam_step(blob, np.zeros(mlp.NPARAM), np.zeros(mlp.NPARAM), g, 1, lr=1e-3)
    p = mlp.unpack(nb)
    gg = mlp.unpack(g)
    assert not p["mu"].any() and not p["sc"].any()
    for name in mlp.TRAINED:
        assert np.allclose(p[name], -1e-3 * gg[name] / (np.abs(gg[name]) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_plog2():
    f = mlp.plog2_f32
    for k in (-126, -40, -1, 0, 1, 7, 24, 127):
        assert f(np.float32(2.0 ** k)) == k
    assert f(np.float32(3.0)) == 1.5 and f(np.float32(0.75)) == np.float32(-0.5)
    assert f(np.float32(0.0)) == -150 and f(np.float32(1e-40)) == -150 and f(np.float32(np.inf)) == 128
    xs = np.float32(2.0) ** np.random.default_rng(4).uniform(-120, 120, 4000).astype(np.float32)
    xs = np.sort(xs)
    v = f(xs)
    assert np.all(np.diff(v) >= 0)
    # chord of log2 on each octave: never above log2, at most 0.0861 below it
    err = np.log2(xs.astype(np.float64)) - v.astype(np.float64)
    assert err.min() > -1e-6 and err.max() < 0.0861


def test_fp32_inference_close_to_fp64():
    x, _ = _data(200, seed=11)
    blob = mlp.init(seed=12)
    o64, _ = mlp.forward(blob.astype(np.float64), x.astype(np.float32).astype(np.float64))
    o32 = mlp.infer_f32(blob, x)
    assert o32.dtype == np.float32
    assert np.allclose(o32, o64, rtol=1e-4, atol=1e-4)

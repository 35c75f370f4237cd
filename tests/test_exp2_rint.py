"""The frontier's FP32 exp2 takes rint(x) and the integer exponent from one
FP32 addition of 1.5 * 2^23 (round-to-nearest-even puts rint(x) in the low
bits of the sum) instead of rintf and a float-to-int conversion.  Emulated in
numpy float32 over the whole argument range the kernel uses (-125 <= x <= 0):
the same k, the same integer, for every half-integer, its neighbours and
random arguments."""
import numpy as np


def test_magic_add_equals_rint():
    rng = np.random.default_rng(0)
    half = (np.arange(-126, 1) + 0.5).astype(np.float32)
    xs = np.concatenate([rng.uniform(-125, 0, 2_000_000).astype(np.float32), half,
                         np.nextafter(half, np.float32(-200)), np.nextafter(half, np.float32(200)),
                         np.arange(-125, 1).astype(np.float32), np.array([-0.0, -1e-30, -125.0], np.float32)])
    x = xs[(xs >= -125) & (xs <= 0)]
    magic = np.float32(12582912.0)                   # 1.5 * 2^23
    t = (x + magic).astype(np.float32)
    k = (t - magic).astype(np.float32)
    ki = t.view(np.int32) - magic.view(np.int32)
    assert np.array_equal(k, np.rint(x))
    assert np.array_equal(ki, np.rint(x).astype(np.int32))

"""The frontier reduces its FP64 group sums onto lane 0 with shfl_down steps
(only the lanes whose partial sum lane 0 still reads add) instead of the
full xor butterfly.  Emulated here in IEEE doubles: lane 0's result is the
butterfly's, bit for bit, for adversarial and random inputs."""
import numpy as np


def _xor_butterfly(v):
    v = np.array(v, dtype=np.float64)
    for m in (16, 8, 4, 2, 1):
        v = v + v[np.arange(32) ^ m]
    return v[0]


def _down_lane0(v):
    v = np.array(v, dtype=np.float64)
    for m in (16, 8, 4, 2, 1):
        o = np.concatenate([v[m:], v[:m]])           # shfl_down: lane l reads lane l + m
        lanes = np.arange(32) < m
        v = np.where(lanes, v + o, v)
    return v[0]


def test_lane0_sum_equals_butterfly():
    rng = np.random.default_rng(7)
    cases = [rng.standard_normal(32) * 10.0 ** rng.uniform(-8, 8, 32) for _ in range(2000)]
    cases.append(np.array([1e16, 1.0, -1e16, 1.0] * 8))
    cases.append(np.array([2.0 ** -1074] * 31 + [1.0]))
    cases.append(np.zeros(32))
    for v in cases:
        a, b = _xor_butterfly(v), _down_lane0(v)
        assert a == b or (np.isnan(a) and np.isnan(b)), (v, a, b)
        assert np.signbit(a) == np.signbit(b)

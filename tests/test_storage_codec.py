"""The 24-bit population storage's encoding, as the tests state it (helpers.f24_value), against
values worked out by hand. The GPU round trip must equal this statement bit for bit
(test_storage24_gpu.py)."""
import numpy as np

from helpers import f24_value


def test_f24_keeps_eight_more_bits_than_fp16():
    # 1 + 2^-12: FP16 cuts it to 1 (spacing 2^-10); the byte keeps 2^-12 = 64 steps of 2^-18 exactly
    assert f24_value(np.float32(1 + 2.0 ** -12), 1.0) == np.float32(1 + 2.0 ** -12)
    # halfway between two FP16 values: 128 steps, kept exactly (no clamping)
    assert f24_value(np.float32(1 + 2.0 ** -11), 1.0) == np.float32(1 + 2.0 ** -11)
    # 1 + 2^-20: a quarter step, rounds back to 1
    assert f24_value(np.float32(1 + 2.0 ** -20), 1.0) == np.float32(1.0)
    # 1 + 3 * 2^-19: 1.5 steps, a tie, rounds to the even count 2; the sign follows h
    assert f24_value(np.float32(1 + 3 * 2.0 ** -19), 1.0) == np.float32(1 + 2.0 ** -17)
    assert f24_value(np.float32(-(1 + 3 * 2.0 ** -19)), 1.0) == np.float32(-(1 + 2.0 ** -17))


def test_f24_carries_into_the_half():
    # 1 + 2^-10 - 2^-20 is 255.75 steps above 1: rounds to 256, which carries to the FP16 value
    # 1 + 2^-10 with no remainder
    assert f24_value(np.float32(1 + 2.0 ** -10 - 2.0 ** -20), 1.0) == np.float32(1 + 2.0 ** -10)
    # the carry crosses a binade: 2 - 2^-22 is cut to 2 - 2^-10 and carries to 2
    assert f24_value(np.float32(2 - 2.0 ** -22), 1.0) == np.float32(2.0)
    assert f24_value(np.float32(-(2 - 2.0 ** -22)), 1.0) == np.float32(-2.0)
    # beyond FP16's largest value (65504) the value saturates at 65504 + 255 steps of 2^-3
    assert f24_value(np.float32(1e6), 1.0) == np.float32(65504 + 255 * 2.0 ** -3)


def test_f24_scale_and_small_values():
    # a power-of-two scale is exact: 1.25 * 2^-20 stored at scale 2^10 is an FP16 normal, kept exactly
    assert f24_value(np.float32(1.25 * 2.0 ** -20), 2.0 ** 10) == np.float32(1.25 * 2.0 ** -20)
    # below FP16's subnormals the byte alone holds the value in steps of 2^-32
    assert f24_value(np.float32(5 * 2.0 ** -32), 1.0) == np.float32(5 * 2.0 ** -32)
    assert f24_value(np.float32(-5 * 2.0 ** -32), 1.0) == np.float32(-5 * 2.0 ** -32)
    assert f24_value(np.float32(0.0), 1.0) == 0.0


def test_f24_relative_error_bound():
    """At most 2^-19 relative over FP16's normal range (half a step of ulp(h) / 256 against |x| >=
    |h|), against 2^-11 for FP16 alone."""
    rng = np.random.default_rng(5)
    x = np.float32(rng.uniform(2.0 ** -13, 6e4, 200000) * rng.choice([-1.0, 1.0], 200000))
    rel = np.abs(f24_value(x, 1.0).astype(np.float64) / x - 1)
    assert rel.max() <= 2.0 ** -19
    rel16 = np.abs(x.astype(np.float16).astype(np.float64) / x - 1)
    assert 2.0 ** -12 < rel16.max() <= 2.0 ** -11

"""The FP32 error bound behind the undecided band of the block-level decisions.

A block's level (Section 3.1, Eq. 1-3) compares squared norms of speed and acceleration
with thresholds.  The definition is the FP64 comparison of the FP64 square norm of the
FP32 components with the FP64 threshold; the kernels form the square norm in FP32 and
compare it with the threshold rounded to FP32, and take the exact FP64 decision only when
the FP32 maximum lies within 1e-6 (relative) of a threshold.  That is sound if the FP32
square norm is within 3e-7 of the FP64 one and the rounded threshold within 6e-8 of the
FP64 one, the band then exceeding the sum of both errors more than twice.  These checks
measure both errors on adversarial and random inputs, for the evaluation orders the
compiler may choose (separate products and sums, or fused multiply-adds).
"""
import numpy as np

BAND = 1e-6           # undecided band of a block maximum
NORM_ERR = 3e-7       # claimed bound on the FP32 square norm's relative error
THR_ERR = 6e-8        # claimed bound on the rounded threshold's relative error


def _fma32(a, b, c):
    # a * b + c rounded once to FP32 (the product of two FP32 values is exact in FP64,
    # and the FP64 sum's own rounding is far below an FP32 ulp)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _norms32(x, y, z):
    """The orders a compiler may use for x*x + y*y + z*z in FP32."""
    sep = (x * x + y * y) + z * z                      # three products, two sums
    fused = _fma32(z, z, _fma32(y, y, x * x))          # one product, two fused steps
    fused2 = _fma32(x, x, _fma32(y, y, z * z))
    return sep, fused, fused2


def _exact(x, y, z):
    x64, y64, z64 = (t.astype(np.float64) for t in (x, y, z))
    return (x64 * x64 + y64 * y64) + z64 * z64


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-3, 3, size=(n, 1))
    v = (rng.standard_normal((n, 3)) * mag).astype(np.float32)
    # adversarial: components whose squares round the same way (just above a power of two)
    u = (1.0 + rng.integers(1, 64, size=(n // 4, 3)) * 2.0 ** -23).astype(np.float32)
    u *= (2.0 ** rng.integers(-10, 10, size=(n // 4, 1))).astype(np.float32)
    return np.concatenate([v, u])


def test_fp32_square_norm_is_within_the_claimed_error_of_the_fp64_one():
    v = _samples(400_000, seed=17)
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    ref = _exact(x, y, z)
    ok = ref > 0
    for f32 in _norms32(x, y, z):
        rel = np.abs(f32.astype(np.float64) - ref)[ok] / ref[ok]
        assert rel.max() <= NORM_ERR, rel.max()


def test_rounded_thresholds_are_within_the_claimed_error():
    rng = np.random.default_rng(5)
    thr = 10.0 ** rng.uniform(-6, 12, size=200_000)
    rel = np.abs(thr.astype(np.float32).astype(np.float64) - thr) / thr
    assert rel.max() <= THR_ERR, rel.max()


def test_band_exceeds_both_errors_with_margin():
    assert BAND > 2.0 * (NORM_ERR + THR_ERR)


def test_decisions_outside_the_band_agree_with_fp64():
    # components scaled so that the square norm lands in a narrow window around a
    # threshold: outside the band the FP32 decision (every evaluation order) equals the
    # FP64 one; inside it the kernels defer to the FP64 form, so nothing is asserted there
    rng = np.random.default_rng(23)
    thr = 2.7183 ** 2 * 1.0001
    n = 300_000
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.sqrt(thr) * (1.0 + rng.uniform(-2e-5, 2e-5, size=(n, 1)))
    v = (d * r).astype(np.float32)
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    ref_le = _exact(x, y, z) <= thr
    t32 = np.float32(thr)
    for f32 in _norms32(x, y, z):
        outside = np.abs(f32 - t32) > np.float32(BAND) * t32
        assert outside.sum() > n // 2
        assert np.array_equal((f32 <= t32)[outside], ref_le[outside])

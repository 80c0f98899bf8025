"""The integer truncation tests of the kernels, checked on the CPU.

The kernels decide |c| < delta (and the relative |c| <= eps0 * max) on the
magnitude bits of the stored coefficient: IEEE magnitudes of one format
order like their bit patterns.  For FP64 the threshold is delta's own bits.
For FP32 the host rounds the FP64 threshold to a float: up (the smallest
float >= delta) for the absolute test, down (the largest float <= thr) for
the strict relative test, so that the test on a float value equals the
comparison of that value with the FP64 threshold.  This is the rule
written with numpy, checked against direct comparisons on values around
many thresholds."""
import numpy as np


def _mag64(v):
    return np.asarray(v, dtype=np.float64).view(np.uint64) & np.uint64(0x7FFFFFFFFFFFFFFF)


def _mag32(v):
    return np.asarray(v, dtype=np.float32).view(np.uint32) & np.uint32(0x7FFFFFFF)


def _ge_bits32(d):
    f = np.float32(d)
    if float(f) < d:
        f = np.nextafter(f, np.float32(np.inf))
    return _mag32(f)


def _gt_bits32(d):
    f = np.float32(d)
    if float(f) > d:
        f = np.nextafter(f, np.float32(0))
    return _mag32(f)


def _around(rng, d, dtype):
    """Values of type dtype at and around +-d: neighbours in ulps, and random."""
    base = np.asarray(d, dtype=dtype)
    near = [base]
    up = down = base
    for _ in range(4):
        up = np.nextafter(up, dtype(np.inf))
        down = np.nextafter(down, dtype(0))
        near += [up, down]
    vals = np.array(near + list(rng.uniform(0.5 * d, 2 * d, 64).astype(dtype)), dtype=dtype)
    return np.concatenate([vals, -vals, np.array([0.0, -0.0], dtype=dtype)])


def test_fp64_bits_order_like_values():
    rng = np.random.default_rng(1)
    for d in list(10.0 ** rng.uniform(-300, 2, 200)) + [1e-4, 3.5e-6, 1e-5]:
        v = _around(rng, d, np.float64)
        keep_bits = (_mag64(v) != 0) & (_mag64(v) >= _mag64(d))
        keep_vals = (v != 0) & (np.abs(v) >= d)
        assert np.array_equal(keep_bits, keep_vals), d


def test_fp32_absolute_rule_equals_fp64_comparison():
    rng = np.random.default_rng(2)
    for d in list(10.0 ** rng.uniform(-37, 2, 300)) + [1e-4, 3.5e-6, 1e-5, 0.1]:
        v = _around(rng, d, np.float32)
        keep_bits = (_mag32(v) != 0) & (_mag32(v) >= _ge_bits32(d))
        keep_vals = (v != 0) & (np.abs(v.astype(np.float64)) >= d)
        assert np.array_equal(keep_bits, keep_vals), d


def test_fp32_relative_rule_equals_fp64_comparison():
    """Relative mode keeps c iff |c| > thr = eps0 * max|c| (formed in FP64)."""
    rng = np.random.default_rng(3)
    for thr in list(10.0 ** rng.uniform(-37, 1, 300)) + [1e-5 * 0.9531153132139318]:
        v = _around(rng, thr, np.float32)
        keep_bits = _mag32(v) > _gt_bits32(thr)
        keep_vals = np.abs(v.astype(np.float64)) > thr
        assert np.array_equal(keep_bits, keep_vals), thr

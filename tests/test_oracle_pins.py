"""The oracle against what the paper and the mathematics fix (CPU only)."""
import math
from fractions import Fraction
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1109_1264_gb300 import inputs
import oracle_pins


@pytest.fixture(scope="module")
def libpath():
    return oracle.build()


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(check, libpath):
    check(libpath)


def test_exact_sum_matches_fsum():
    """The vectorised exact summation agrees with math.fsum (an independent
    correctly rounded summation) on hard cases."""
    rng = np.random.default_rng(1)
    for n in (1, 2, 17, 1000, 50000):
        p = rng.standard_normal(n) * 10.0 ** rng.uniform(-20, 20, n)
        assert exact.exact_sum(p) == math.fsum(p.tolist())
    p = np.array([1e100, 1.0, -1e100, 1e-100])
    assert exact.exact_sum(p) == math.fsum(p.tolist()) == 1.0


def test_exact_dot_matches_fractions():
    rng = np.random.default_rng(2)
    for dt in (np.float64, np.float32):
        for n in (0, 1, 5, 64, 300):
            x = (rng.standard_normal(n) * 10.0 ** rng.uniform(-8, 8, n)).astype(dt)
            y = (rng.standard_normal(n) * 10.0 ** rng.uniform(-8, 8, n)).astype(dt)
            assert exact.exact_dot(x, y) == float(exact.fraction_dot(x, y)), (dt, n)


def _golden_splitmix():
    rows = []
    for line in open(os.path.join(oracle_pins.GOLDEN, "splitmix64.txt")):
        if line.strip() and not line.startswith("#"):
            s, k, v = line.split()
            rows.append((int(s), int(k), int(v, 0)))
    return rows


def test_splitmix64_reference_outputs():
    """The counter-based input generator reproduces SplitMix64's published
    output sequence."""
    for state, k, want in _golden_splitmix():
        assert int(inputs.splitmix64(state, np.array([k - 1]))[0]) == want


def test_hash_uniform_exact_and_in_range():
    """FP64 / FP32 values are 2*(h >> 11)*2^-53 - 1 and 2*(h >> 40)*2^-24 - 1,
    recomputed here with Python integers."""
    mask = (1 << 64) - 1
    key = 987654321

    def mix(i):
        z = (key + (i + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)

    got64 = inputs.hash_uniform(key, 300, np.float64, offset=5)
    got32 = inputs.hash_uniform(key, 300, np.float32, offset=5)
    for j in range(300):
        h = mix(j + 5)
        assert Fraction(float(got64[j])) == 2 * Fraction(h >> 11, 2 ** 53) - 1
        assert Fraction(float(got32[j])) == 2 * Fraction(h >> 40, 2 ** 24) - 1
    assert got64.min() >= -1 and got64.max() < 1


def test_uniform_vectors_recipe():
    a, b = inputs.uniform_vectors(0, 1000, 2)
    rng = np.random.default_rng(0)
    assert np.array_equal(a, rng.uniform(-1, 1, 1000))
    assert np.array_equal(b, rng.uniform(-1, 1, 1000))


def test_fixed_point_dot_matches_the_exact_dot():
    """The piecewise fixed-point dot product equals exact_dot (an
    independent error-free-transformation method) bit for bit, for FP64 and
    FP32 counter-based data of random sign and of one sign, cut into pieces
    of uneven length; with Fractions on a tiny case; and it rejects values
    that are not integers at the stated scale."""
    for dt, fb in ((np.float64, 52), (np.float32, 23)):
        x = inputs.hash_uniform(71, 40_003, dt)
        y = inputs.hash_uniform(72, 40_003, dt)
        for xs, ys in ((x, y), (np.abs(x), np.abs(y)), (x, x)):
            f = exact.FixedPointDot(fb, fb)
            for lo, hi in ((0, 1), (1, 777), (777, 30_000), (30_000, 40_003)):
                f.add(xs[lo:hi], ys[lo:hi])
            assert f.value() == exact.exact_dot(xs, ys), dt
            assert f.abs_value() == exact.abs_dot(xs, ys), dt
        f = exact.FixedPointDot(fb, fb)
        f.add(x[:9], y[:9])
        assert f.value() == float(exact.fraction_dot(x[:9], y[:9]))
    # extreme integers: |a| = 2^52 exactly, and the most negative split halves
    a = np.array([1.0, -1.0, -1.0 + 2.0 ** -52, 1.0 - 2.0 ** -52, -2.0 ** -52])
    f = exact.FixedPointDot(52, 52)
    f.add(a, a[::-1].copy())
    assert f.value() == float(exact.fraction_dot(a, a[::-1]))
    with pytest.raises(ValueError):
        exact.FixedPointDot(10, 10).add(np.array([2.0 ** -11]), np.array([1.0]))

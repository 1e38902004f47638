"""Pins of the oracle's random-number and arithmetic building blocks.

Each test ties an oracle function to something outside the oracle: published
SplitMix64 outputs, the C library's log/cos/sin (accuracy of our FP32 series
only), closed forms,
exact rational arithmetic, and the geometry of the uniform distribution on the
sphere (Archimedes: the z-coordinate of a uniform point on S^2 is uniform on
[-1, 1]).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def test_mix64_matches_published_splitmix64_outputs():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for k, hexv in rows:
        assert oracle.mix64((int(k) * GAMMA) & M64) == int(hexv, 16)


def test_u53_range_and_endpoints():
    assert oracle.u53(0) == 0.0
    assert oracle.u53(M64) == 1.0 - 2.0 ** -53
    assert oracle.u53(1 << 11) == 2.0 ** -53


def test_word_is_uniform_and_field_sensitive():
    # every field changes the word; u53 of the words is close to U[0,1)
    base = oracle.word(0, 1, 2, 3, 4, 5)
    for i in range(6):
        f = [0, 1, 2, 3, 4, 5]
        f[i] += 1
        assert oracle.word(*f) != base
    u = np.array([oracle.u53(oracle.word(7, 1, 0, 1, 0, c)) for c in range(20000)])
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1.0 / 12.0) < 0.005
    hist, _ = np.histogram(u, bins=10, range=(0, 1))
    assert hist.min() > 1800 and hist.max() < 2200


def test_child_keys_distinct_along_paths():
    seen = {1}
    frontier = [1]
    for _ in range(12):
        nxt = []
        for k in frontier:
            for s in (0, 1):
                c = oracle.child_key(k, s)
                assert c not in seen
                seen.add(c)
                nxt.append(c)
        frontier = nxt


def test_lnf_special_values_are_exact():
    assert oracle.lnf(1.0) == 0.0
    ln2 = oracle.lnf(2.0)
    assert oracle.lnf(0.5) == -ln2
    assert ln2 == np.float32(math.log(2.0))
    for k in range(1, 25):
        # m = 1 exactly, so the result is the single FP32 rounding of -k * ln2f
        assert oracle.lnf(2.0 ** -k) == np.float32(-k * float(np.float32(math.log(2.0))))


def test_lnf_accuracy_against_libm():
    rng = np.random.default_rng(1)
    # the Box-Muller inputs: u = j 2^-24, j in [1, 2^24]
    js = np.concatenate([rng.integers(1, 2 ** 24 + 1, 6000), np.arange(1, 300),
                         2 ** 24 - np.arange(0, 300)])
    for j in js:
        u = np.float32(float(j) * 2.0 ** -24)
        ref = math.log(float(u))
        got = float(oracle.lnf(u))
        assert abs(got - ref) <= 3 * float(np.spacing(np.float32(abs(ref)))) + 2.0 ** -26, (u, got, ref)


def test_sincos2pif_quadrant_points_and_accuracy():
    assert oracle.sincos2pif(0.0) == (1.0, 0.0)
    c, s = oracle.sincos2pif(0.25)
    assert c == 0.0 and s == 1.0
    c, s = oracle.sincos2pif(0.5)
    assert c == -1.0 and s == 0.0
    c, s = oracle.sincos2pif(0.75)
    assert c == 0.0 and s == -1.0
    rng = np.random.default_rng(2)
    for j in rng.integers(0, 2 ** 24, 6000):
        u = float(j) * 2.0 ** -24  # exact in FP32
        c, s = oracle.sincos2pif(u)
        assert abs(float(c) - math.cos(2 * math.pi * u)) < 4e-7
        assert abs(float(s) - math.sin(2 * math.pi * u)) < 4e-7


def test_direction_unit_norm_and_determinism():
    for d in (1, 2, 3, 10, 64, 127):
        for j in range(3):
            r = oracle.direction(0, 5, 12345, j, d)
            assert np.array_equal(r.astype(np.float32).astype(np.float64), r)  # FP32 values
            assert abs(math.fsum(r * r) - 1.0) < (d + 4) * 2.0 ** -23
            assert np.array_equal(r, oracle.direction(0, 5, 12345, j, d))
    assert not np.array_equal(oracle.direction(0, 5, 12345, 0, 8), oracle.direction(0, 5, 12345, 1, 8))
    assert not np.array_equal(oracle.direction(0, 5, 12345, 0, 8), oracle.direction(1, 5, 12345, 0, 8))
    # d = 1: the unit directions are +1 and -1 (up to the FP32 rounding of
    # g * (1/|g|)), and both must occur
    vals = np.array([oracle.direction(0, 0, k, 0, 1)[0] for k in range(40)])
    assert np.all(np.abs(np.abs(vals) - 1.0) <= 2.0 ** -23)
    assert set(np.sign(vals)) == {1.0, -1.0}


def test_direction_uniform_on_sphere_archimedes():
    # For r uniform on S^2 each coordinate is uniform on [-1, 1]; a dropped
    # series term or a wrong quadrant in the Gaussian breaks this.
    zs = np.array([oracle.direction(3, 0, k, 0, 3) for k in range(6000)])
    for col in range(3):
        z = np.sort(zs[:, col])
        cdf = (z + 1.0) / 2.0
        ks = np.max(np.abs(cdf - (np.arange(1, len(z) + 1) / len(z))))
        assert ks < 1.63 / math.sqrt(len(z)) * 1.2, (col, ks)  # ~1% level
    # and for d = 2 the angle is uniform
    a = np.array([oracle.direction(4, 1, k, 2, 2) for k in range(6000)])
    ang = np.sort((np.arctan2(a[:, 1], a[:, 0]) + np.pi) / (2 * np.pi))
    ks = np.max(np.abs(ang - np.arange(1, len(ang) + 1) / len(ang)))
    assert ks < 1.63 / math.sqrt(len(ang)) * 1.2


def test_direction_gaussian_moments_in_high_dim():
    d = 256
    R = np.array([oracle.direction(9, 0, k, 0, d) for k in range(400)]) * math.sqrt(d)
    v = R.ravel()
    assert abs(v.mean()) < 0.01
    assert abs(v.var() - 1.0) < 0.02
    assert abs(np.mean(v ** 4) - 3.0) < 0.1  # Gaussian kurtosis
    # distinct coordinates are uncorrelated (sin and cos halves of one pair)
    assert abs(np.mean(R[:, 0] * R[:, 1])) < 0.1


def test_proj_exact_for_small_integers_and_bounded_otherwise():
    x = np.array([1, -2, 3, 4, -5, 6], np.float32)
    r = np.array([0.5, 0.25, -1.0, 2.0, 0.125, -0.75])
    assert oracle.proj(x, r) == float(sum(Fraction(float(a)) * Fraction(b) for a, b in zip(x, r)))
    rng = np.random.default_rng(3)
    for _ in range(300):
        d = int(rng.integers(1, 200))
        x = rng.standard_normal(d).astype(np.float32)
        r = rng.standard_normal(d)
        exact = float(sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, r)))
        bound = d * 2.0 ** -53 * float(np.sum(np.abs(x.astype(np.float64) * r))) * 1.01
        assert abs(oracle.proj(x, r) - exact) <= bound


def test_csum_worked_example_lane_order():
    # 33 values: 2^53 at position 0, ones at positions 1 and 33.  Lane 1 sums
    # 1 + 1 = 2 before the lanes are folded, so the canonical sum is 2^53 + 2
    # exactly, while a left-to-right sum would lose both ones.
    v = np.zeros(34)
    v[0] = 2.0 ** 53
    v[1] = 1.0
    v[33] = 1.0
    assert oracle.csum(v) == 2.0 ** 53 + 2.0
    seq = 0.0
    for a in v:
        seq += a
    assert seq == 2.0 ** 53


def test_csum_exact_on_integers_and_bounded_on_random():
    rng = np.random.default_rng(4)
    for m in (0, 1, 31, 32, 33, 4095, 4096, 4097, 9000, 300000):
        v = rng.integers(-1000, 1000, size=m).astype(np.float64)
        assert oracle.csum(v) == float(v.sum())
    for m in (5, 100, 5000, 200000):
        v = rng.standard_normal(m) * np.exp(rng.uniform(-5, 5, m))
        err = abs(oracle.csum(v) - math.fsum(v))
        assert err <= (m / 32 + 32) * 2.0 ** -53 * np.sum(np.abs(v))


def test_d32_symmetric_and_close_to_fp64():
    rng = np.random.default_rng(5)
    for d in (1, 10, 64, 128):
        for _ in range(100):
            x = (rng.standard_normal(d) * 3).astype(np.float32)
            y = (rng.standard_normal(d) * 3).astype(np.float32)
            a, b = oracle.d32(x, y), oracle.d32(y, x)
            assert a == b
            exact = float(sum((Fraction(float(p)) - Fraction(float(q))) ** 2 for p, q in zip(x, y)))
            # d rounded differences and d rounded fma steps in FP32
            assert abs(float(a) - exact) <= (2 * d + 2) * 2.0 ** -24 * exact
    assert oracle.d32(np.ones(7, np.float32), np.ones(7, np.float32)) == 0.0

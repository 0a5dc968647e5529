"""Pins of the oracle's input encoding (Sec. 3.6, Table 1; cheap primitives of Sec. 5 / Fig. 7).

Each test checks the oracle against something other than itself: exact values
of the triangle wave and the sine at dyadic points, trigonometric identities,
quadrature of the kernels, partition-of-unity and mirror invariants of the
one-blob bins, and the 62 + 2 = 64 feature layout of Table 1.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2106_12372_gb300 import synth

pytestmark = pytest.mark.usefixtures("oracle_lib")


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def test_tri_exact_values(O):
    # Fig. 7: tri(x) = 2|x mod 2 - 1| - 1.
    table = {0.0: 1.0, 0.25: 0.5, 0.5: 0.0, 1.0: -1.0, 1.5: 0.0, 2.0: 1.0, -0.5: 0.0, -1.0: -1.0, 3.75: 0.5}
    for x, v in table.items():
        assert O.tri(x) == v, x


def test_tri_period_and_symmetry(O):
    rng = np.random.default_rng(1)
    for x in rng.uniform(-50, 50, 200):
        assert abs(O.tri(x + 2.0) - O.tri(x)) < 1e-12
        assert abs(O.tri(-x) - O.tri(x)) < 1e-12
        assert -1.0 <= O.tri(x) <= 1.0


@pytest.mark.parametrize("d", range(12))
def test_cheap_frequency_matches_sine_at_dyadic_points(O, d):
    # tri(2^d x - 1/2) agrees with sin(2^d pi x) wherever 2^(d+1) x is an integer
    # (values 0, +1, -1) -- the triangle wave replaces the sine with the same phase and period.
    for m in range(0, 2 ** (d + 2) + 1):
        x = m / 2.0 ** (d + 1)
        ref = round(math.sin(math.pi * 2.0 ** d * x))
        assert O.freq_feature(x, d, O.ENC_CHEAP) == ref


@pytest.mark.parametrize("d", range(11))
def test_exact_frequency_double_angle(O, d):
    # sin(2^(d+1) pi x) = 2 sin(2^d pi x) cos(2^d pi x), with cos(2^d pi x) = f_d(x + 2^-(d+1)).
    rng = np.random.default_rng(d)
    for x in rng.uniform(0, 1, 50):
        lhs = O.freq_feature(x, d + 1, O.ENC_EXACT)
        rhs = 2.0 * O.freq_feature(x, d, O.ENC_EXACT) * O.freq_feature(x + 2.0 ** -(d + 1), d, O.ENC_EXACT)
        assert abs(lhs - rhs) < 1e-9


@pytest.mark.parametrize("d", range(12))
def test_frequency_periods(O, d):
    rng = np.random.default_rng(100 + d)
    for x in rng.uniform(0, 1, 50):
        for mode in (O.ENC_CHEAP, O.ENC_EXACT):
            assert abs(O.freq_feature(x + 2.0 ** (1 - d), d, mode) - O.freq_feature(x, d, mode)) < 1e-9
        assert abs(O.freq_feature(x, d, O.ENC_EXACT) - math.sin(math.pi * 2.0 ** d * x)) < 1e-9


def test_quartic_is_a_density(O):
    val, _ = integrate.quad(O.quartic, -1.0, 1.0)
    assert abs(val - 1.0) < 1e-12
    assert O.quartic(0.0) == 15.0 / 16.0
    assert O.quartic(1.0) == 0.0 and O.quartic(-1.5) == 0.0


def test_quartic_cdf_is_antiderivative(O):
    for y in np.linspace(-1.2, 1.2, 25):
        val, _ = integrate.quad(O.quartic, 0.0, float(y), points=[-1.0, 1.0] if abs(y) > 1 else None)
        assert abs(O.quartic_cdf(y) - val) < 1e-12
    assert abs(O.quartic_cdf(1.0) - 0.5) < 1e-15 and abs(O.quartic_cdf(-1.0) + 0.5) < 1e-15


def test_oneblob_partition_of_unity(O):
    for s in np.linspace(0, 1, 81):
        for mode in (O.ENC_CHEAP,):
            b = O.oneblob(s, 4, mode)
            assert np.all(b >= -1e-15)
            if 0.25 <= s <= 0.75:
                assert abs(b.sum() - 1.0) < 1e-12
            else:  # mass that falls outside [0, 1] is lost (no wrap)
                assert abs(b.sum() - (O.quartic_cdf(4 - 4 * s) - O.quartic_cdf(-4 * s))) < 1e-12
                assert b.sum() < 1.0


def test_oneblob_mirror_symmetry(O):
    for s in np.linspace(0, 1, 41):
        for mode in (O.ENC_CHEAP, O.ENC_EXACT):
            assert np.allclose(O.oneblob(s, 4, mode), O.oneblob(1 - s, 4, mode)[::-1], atol=1e-13)


@pytest.mark.parametrize("s", [0.0, 0.1, 0.3, 0.5, 0.62, 0.9, 1.0])
def test_oneblob_bins_hold_kernel_mass(O, s):
    k = 4
    q = O.oneblob(s, k, O.ENC_CHEAP)
    g = O.oneblob(s, k, O.ENC_EXACT)
    for i in range(k):
        lo, hi = i / k, (i + 1) / k
        mq, _ = integrate.quad(lambda t: k * O.quartic(k * (t - s)), lo, hi, points=[s - 1 / k, s, s + 1 / k])
        mg = stats.norm(loc=s, scale=1.0 / k).cdf(hi) - stats.norm(loc=s, scale=1.0 / k).cdf(lo)
        assert abs(q[i] - mq) < 1e-10
        assert abs(g[i] - mg) < 1e-12


def test_encode_layout_matches_table_1(O):
    rec = synth.make_records(37, seed=5)
    for pad in (1.0, 0.0):
        for mode in (O.ENC_CHEAP, O.ENC_EXACT):
            enc = O.encode(rec, mode, pad)
            assert enc.shape == (37, 64)
            for r in range(37):
                x = rec[r].astype(np.float64)
                for j in range(3):
                    for d in range(12):
                        assert enc[r, 12 * j + d] == O.freq_feature(x[j], d, mode)
                assert np.array_equal(enc[r, 36:40], O.oneblob(x[3], 4, mode))
                assert np.array_equal(enc[r, 40:44], O.oneblob(x[4], 4, mode))
                assert np.array_equal(enc[r, 44:48], O.oneblob(x[5], 4, mode))
                assert np.array_equal(enc[r, 48:52], O.oneblob(x[6], 4, mode))
                assert np.allclose(enc[r, 52:56], O.oneblob(1.0 - math.exp(-x[7]), 4, mode), atol=1e-15)
                assert np.array_equal(enc[r, 56:62], x[8:14])
                assert np.all(enc[r, 62:64] == pad)


def test_encoding_dimension_count():
    # Table 1: 3x12 + 2x4 + 2x4 + 4 + 3 + 3 = 62, padded to 64 (Sec. 3.6).
    assert 3 * 12 + 2 * 4 + 2 * 4 + 4 + 3 + 3 == 62


def test_encode_value_ranges(O):
    rec = synth.make_records(2000, seed=6)
    enc = O.encode(rec, O.ENC_CHEAP, 1.0)
    assert np.all(np.abs(enc[:, :36]) <= 1.0)
    assert np.all(enc[:, 36:56] >= -1e-15) and np.all(enc[:, 36:56] <= 1.0)
    # the two sphere coordinates and roughness stay inside [0, 1]
    assert np.all((rec[:, 3:8] >= 0) & (rec[:, 3:8] <= 1))

"""Pins of the oracle's quantiser and dequantiser (convention C11) against the
HEVC step-size law Qstep = 2^((qP-4)/6), the published levelScale, and the
dead-zone round-trip bound."""
import numpy as np
import pytest

from conftest import read_golden

B = 10


def coeff_step(qp, L):
    """Quantisation step in the coefficient domain: Qstep * 2^(15 - B - log2 N)."""
    qP = qp + 6 * (B - 8)
    return 2.0 ** ((qP - 4) / 6.0) * 2.0 ** (15 - B - L)


@pytest.mark.parametrize("L", [2, 3, 4, 5])
@pytest.mark.parametrize("qp", [10, 17, 22, 27, 32, 37, 45])
def test_dequant_unit_level_is_the_step(xvo, qp, L):
    s = coeff_step(qp, L)
    big = max(1, min(64, int(30000 / s)))  # stay below the int16 clip
    got = int(xvo.dequant(big, qp, L)) / big
    assert abs(got / s - 1) < 0.01 + 1.0 / (big * s)


def test_dequant_follows_level_scale_table(xvo):
    """d(level) for qP % 6 = r grows like levelScale[r]; one period apart doubles."""
    ls = read_golden("hevc_level_scale.txt")["LEVELSCALE"][0]
    L = 5
    base = 24 - 12  # qP = 24
    vals = [int(xvo.dequant(100, base + r, L)) for r in range(6)]
    for r in range(6):
        assert abs(vals[r] / vals[0] - ls[r] / ls[0]) < 2e-3
    assert int(xvo.dequant(100, base + 6, L)) == 2 * vals[0]


@pytest.mark.parametrize("L", [2, 3, 4, 5])
@pytest.mark.parametrize("qp", [-12, 0, 22, 27, 32, 51])
def test_quant_round_trip_bound_and_symmetry(xvo, qp, L):
    s = coeff_step(qp, L)
    c = np.unique(np.concatenate([np.arange(-2000, 2001, 7), np.array([0, 1, -1, 32767, -32767])]))
    c = c[np.abs(c) < 2 ** 15]
    c = c[np.abs(c) < 32000 * s]  # keep clear of the asymmetric int16 level clip
    lv = xvo.quant(c, qp, L)
    assert np.array_equal(xvo.quant(-c, qp, L), -lv)
    assert np.all(np.diff(lv) >= 0)
    d = xvo.dequant(lv, qp, L)
    # dead zone with rounding offset 85/512: error at most (1 - 85/512) of a
    # step; the integer scales realise the step to within 1%
    assert np.abs(d - c).max() <= (1 - 85 / 512) * s * 1.01 + 2
    # magnitudes below the dead zone quantise to zero
    small = c[np.abs(c) < 0.83 * s * 0.999]
    assert not xvo.quant(small, qp, L).any()


def test_level_clipped_to_int16(xvo):
    assert int(xvo.quant(32767, -12, 5)) <= 32767
    assert int(xvo.dequant(32767, 51, 2)) == 32767
    assert int(xvo.dequant(-32768, 51, 2)) == -32768

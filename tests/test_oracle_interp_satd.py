"""Pins of the oracle's quarter-sample interpolation (C8) and SATD (C9)."""
import numpy as np
import pytest
import scipy.linalg

from conftest import read_golden

ALL_FRAC = [(fx, fy) for fy in range(4) for fx in range(4)]


@pytest.mark.parametrize("fx,fy", ALL_FRAC)
def test_constant_plane_is_fixed(xvo, fx, fy):
    ref = np.full((24, 24), 777, np.uint16)
    out = xvo.interp_block(ref, 4, 4, 8, 8, 4 * 1 + fx, 4 * -2 + fy)
    assert np.all(out == 777)


def test_full_pel_is_a_shifted_copy(xvo):
    rng = np.random.default_rng(0)
    ref = rng.integers(0, 1024, (32, 32)).astype(np.uint16)
    out = xvo.interp_block(ref, 8, 8, 8, 8, 4 * 3, 4 * -2)
    assert np.array_equal(out, ref[6:14, 11:19])


def test_impulse_recovers_published_taps(xvo):
    """An impulse of 64 on a 512 background returns 512 + f[i] exactly."""
    taps = read_golden("hevc_luma_filter.txt")
    names = {1: "QUARTER", 2: "HALF", 3: "THREEQUARTER"}
    ref = np.full((16, 32), 512, np.uint16)
    ref[8, 16] = 512 + 64
    for frac, name in names.items():
        f = taps[name][0]
        # horizontal: output x uses taps at x + i - 3, i = 0..7
        out = xvo.interp_block(ref, 0, 8, 32, 1, frac, 0)[0]
        got = [int(out[16 - (i - 3)]) - 512 for i in range(8)]
        assert got == f
        refv = np.ascontiguousarray(ref.T)
        out = xvo.interp_block(refv, 8, 0, 1, 32, 0, frac)[:, 0]
        got = [int(out[16 - (i - 3)]) - 512 for i in range(8)]
        assert got == f


def test_half_pel_of_a_ramp_is_exact(xvo):
    """The half-sample filter has first moment 1/2: on v = 4x + 4y + 100 the
    half positions give exactly v + 2 (one axis) and v + 4 (both)."""
    yy, xx = np.mgrid[0:40, 0:40]
    ref = (4 * xx + 4 * yy + 100).astype(np.uint16)
    base = ref[10:18, 10:18].astype(int)
    assert np.array_equal(xvo.interp_block(ref, 10, 10, 8, 8, 2, 0).astype(int), base + 2)
    assert np.array_equal(xvo.interp_block(ref, 10, 10, 8, 8, 0, 2).astype(int), base + 2)
    assert np.array_equal(xvo.interp_block(ref, 10, 10, 8, 8, 2, 2).astype(int), base + 4)


def test_borders_clamp(xvo):
    rng = np.random.default_rng(3)
    ref = rng.integers(0, 1024, (16, 16)).astype(np.uint16)
    padded = np.pad(ref, 40, mode="edge")
    for mvx, mvy in [(-80, -80), (-37, 13), (55, -61), (3, 90)]:
        a = xvo.interp_block(ref, 0, 0, 16, 16, mvx, mvy)
        b = xvo.interp_block(padded, 40, 40, 16, 16, mvx, mvy)
        assert np.array_equal(a, b)


def test_hadamard_matches_scipy(xvo):
    H = scipy.linalg.hadamard(8)
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.integers(-1023, 1024, (8, 8))
        assert np.array_equal(xvo.hadamard8(d), H @ d @ H.T)


def test_hadamard_parseval(xvo):
    rng = np.random.default_rng(2)
    d = rng.integers(-500, 500, (8, 8))
    h = xvo.hadamard8(d).astype(np.int64)
    assert (h ** 2).sum() == 64 * (d.astype(np.int64) ** 2).sum()


def test_satd_closed_forms(xvo):
    for c in (-9, 0, 1, 300):
        assert xvo.satd(np.full((8, 8), c)) == 16 * abs(c)
        assert xvo.satd(np.full((16, 16), c)) == 4 * 16 * abs(c)
        assert xvo.satd(np.full((4, 4), c)) == 8 * abs(c)
    for e in (-5, 7):
        d = np.zeros((8, 8), np.int32)
        d[3, 5] = e
        assert xvo.satd(d) == 16 * abs(e)


def test_satd_against_scipy_hadamard(xvo):
    H = scipy.linalg.hadamard(8)
    rng = np.random.default_rng(4)
    d = rng.integers(-1023, 1024, (16, 24))
    want = 0
    for by in range(0, 16, 8):
        for bx in range(0, 24, 8):
            s = int(np.abs(H @ d[by:by + 8, bx:bx + 8] @ H.T).sum())
            want += (s + 2) >> 2
    assert xvo.satd(d) == want

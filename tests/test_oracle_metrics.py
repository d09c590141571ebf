"""The oracle's SSIM (Wang et al. 2004) and spectral angle (Kruse et al.
1993), pinned by closed forms, invariants and exact counts."""
import math

import numpy as np
import pytest

import oracle


def test_ssim_window_is_the_normalised_gaussian():
    w = oracle.ssim_window()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w[::-1], rtol=0, atol=0)
    # ratios of a Gaussian with sigma 1.5: w[k] / w[5] = exp(-(k-5)^2 / 4.5)
    for k in range(11):
        assert math.isclose(w[k] / w[5], math.exp(-((k - 5) ** 2) / 4.5), rel_tol=1e-14)


def test_ssim_identical_images_is_one_and_counts_valid_windows():
    X = np.random.default_rng(1).uniform(-3, 8, (23, 31))
    s, n = oracle.ssim_image(X, X, 11.0)
    assert n == (23 - 10) * (31 - 10)
    assert abs(s / n - 1.0) < 1e-14


@pytest.mark.parametrize("a,b,L", [(0.2, 0.7, 1.0), (5.0, 5.5, 10.0), (-3.0, 1.0, 4.0), (100.0, 0.0, 250.0)])
def test_ssim_constant_images_closed_form(a, b, L):
    """No variance anywhere: only the luminance term is left,
    (2ab + C1) / (a^2 + b^2 + C1) with C1 = (0.01 L)^2."""
    X = np.full((14, 12), a)
    Y = np.full((14, 12), b)
    s, n = oracle.ssim_image(X, Y, L)
    C1 = (0.01 * L) ** 2
    assert n == 4 * 2
    assert math.isclose(s / n, (2 * a * b + C1) / (a * a + b * b + C1), rel_tol=1e-12)


def test_ssim_symmetry_and_scale_invariance():
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (19, 26))
    Y = np.clip(X + rng.normal(0, 0.1, X.shape), 0, 1)
    s1, n1 = oracle.ssim_image(X, Y, 1.0)
    s2, _ = oracle.ssim_image(Y, X, 1.0)
    assert abs(s1 - s2) < 1e-12
    # scale invariance (the data range scales with the data; an offset would
    # change the luminance term, which compares absolute means)
    s3, _ = oracle.ssim_image(40 * X, 40 * Y, 40.0)
    assert abs(s1 / n1 - s3 / n1) < 1e-12
    s4, _ = oracle.ssim_image(X + 5, Y + 5, 1.0)
    assert s4 / n1 > s1 / n1  # equal shift: closer luminance ratio
    assert 0 < s1 / n1 < 1


def test_ssim_decreases_with_noise():
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (30, 30))
    E = rng.normal(0, 1, X.shape)
    vals = [oracle.ssim_image(X, X + k * E, 1.0)[0] for k in (0.0, 0.01, 0.05, 0.2, 1.0)]
    assert all(a > b for a, b in zip(vals, vals[1:]))


def test_ssim_skips_windows_with_a_non_finite_sample():
    X = np.random.default_rng(4).uniform(0, 1, (16, 16))
    X[0, 0] = np.nan  # only the window whose top-left sample it is
    _, n = oracle.ssim_image(X, np.nan_to_num(X), 1.0)
    assert n == 6 * 6 - 1
    X[8, 8] = np.inf  # inside every window
    _, n = oracle.ssim_image(X, np.nan_to_num(X), 1.0)
    assert n == 0


def grid_cube(rng, bands=5, T=2, H=16, W=18):
    """Integers in [0, 1023] with min/max fixed at (0, 1023): x^ = q exactly."""
    cube = rng.integers(0, 1024, (bands, T, H, W)).astype(np.uint16)
    mm = np.array([[0.0, 1023.0]] * bands)
    return cube, mm


def planes_of(cube, ctu=8):
    mm = np.array([[0.0, 1023.0]] * cube.shape[0])
    return oracle.quantize_pack(cube, ctu, mm)


def test_ssim_cube_band_mapping():
    """Band b is group b/3, channel b%3: a perfect reconstruction gives 1 in
    every band; disturbing one (group, channel) lowers only that band."""
    rng = np.random.default_rng(5)
    cube, mm = grid_cube(rng)
    planes = planes_of(cube)
    assert np.allclose(oracle.ssim(cube, planes, mm), 1.0, rtol=0, atol=1e-14)
    rec = planes.copy()
    rec[1, :, 0] = np.clip(rec[1, :, 0].astype(int) + rng.integers(-40, 41, rec[1, :, 0].shape), 0, 1023)
    s = oracle.ssim(cube, rec, mm)  # group 1, channel 0 = band 3
    assert np.all(np.abs(s[[0, 1, 2, 4]] - 1.0) < 1e-14) and s[3] < 0.999


def sa_case(spectra_s, spectra_r, lo=0.0, hi=1023.0):
    """One frame, one row: pixel k has spectrum spectra_s[k] (original) and
    levels spectra_r[k] (reconstruction)."""
    s = np.asarray(spectra_s, np.float32).T[:, None, None, :]     # [bands, 1, 1, npix]
    r = np.asarray(spectra_r, np.int64)
    bands, npix = s.shape[0], s.shape[3]
    mm = np.array([[lo, hi]] * bands)
    G = (bands + 2) // 3
    rec = np.zeros((G, 1, 3, 8, 8 * ((npix + 7) // 8)), np.uint16)
    for b in range(bands):
        rec[b // 3, 0, b % 3, 0, :npix] = r[:, b]
    return s, rec, mm


@pytest.mark.parametrize("s,r,want", [
    ([[3, 4]], [[3, 4]], 0.0),
    ([[3, 4]], [[6, 8]], 0.0),                                  # scale invariance
    ([[1, 0]], [[0, 1]], math.pi / 2),
    ([[3, 4]], [[4, 3]], math.acos(24 / 25)),
    ([[1, 2, 2]], [[2, 1, 2]], math.acos(8 / 9)),
    ([[3, 4], [1, 0]], [[4, 3], [0, 1]], (math.acos(24 / 25) + math.pi / 2) / 2),
    # a small angle, where acos of the cosine would lose about 1e-8 rad
    ([[1000, 1000]], [[1000, 1001]], math.atan2(1000, 1000 * 1000 + 1000 * 1001)),
])
def test_sa_closed_forms(s, r, want):
    src, rec, mm = sa_case(s, r)
    v, n = oracle.sa(src, rec, mm)
    assert n == len(s)
    assert math.isclose(v, want, rel_tol=1e-12, abs_tol=1e-12)


def test_sa_opposite_and_skipped_pixels():
    # x^ = q - 512 (min -512, max 511): level 507 is -5, so (5, 0) against (-5, 0) is pi
    src, rec, mm = sa_case([[5, 0], [0, 0], [1, 1]], [[507, 512], [512, 512], [513, 513]], lo=-512.0, hi=511.0)
    v, n = oracle.sa(src, rec, mm)
    assert n == 2  # the zero spectrum is skipped
    assert math.isclose(v, math.pi / 2, rel_tol=1e-12)  # mean of pi and 0
    src2 = src.copy()
    src2[0, 0, 0, 2] = np.nan
    v2, n2 = oracle.sa(src2, rec, mm)
    assert n2 == 1 and math.isclose(v2, math.pi, rel_tol=1e-12)

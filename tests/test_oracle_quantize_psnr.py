"""Pins of min-max quantisation and packing (C1-C3, paper Sec. 2.1) and of
PSNR / bpppb (C13-C14, paper Sec. 2.3)."""
import os

import numpy as np
import pytest

from conftest import GOLDEN


def test_grouping_matches_paper_example(xvo):
    # fixture line "4 : 0 1 2 | 3 3 3" -> bands and the band held by each slot
    with open(os.path.join(GOLDEN, "band_grouping.txt")) as f:
        line = [ln for ln in f if ln.strip() and not ln.startswith("#")][0]
    bands, rest = line.split(":")
    want = [[int(v) for v in grp.split()] for grp in rest.split("|")]
    assert xvo.group_bands(int(bands)) == want


@pytest.mark.parametrize("bands,want", [
    (3, [[0, 1, 2]]),
    (6, [[0, 1, 2], [3, 4, 5]]),
    (10, [[0, 1, 2], [3, 4, 5], [6, 7, 8], [9, 9, 9]]),
    (1, [[0, 0, 0]]),
    (5, [[0, 1, 2], [3, 4, 4]]),
])
def test_grouping_rule(xvo, bands, want):
    assert xvo.group_bands(bands) == want


def test_endpoints_monotone_and_exact_toy(xvo):
    x = np.arange(1024, dtype=np.float32)[None, None, None, :]  # min 0, max 1023
    mm, _ = xvo.minmax(x)
    assert mm.tolist() == [[0.0, 1023.0]]
    q = xvo.quantize_pack(x, 8, mm)
    assert np.array_equal(q[0, 0, 0, 0, :1024], np.arange(1024))
    rng = np.random.default_rng(0)
    y = np.sort(rng.uniform(-3.5, 7.25, 5000)).astype(np.float32)[None, None, None, :]
    mm, _ = xvo.minmax(y)
    qy = xvo.quantize_pack(y, 8, mm)[0, 0, 0, 0, :5000].astype(int)
    assert qy[0] == 0 and qy[-1] == 1023 and np.all(np.diff(qy) >= 0)


def test_u16_equals_f32_for_same_values(xvo):
    rng = np.random.default_rng(1)
    u = rng.integers(0, 10001, (4, 3, 20, 24)).astype(np.uint16)
    f = u.astype(np.float32)
    mu, _ = xvo.minmax(u)
    mf, _ = xvo.minmax(f)
    assert np.array_equal(mu, mf)
    assert np.array_equal(xvo.quantize_pack(u, 16, mu), xvo.quantize_pack(f, 16, mf))


def test_nan_and_constant_band(xvo):
    x = np.full((2, 2, 8, 8), 0.25, np.float32)
    x[0, 1, 3, 3] = np.nan
    x[0, 0, 0, 0] = 1.0
    mm, nn = xvo.minmax(x)
    assert nn.tolist() == [1, 0]
    assert mm.tolist() == [[0.25, 1.0], [0.25, 0.25]]
    q = xvo.quantize_pack(x, 8, mm)
    assert q[0, 1, 0, 3, 3] == 0      # NaN -> 0
    assert q[0, 0, 0, 0, 0] == 1023
    assert not q[0, :, 1].any()        # constant band -> all 0


def test_padding_replicates_edges_and_pad_band(xvo):
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (4, 2, 13, 21)).astype(np.float32)
    mm, _ = xvo.minmax(x)
    q = xvo.quantize_pack(x, 8, mm)
    assert q.shape == (2, 2, 3, 16, 24)
    assert np.array_equal(q[:, :, :, 13:, :], np.repeat(q[:, :, :, 12:13, :], 3, axis=3))
    assert np.array_equal(q[:, :, :, :, 21:], np.repeat(q[:, :, :, :, 20:21], 3, axis=4))
    assert np.array_equal(q[1, :, 1], q[1, :, 0]) and np.array_equal(q[1, :, 2], q[1, :, 0])


def test_psnr_planted_errors(xvo):
    """Toy cube x = q (min 0, max 1023, step 1): recon = q + e on k pixels of band
    b gives SSE10 = k e^2 and PSNR = 10 log10(1023^2 THW / (k e^2))."""
    rng = np.random.default_rng(3)
    bands, T, H, W = 4, 3, 10, 12
    q = rng.integers(1, 1023, (bands, T, H, W))
    q[:, 0, 0, 0] = 0
    q[:, 0, 0, 1] = 1023
    x = q.astype(np.float32)
    mm, _ = xvo.minmax(x)
    planes = xvo.quantize_pack(x, 8, mm)
    recon = planes.copy()
    e, k, b = 3, 7, 1
    ys, xs = rng.choice(H, k), rng.choice(W, k, replace=False)
    for i in range(k):
        recon[b // 3, 1, b % 3, ys[i], xs[i]] += e
    r = xvo.psnr(x, planes, recon, mm)
    n = T * H * W
    assert r["sse10_band"].tolist() == [0, k * e * e, 0, 0]
    assert r["psnr_band"][1] == pytest.approx(10 * np.log10(1023.0 ** 2 * n / (k * e * e)), rel=1e-12)
    assert r["psnr10_band"][1] == pytest.approx(10 * np.log10(1023.0 ** 2 * n / (k * e * e)), rel=1e-12)
    assert np.isinf(r["psnr_band"][0]) and np.isinf(r["psnr_band"][3])


def test_psnr_peak_is_band_max_and_negative_fallback(xvo):
    bands, T, H, W = 2, 1, 4, 4
    x = np.zeros((bands, T, H, W), np.float32)
    x[0] = np.linspace(2, 4, 16).reshape(4, 4)
    x[1] = np.linspace(-6, -2, 16).reshape(4, 4)
    mm, _ = xvo.minmax(x)
    planes = xvo.quantize_pack(x, 4, mm)
    recon = planes.copy()
    recon[0, 0, 0, 1, 1] += 1
    recon[0, 0, 1, 2, 2] += 1
    r = xvo.psnr(x, planes, recon, mm)
    # one pixel off by one 10-bit step; the float error of the others is the quantiser's own
    for b, peak in ((0, 4.0), (1, 4.0)):  # band 1: max <= 0 so the peak is max - min = 4
        assert r["psnr_band"][b] == pytest.approx(10 * np.log10(peak ** 2 / r["mse_band"][b]), rel=1e-12)

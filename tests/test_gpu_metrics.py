"""GPU SSIM and spectral angle against the oracle's double definitions.

Tolerances, from the FP32 arithmetic of the kernels: SSIM runs on values
normalised to [0, 1] (relative rounding u = 2^-24 per operation); a window's
means carry about 121 u of error and its variances, built from deviations
from the local mean, a relative 2 x 121 u, so each window's index is within
a few 1e-5 and the band means, averaging many windows, within 2e-5.  The
spectral angle is an atan2 of FP32 wedge and dot products of at most 16
terms: a relative error of a few 1e-6 per pixel, 1e-5 on the mean."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_util import to_dev
from paper_2506_19656_gb300 import synth

pytestmark = pytest.mark.gpu

SSIM_TOL = 2e-5
SA_RTOL = 1e-5


@pytest.fixture(scope="module")
def xv():
    from paper_2506_19656_gb300 import build, xv as _xv
    build.build()
    oracle.build()
    return _xv


@pytest.fixture(scope="module")
def ctx(xv):
    c = xv.Context(0)
    yield c
    c.close()


def noisy_recon(rng, planes, amp):
    return np.clip(planes.astype(int) + rng.integers(-amp, amp + 1, planes.shape), 0, 1023).astype(np.uint16)


@pytest.mark.parametrize("dtype,shape,amp", [("f32", (5, 3, 40, 57), 6), ("f32", (2, 2, 11, 11), 2),
                                             ("u16", (4, 2, 70, 45), 20), ("f32", (16, 1, 33, 35), 1),
                                             ("offset", (3, 2, 30, 40), 4)])
def test_ssim_and_sa_random(xv, ctx, dtype, shape, amp):
    """Random cubes, including bands with a large offset and a small range
    (the luminance term compares absolute means)."""
    rng = np.random.default_rng(sum(shape) + amp)
    if dtype == "offset":
        cube = (np.array([5.0, 300.0, 1e4])[:, None, None, None] + rng.uniform(0, 1, shape)).astype(np.float32)
    elif dtype == "f32":
        cube = (rng.uniform(-2, 5, shape) + np.linspace(0, 3, shape[-1])).astype(np.float32)
    else:
        cube = rng.integers(0, 10001, shape).astype(np.uint16)
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, 8, mm)
    recon = noisy_recon(rng, planes, amp)
    want = oracle.ssim(cube, recon, mm)
    got = xv.xv_ssim(ctx, to_dev(cube), to_dev(recon), to_dev(mm))
    assert np.allclose(got["ssim_band"], want, rtol=0, atol=SSIM_TOL), (got["ssim_band"], want)
    assert abs(got["ssim_mean"] - want.mean()) <= SSIM_TOL
    wa, wn = oracle.sa(cube, recon, mm)
    ga, gn = xv.xv_sa(ctx, to_dev(cube), to_dev(recon), to_dev(mm))
    assert gn == wn
    assert math.isclose(ga, wa, rel_tol=SA_RTOL), (ga, wa)


def test_metrics_skip_non_finite_and_small_images(xv, ctx):
    rng = np.random.default_rng(9)
    cube = rng.uniform(0, 1, (3, 2, 24, 30)).astype(np.float32)
    cube[1, 0, 5, 7] = np.nan
    cube[2, 1, 0, 0] = np.inf
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, 8, mm)
    recon = noisy_recon(rng, planes, 3)
    want = oracle.ssim(cube, recon, mm)
    got = xv.xv_ssim(ctx, to_dev(cube), to_dev(recon), to_dev(mm))
    assert np.allclose(got["ssim_band"], want, rtol=0, atol=SSIM_TOL)
    wa, wn = oracle.sa(cube, recon, mm)
    ga, gn = xv.xv_sa(ctx, to_dev(cube), to_dev(recon), to_dev(mm))
    assert gn == wn == 2 * 24 * 30 - 2 and math.isclose(ga, wa, rel_tol=SA_RTOL)
    small = cube[:, :, :10, :30].copy()  # no 11 x 11 window fits
    g2 = xv.xv_ssim(ctx, to_dev(small), to_dev(recon), to_dev(mm))
    assert all(math.isnan(v) for v in g2["ssim_band"])


def test_metrics_on_an_encoded_cube(xv, ctx):
    """The tiny workload encoded on the GPU at two QPs: SSIM and SA of the
    GPU reconstruction against the oracle's, and quality ordered by QP."""
    c = synth.WORKLOADS["tiny"]
    cube = synth.make_cube("tiny")
    res = []
    for qp in (22, 37):
        p = xv.xv_params_init(c.ctu, c.R, c.tu_mask, qp)
        buf = xv.alloc_cube_buffers(*cube.shape, p)
        src = to_dev(cube)
        job = xv.make_job(src, p, buf["planes"], buf["recon"], minmax=buf["minmax"], mv=buf["mv"], cost=buf["cost"],
                          levels=buf["levels"], tu_log2=buf["tu_log2"], bits=buf["bits"])
        xv.xv_encode_batch(ctx, [job])
        recon = buf["recon"].view(torch.int16).cpu().numpy().view(np.uint16)
        mm = buf["minmax"].cpu().numpy()
        want = oracle.ssim(cube, recon, mm)
        got = xv.xv_ssim(ctx, src, buf["recon"], buf["minmax"])
        assert np.allclose(got["ssim_band"], want, rtol=0, atol=SSIM_TOL)
        wa, _ = oracle.sa(cube, recon, mm)
        ga, _ = xv.xv_sa(ctx, src, buf["recon"], buf["minmax"])
        assert math.isclose(ga, wa, rel_tol=SA_RTOL)
        res.append((got["ssim_mean"], ga))
    assert res[0][0] > res[1][0] and res[0][1] < res[1][1]


SSIM_WINDOW_TOL = 5e-5  # one window's index: a few 1e-5 (see the module docstring)


def test_ssim_per_window(xv, ctx):
    """One 11 x 11 window per band (T = 1, H = W = 11): the band value is that
    single window's SSIM, so errors cannot average out across windows.  40
    windows over random cubes of several amplitudes, offsets and ranges."""
    rng = np.random.default_rng(77)
    n = 0
    for trial in range(10):
        bands = int(rng.integers(1, 6))
        lo = rng.uniform(-50, 50, (bands, 1, 1, 1))
        scale = rng.uniform(0.01, 100, (bands, 1, 1, 1))
        cube = (lo + scale * rng.uniform(0, 1, (bands, 1, 11, 11))).astype(np.float32)
        mm, _ = oracle.minmax(cube)
        planes = oracle.quantize_pack(cube, 8, mm)
        recon = noisy_recon(rng, planes, int(rng.integers(1, 60)))
        want = oracle.ssim(cube, recon, mm)
        got = xv.xv_ssim(ctx, to_dev(cube), to_dev(recon), to_dev(mm))
        for b in range(bands):
            assert abs(got["ssim_band"][b] - want[b]) <= SSIM_WINDOW_TOL, (trial, b, got["ssim_band"][b], want[b])
            n += 1
    assert n >= 20


def test_spectral_angle_per_pixel(xv, ctx):
    """One pixel per call (T = H = W = 1): the mean angle is that pixel's angle,
    checked at the per-pixel relative error of a few 1e-6 (1e-5 here), for
    spectra of 2 to 16 bands and angles from small to large."""
    rng = np.random.default_rng(78)
    for trial in range(24):
        bands = int(rng.integers(2, 17))
        cube = rng.uniform(0.1, 1, (bands, 1, 1, 1)).astype(np.float32)
        mm = np.stack([cube.reshape(bands) - rng.uniform(0.05, 0.5, bands),
                       cube.reshape(bands) + rng.uniform(0.05, 0.5, bands)], axis=1)
        planes = oracle.quantize_pack(cube, 8, mm)
        recon = noisy_recon(rng, planes, int(rng.integers(1, 200)))
        wa, wn = oracle.sa(cube, recon, mm)
        ga, gn = xv.xv_sa(ctx, to_dev(cube), to_dev(recon), to_dev(mm))
        assert gn == wn == 1
        assert math.isclose(ga, wa, rel_tol=SA_RTOL, abs_tol=1e-9), (trial, ga, wa)

"""xv_psnr_noalloc: the PSNR entry point for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Checked
through the C ABI against xv_psnr, on two calls in a row with different
inputs, so a second call that read anything the first left behind would fail.
This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _case(seed, bands, T, H, W, ctu, dtype):
    import oracle
    rng = np.random.default_rng(seed)
    if dtype == "f32":
        cube = rng.uniform(-3, 7, (bands, T, H, W)).astype(np.float32)
        cube[0, 0, 1, 1] = np.nan
    else:
        cube = rng.integers(0, 10001, (bands, T, H, W)).astype(np.uint16)
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, ctu, mm)
    recon = np.clip(planes.astype(int) + rng.integers(-4, 5, planes.shape), 0, 1023).astype(np.uint16)
    want = oracle.psnr(cube, planes, recon, mm)
    return (to_dev(cube), to_dev(planes), to_dev(recon), to_dev(mm)), want


def _same(a, b):
    for x, y in zip(a["psnr_band"], b["psnr_band"]):
        assert (np.isinf(x) and np.isinf(y)) or abs(x - y) <= 1e-9 * abs(y)
    assert a["sse10_band"] == b["sse10_band"]
    for x, y in zip(a["mse_band"], b["mse_band"]):
        assert abs(x - y) <= 1e-12 * max(abs(y), 1e-300)


def test_noalloc_psnr_matches_xv_psnr_twice():
    import oracle
    from paper_2506_19656_gb300 import build, xv
    build.build()
    oracle.build()
    ctx = xv.Context(0)
    try:
        first = _case(1, 10, 4, 70, 90, 16, "f32")    # 10 bands
        second = _case(2, 4, 3, 33, 41, 8, "u16")     # fewer bands, other sizes
        # 786,432 samples in each of two bands: the partial sums per band
        # reach their maximum of 256 blocks (each block then takes more
        # samples; with more bands one wave of resident blocks caps them lower)
        third = _case(3, 2, 3, 512, 512, 32, "f32")
        for args, oracle_want in (first, second, third):
            want = xv.xv_psnr(ctx, *args)
            got = xv.xv_psnr_noalloc(*args)
            torch.cuda.synchronize()
            _same(got, want)
            # and against the oracle's definition itself
            for x, y in zip(got["psnr_band"], oracle_want["psnr_band"]):
                assert (np.isinf(x) and np.isinf(y)) or abs(x - y) <= 1e-9 * abs(y)
            assert got["sse10_band"] == [int(v) for v in oracle_want["sse10_band"]]
    finally:
        ctx.close()


def test_noalloc_rejects_too_many_bands():
    from paper_2506_19656_gb300 import build, xv
    build.build()
    src = torch.zeros((17, 1, 8, 8), dtype=torch.float32, device="cuda")
    planes = torch.zeros((6, 1, 3, 8, 8), dtype=torch.uint16, device="cuda")
    mm = torch.zeros((17, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(xv.XvError) as e:
        xv.xv_psnr_noalloc(src, planes, planes, mm)
    assert e.value.status == xv.XV_EINVAL

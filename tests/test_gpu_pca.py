"""GPU PCA over bands against the oracle: the fit, the projection and its
inverse, and PCA -> encode -> decode -> inverse on a small cube.

Tolerances: the fit's covariance is accumulated in double from centred
double values (the oracle's definition, summed in another order: about
1e-15 relative), so eigenvalues agree to 1e-9 and eigenvectors to
1e-15 / (relative gap) -- 1e-8 even for the 4^-9 variance of the 10-band
case, checked at 1e-6.  Projection and inverse are FP32 sums of at most 16
products: 1e-5 of the data's scale."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


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


def mixed_cube(seed, bands, shape, dtype):
    """Bands mixed from sources with well-separated variances, plus an offset."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    sd = 2.0 ** -np.arange(bands)  # variances 4^-k
    Q, _ = np.linalg.qr(rng.normal(0, 1, (bands, bands)))
    x = Q @ (sd[:, None] * rng.normal(0, 1, (bands, n))) + rng.uniform(-1, 3, (bands, 1))
    x = x.reshape((bands,) + shape)
    if dtype == "u16":
        return np.clip(np.round(3000 + 400 * x), 0, 65535).astype(np.uint16)
    return x.astype(np.float32)


@pytest.mark.parametrize("bands,shape,dtype", [(5, (3, 40, 50), "f32"), (10, (2, 64, 64), "f32"),
                                               (16, (1, 48, 40), "f32"), (4, (2, 50, 60), "u16")])
def test_pca_fit_project_inverse(xv, ctx, bands, shape, dtype):
    cube = mixed_cube(bands * 11 + len(dtype), bands, shape, dtype)
    wm, wc, wv = oracle.pca_fit(cube)
    d = to_dev(cube)
    gm, gc, gv = xv.xv_pca_fit(ctx, d)
    assert np.allclose(gm, wm, rtol=1e-9, atol=1e-9 * np.abs(wm).max())
    assert np.allclose(gv, wv, rtol=1e-9, atol=1e-12 * wv[0])
    assert np.allclose(gc, wc, atol=1e-6)
    npc = max(1, bands - 1)
    z = torch.empty((npc,) + shape, dtype=torch.float32, device="cuda")
    xv.xv_pca_project(ctx, d, gm, gc, npc, z)
    wz = oracle.pca_project(cube, gm, gc, npc)
    scale = float(np.abs(cube.astype(np.float64) - gm[:, None, None, None]).max())
    assert np.allclose(to_np(z), wz, rtol=0, atol=1e-5 * scale)
    back = torch.empty(cube.shape, dtype=torch.float32, device="cuda")
    xv.xv_pca_inverse(ctx, z, gm, gc, back)
    wb = oracle.pca_inverse(to_np(z), gm, gc)
    assert np.allclose(to_np(back), wb, rtol=0, atol=1e-5 * (scale + np.abs(gm).max()))
    # all components: the GPU round trip gives the cube back
    zf = torch.empty(cube.shape, dtype=torch.float32, device="cuda")
    xv.xv_pca_project(ctx, d, gm, gc, bands, zf)
    xv.xv_pca_inverse(ctx, zf, gm, gc, back)
    assert np.allclose(to_np(back), cube.astype(np.float32), rtol=0, atol=2e-5 * (scale + np.abs(gm).max()))


def test_pca_then_encode_decode_inverse(xv, ctx):
    """Nine of ten components packed into three videos (the paper's "PCA - 9
    bands" test), encoded and decoded on the GPU, back to ten bands: the
    encode is bit-exact with the oracle on the GPU's components, and the
    inverse matches the oracle's on the decoded reconstruction."""
    cube = mixed_cube(7, 10, (4, 48, 64), "f32")
    d = to_dev(cube)
    gm, gc, _ = xv.xv_pca_fit(ctx, d)
    z = torch.empty((9, 4, 48, 64), dtype=torch.float32, device="cuda")
    xv.xv_pca_project(ctx, d, gm, gc, 9, z)
    p = xv.xv_params_init(16, 8, 0b11100, 27)
    buf = xv.alloc_cube_buffers(9, 4, 48, 64, p)
    job = xv.make_job(z, p, buf["planes"], buf["recon"], minmax=buf["minmax"], mv=buf["mv"], cost=buf["cost"],
                      levels=buf["levels"], tu_log2=buf["tu_log2"], bits=buf["bits"])
    xv.xv_encode_batch(ctx, [job])
    want = oracle.encode_cube(to_np(z), 16, 8, 0b11100, 27)
    assert np.array_equal(to_np(buf["recon"]), want["recon"])
    out = torch.empty((9, 4, 48, 64), dtype=torch.float32, device="cuda")
    dj = xv.make_djob(p, buf["levels"], buf["mv"], buf["tu_log2"], torch.empty_like(buf["recon"]),
                      minmax=buf["minmax"], dst=out, bands=9, H=48, W=64)
    xv.xv_decode_batch(ctx, [dj])
    assert np.array_equal(to_np(out), oracle.unpack(want["recon"], want["mm"], 9, 48, 64))
    back = torch.empty(cube.shape, dtype=torch.float32, device="cuda")
    xv.xv_pca_inverse(ctx, out, gm, gc, back)
    wb = oracle.pca_inverse(to_np(out), gm, gc)
    assert np.allclose(to_np(back), wb, rtol=0, atol=1e-5 * float(np.abs(wb).max()))


def test_pca_all_bands_one_qp_per_group(xv, ctx):
    """The paper's "PCA - all bands" test (Sec. 3, Tab. 5): all ten components
    of a DeepExtremeCubes-shaped prefix, packed three to a group, every group
    at its own QP (later components at lower quality) through
    xv_split_groups + one xv_encode_batch.  Each group equals the oracle's
    encode of its three components at that group's QP, and a group equals
    the whole-cube encode's group at the same QP (the split changes nothing
    but the QP)."""
    from paper_2506_19656_gb300 import synth
    cfg = synth.WORKLOADS["deepextremecubes"]
    cube = synth.make_cube("deepextremecubes", T=4)
    src = to_dev(cube)
    mean, comps, _ = xv.xv_pca_fit(ctx, src)
    z = torch.empty(cube.shape, dtype=torch.float32, device="cuda")
    xv.xv_pca_project(ctx, src, mean, comps, cube.shape[0], z)
    zh = to_np(z)
    qps = [22, 27, 32, 37]
    p = xv.xv_params_init(cfg.ctu, cfg.R, cfg.tu_mask, qps[0])
    buf = xv.alloc_cube_buffers(cube.shape[0], 4, cfg.H, cfg.W, p)
    whole = xv.make_job(z, p, buf["planes"], buf["recon"], minmax=buf["minmax"], mv=buf["mv"], cost=buf["cost"],
                        levels=buf["levels"], tu_log2=buf["tu_log2"], bits=buf["bits"])
    jobs = xv.xv_split_groups(whole, qps)
    assert len(jobs) == 4 and [j.bands for j in jobs] == [3, 3, 3, 1] and [j.p.qp for j in jobs] == qps
    res = xv.xv_encode_batch(ctx, jobs)
    for g, (qp, r) in enumerate(zip(qps, res)):
        b0, b1 = 3 * g, min(3 * g + 3, cube.shape[0])
        want = oracle.encode_cube(np.ascontiguousarray(zh[b0:b1]), cfg.ctu, cfg.R, cfg.tu_mask, qp)
        assert np.array_equal(to_np(buf["planes"][g]), want["planes"][0])
        assert np.array_equal(to_np(buf["recon"][g]), want["recon"][0])
        assert np.array_equal(to_np(buf["mv"][g]), want["mv"][0])
        assert np.array_equal(to_np(buf["levels"][g]), want["levels"][0])
        assert np.array_equal(to_np(buf["bits"][g]).astype(np.uint64), want["bits"][0])
        assert r["total_bits"] == want["total_bits"]
        for a, w in zip(r["psnr_band"], want["psnr_band"]):
            assert (np.isinf(a) and np.isinf(w)) or abs(a - w) <= 1e-9 * abs(w)
    recon_g0 = to_np(buf["recon"][0]).copy()
    xv.xv_encode_batch(ctx, [whole])  # every group at qps[0]
    assert np.array_equal(to_np(buf["recon"][0]), recon_g0)

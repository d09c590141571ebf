"""GPU parity of each C-ABI entry point against the CPU oracle, element by
element: integer outputs bit-exact, PSNR within 1e-9 relative."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import to_dev, to_np
from paper_2506_19656_gb300 import synth

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


def quantize_on_gpu(xv, ctx, cube, ctu, minmax=None):
    bands, T, H, W = cube.shape
    G, Hp, Wp = xv.xv_plane_geometry(bands, H, W, ctu)
    src = to_dev(cube)
    mm = torch.zeros((bands, 2), dtype=torch.float64, device="cuda") if minmax is None else to_dev(minmax)
    planes = torch.empty((G, T, 3, Hp, Wp), dtype=torch.uint16, device="cuda")
    xv.xv_quantize_pack(ctx, src, ctu, mm, planes, minmax_fixed=minmax is not None)
    torch.cuda.synchronize()
    return to_np(planes), to_np(mm)


@pytest.mark.parametrize("shape,ctu", [((3, 4, 64, 64), 8), ((10, 3, 37, 53), 16), ((4, 2, 100, 130), 64),
                                       ((1, 1, 1, 1), 8), ((7, 2, 33, 17), 32)])
def test_quantize_pack_f32(xv, ctx, shape, ctu):
    rng = np.random.default_rng(sum(shape) + ctu)
    cube = rng.normal(0.3, 2.0, shape).astype(np.float32)
    if cube.size > 10:
        cube.flat[rng.choice(cube.size, 5, replace=False)] = np.nan
        cube.flat[3] = np.inf
    planes, mm = quantize_on_gpu(xv, ctx, cube, ctu)
    want_mm, _ = oracle.minmax(cube)
    assert np.array_equal(mm, want_mm)
    assert np.array_equal(planes, oracle.quantize_pack(cube, ctu, want_mm))


def test_quantize_pack_rounding_boundaries(xv, ctx):
    """Samples at exact and near half-step boundaries take the double path."""
    lo, hi = -1.25, 3.5
    k = np.arange(0, 1024, dtype=np.float64)
    x = lo + (k + 0.5) * (hi - lo) / 1023.0
    near = np.concatenate([x, np.nextafter(x.astype(np.float32), np.float32(9)),
                           np.nextafter(x.astype(np.float32), np.float32(-9))]).astype(np.float32)
    near = np.concatenate([near, np.array([lo, hi], np.float32)])
    cube = np.resize(near, (2, 3, 16, 128)).astype(np.float32)
    planes, mm = quantize_on_gpu(xv, ctx, cube, 16)
    assert np.array_equal(planes, oracle.quantize_pack(cube, 16, oracle.minmax(cube)[0]))


def test_quantize_pack_u16_and_fixed_minmax(xv, ctx):
    cube = synth.dynamicearthnet_cube(7, T=2, H=96, W=80, bands=4, n_seeds=20)
    planes, mm = quantize_on_gpu(xv, ctx, cube, 64)
    want_mm, _ = oracle.minmax(cube)
    assert np.array_equal(mm, want_mm)
    assert np.array_equal(planes, oracle.quantize_pack(cube, 64, want_mm))
    fixed = np.array([[100.0, 9000.0], [0.0, 10000.0], [3.3, 4444.4], [2000.0, 2001.0]])
    planes, _ = quantize_on_gpu(xv, ctx, cube, 64, minmax=fixed)
    assert np.array_equal(planes, oracle.quantize_pack(cube, 64, fixed))


def me_case(seed, G, Hp, Wp, smooth=1.5):
    ref = synth.random_planes(seed, G, 1, Hp, Wp, smooth=smooth)[:, 0]
    rng = np.random.default_rng(seed + 1)
    cur = np.empty_like(ref)
    for g in range(G):
        sx, sy = rng.integers(-5, 6, 2)
        cur[g] = np.roll(ref[g], (sy, sx), axis=(1, 2))
        noise = rng.integers(-6, 7, cur[g].shape)
        cur[g] = np.clip(cur[g].astype(int) + noise, 0, 1023)
    return cur, ref


@pytest.mark.parametrize("ctu,R,Hp,Wp,G", [(8, 16, 64, 64, 1), (16, 32, 128, 96, 2), (32, 16, 96, 160, 2),
                                           (64, 64, 128, 192, 1), (8, 3, 24, 40, 3), (16, 7, 16, 16, 1)])
def test_motion_search(xv, ctx, ctu, R, Hp, Wp, G):
    cur, ref = me_case(ctu * 100 + R, G, Hp, Wp)
    p = xv.xv_params_init(ctu, R, 1 << 3, 27)
    npu = (Hp // ctu) * (Wp // ctu)
    mv = torch.zeros((G, npu, 2), dtype=torch.int16, device="cuda")
    cost = torch.zeros((G, npu), dtype=torch.int32, device="cuda")
    mvi = torch.zeros_like(mv)
    costi = torch.zeros_like(cost)
    dcur, dref = to_dev(cur), to_dev(ref)
    xv.xv_motion_search(ctx, dcur, dref, G, 3 * Hp * Wp, Hp, Wp, p, mv, cost, mvi, costi, npu)
    torch.cuda.synchronize()
    for g in range(G):
        wmi, wci = oracle.me_int(cur[g, 0], ref[g, 0], ctu, R, p.lambda_mv_fp16)
        wm, wc = oracle.me_qpel(cur[g, 0], ref[g, 0], ctu, p.lambda_mv_fp16, wmi)
        assert np.array_equal(to_np(mvi)[g], wmi)
        assert np.array_equal(to_np(costi)[g].astype(np.uint32), wci)
        assert np.array_equal(to_np(mv)[g], wm)
        assert np.array_equal(to_np(cost)[g].astype(np.uint32), wc)


def pruning_case(kind, Hp, Wp, seed):
    """Frames on which the sub-block bound of the integer search is weak,
    tight or tied everywhere: (cur, ref) channel-0 planes as [1, 3, Hp, Wp]."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:Hp, 0:Wp]
    if kind == "flat":  # every SAD is 0: the motion cost alone decides
        ref = np.full((Hp, Wp), 300)
        cur = ref.copy()
    elif kind == "flat_offset":  # every SAD is the same non-zero value
        ref = np.full((Hp, Wp), 310)
        cur = np.full((Hp, Wp), 300)
    elif kind == "noise":  # independent noise: weak bounds, most units survive
        ref = rng.integers(0, 1024, (Hp, Wp))
        cur = rng.integers(0, 1024, (Hp, Wp))
    elif kind == "stripes8":  # period 8: equal SADs at vectors 8 apart
        ref = np.where(x % 8 < 4, 800, 100)
        cur = np.roll(ref, 3, axis=1)
    elif kind == "zero_sum_tiles":  # every 4x4 box sum equal: every bound is 0
        a = rng.integers(-200, 201, (4, 4))
        a -= a.sum() // 16
        a[3, 3] -= a.sum()
        ref = 512 + a[y % 4, x % 4]
        cur = np.clip(np.roll(ref, (1, 2), axis=(0, 1)) + rng.integers(-3, 4, (Hp, Wp)), 0, 1023)
    else:  # "checker": period 2 in both axes
        ref = np.where((x + y) % 2 == 0, 900, 50)
        cur = np.roll(ref, (1, 0), axis=(0, 1))
    out = []
    for pl in (cur, ref):
        f = np.zeros((1, 3, Hp, Wp), np.uint16)
        f[0, 0] = pl
        f[0, 1] = pl[::-1]
        f[0, 2] = 512
        out.append(f)
    return out


@pytest.mark.parametrize("kind", ["flat", "flat_offset", "noise", "stripes8", "zero_sum_tiles", "checker"])
@pytest.mark.parametrize("ctu,R,Hp,Wp", [(8, 16, 24, 32), (8, 4, 16, 24), (16, 32, 48, 32), (16, 5, 32, 48),
                                         (32, 16, 64, 96), (32, 12, 64, 64), (64, 64, 128, 128), (64, 9, 64, 128)])
def test_motion_search_pruning_adversarial(xv, ctx, kind, ctu, R, Hp, Wp):
    """The integer search skips candidates by an exact bound: on ties, weak
    bounds and periodic textures its result is still the full search's."""
    cur, ref = pruning_case(kind, Hp, Wp, ctu * 1000 + R)
    p = xv.xv_params_init(ctu, R, 1 << 3, 27)
    npu = (Hp // ctu) * (Wp // ctu)
    mv = torch.zeros((1, npu, 2), dtype=torch.int16, device="cuda")
    cost = torch.zeros((1, npu), dtype=torch.int32, device="cuda")
    mvi = torch.zeros_like(mv)
    costi = torch.zeros_like(cost)
    xv.xv_motion_search(ctx, to_dev(cur), to_dev(ref), 1, 3 * Hp * Wp, Hp, Wp, p, mv, cost, mvi, costi, npu)
    torch.cuda.synchronize()
    wmi, wci = oracle.me_int(cur[0, 0], ref[0, 0], ctu, R, p.lambda_mv_fp16)
    wm, wc = oracle.me_qpel(cur[0, 0], ref[0, 0], ctu, p.lambda_mv_fp16, wmi)
    assert np.array_equal(to_np(mvi)[0], wmi)
    assert np.array_equal(to_np(costi)[0].astype(np.uint32), wci)
    assert np.array_equal(to_np(mv)[0], wm)
    assert np.array_equal(to_np(cost)[0].astype(np.uint32), wc)


@pytest.mark.parametrize("ctu,mask,qp", [(8, 0b1000, 27), (16, 0b11100, 22), (32, 0b111100, 32),
                                         (64, 0b111100, 27), (16, 0b10000, -12), (32, 0b100, 51)])
@pytest.mark.parametrize("first", [True, False])
def test_transform_quant_recon(xv, ctx, ctu, mask, qp, first):
    G, Hp, Wp = 2, 2 * ctu, 3 * ctu
    cur, ref = me_case(ctu + qp, G, Hp, Wp)
    npu = (Hp // ctu) * (Wp // ctu)
    rng = np.random.default_rng(qp + 100)
    mv = rng.integers(-4 * 9, 4 * 9 + 1, (G, npu, 2)).astype(np.int16)
    p = xv.xv_params_init(ctu, 8, mask, qp)
    recon = torch.zeros((G, 3, Hp, Wp), dtype=torch.uint16, device="cuda")
    levels = torch.zeros((G, 3, Hp, Wp), dtype=torch.int16, device="cuda")
    tu = torch.zeros((G, npu), dtype=torch.uint8, device="cuda")
    bits = torch.zeros((G,), dtype=torch.int64, device="cuda")
    dref = None if first else to_dev(ref)
    xv.xv_transform_quant_recon(ctx, to_dev(cur), dref, to_dev(mv), G, 3 * Hp * Wp, Hp, Wp, p, npu, recon, levels,
                                tu, bits, 1)
    torch.cuda.synchronize()
    for g in range(G):
        w = oracle.tqr_frame(cur[g], None if first else ref[g], mv[g], ctu, mask, qp)
        assert np.array_equal(to_np(recon)[g], w["recon"])
        assert np.array_equal(to_np(levels)[g], w["levels"])
        assert np.array_equal(to_np(tu)[g], w["tu_log2"])
        assert int(to_np(bits)[g]) == w["bits"]


@pytest.mark.parametrize("mask", [0b100000, 0b101000, 0b110100, 0b011000, 0b111100])
@pytest.mark.parametrize("qp,content", [(-12, "extreme"), (0, "smooth"), (22, "extreme"), (45, "smooth")])
def test_transform_ctu32_size_subsets(xv, ctx, mask, qp, content):
    """CTU 32's warp-owned transform over subsets of the TU sizes (its
    best/current buffers swap only on improving sizes) and QPs from -12 to 45,
    on smooth planes and on extreme ones (full-range noise against an
    unrelated reference: residuals near +-1023, the largest coefficients and
    levels): every output equals the oracle's."""
    ctu, G, Hp, Wp = 32, 2, 64, 96
    if content == "smooth":
        cur, ref = me_case(700 + qp, G, Hp, Wp)
    else:
        rng = np.random.default_rng(800 + qp)
        cur = rng.integers(0, 1024, (G, 3, Hp, Wp)).astype(np.uint16)
        ref = (1023 - cur).astype(np.uint16)
    npu = (Hp // ctu) * (Wp // ctu)
    rng = np.random.default_rng(qp + 900)
    mv = rng.integers(-4 * 9, 4 * 9 + 1, (G, npu, 2)).astype(np.int16)
    p = xv.xv_params_init(ctu, 8, mask, qp)
    recon = torch.zeros((G, 3, Hp, Wp), dtype=torch.uint16, device="cuda")
    levels = torch.zeros((G, 3, Hp, Wp), dtype=torch.int16, device="cuda")
    tu = torch.zeros((G, npu), dtype=torch.uint8, device="cuda")
    bits = torch.zeros((G,), dtype=torch.int64, device="cuda")
    xv.xv_transform_quant_recon(ctx, to_dev(cur), to_dev(ref), to_dev(mv), G, 3 * Hp * Wp, Hp, Wp, p, npu, recon,
                                levels, tu, bits, 1)
    torch.cuda.synchronize()
    for g in range(G):
        w = oracle.tqr_frame(cur[g], ref[g], mv[g], ctu, mask, qp)
        assert np.array_equal(to_np(recon)[g], w["recon"])
        assert np.array_equal(to_np(levels)[g], w["levels"])
        assert np.array_equal(to_np(tu)[g], w["tu_log2"])
        assert int(to_np(bits)[g]) == w["bits"]


@pytest.mark.parametrize("dtype", ["f32", "u16"])
def test_psnr(xv, ctx, dtype):
    rng = np.random.default_rng(5)
    if dtype == "f32":
        cube = rng.uniform(-2, 5, (5, 3, 30, 41)).astype(np.float32)
        cube[1, 1, 2, 3] = np.nan
    else:
        cube = rng.integers(0, 10001, (5, 3, 30, 41)).astype(np.uint16)
    ctu = 16
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, ctu, mm)
    recon = np.clip(planes.astype(int) + rng.integers(-3, 4, planes.shape), 0, 1023).astype(np.uint16)
    recon[1, :, 1] = planes[1, :, 1]  # band 4 exact -> +inf
    w = oracle.psnr(cube, planes, recon, mm)
    g = xv.xv_psnr(ctx, to_dev(cube), to_dev(planes), to_dev(recon), to_dev(mm))
    for b in range(5):
        if np.isinf(w["psnr_band"][b]):
            assert np.isinf(g["psnr_band"][b])
        else:
            assert abs(g["psnr_band"][b] - w["psnr_band"][b]) <= 1e-9 * abs(w["psnr_band"][b])
        assert g["sse10_band"][b] == int(w["sse10_band"][b])


def test_psnr_magnitudes(xv, ctx):
    """The FP32 (float-float) accumulation against the oracle's double
    definition on awkward bands: tiny and huge magnitudes (the latter on the
    double path), values around zero, and a large offset with a small range
    (heavy cancellation in x - x^)."""
    rng = np.random.default_rng(11)
    shape = (3, 17, 33)
    bands = [rng.uniform(-1e-12, 3e-12, shape), rng.uniform(1e20, 4e20, shape),
             rng.uniform(-1e-3, 1e-3, shape), 1e6 + rng.uniform(0, 1, shape),
             rng.uniform(-7e14, 7e14, shape), rng.uniform(0, 1, shape)]
    cube = np.stack(bands).astype(np.float32)
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, 16, mm)
    recon = np.clip(planes.astype(int) + rng.integers(-2, 3, planes.shape), 0, 1023).astype(np.uint16)
    w = oracle.psnr(cube, planes, recon, mm)
    g = xv.xv_psnr(ctx, to_dev(cube), to_dev(planes), to_dev(recon), to_dev(mm))
    for b in range(len(bands)):
        assert abs(g["psnr_band"][b] - w["psnr_band"][b]) <= 1e-9 * abs(w["psnr_band"][b]), b
        assert g["sse10_band"][b] == int(w["sse10_band"][b])

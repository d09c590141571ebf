"""GPU decoder parity: xv_decode_frame / xv_decode_batch / xv_unpack against
the oracle's decoder, and decode(GPU encode) against the encoder's own
reconstruction and rate."""
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


def random_coded(seed, G, T, Hp, Wp, ctu, R, level_span=60, zero_frac=0.7):
    """Arbitrary coded data (not an encoder's): sparse levels, vectors within
    +-(4R + 3) quarter samples, any allowed TU size per CU."""
    rng = np.random.default_rng(seed)
    levels = rng.integers(-level_span, level_span + 1, (G, T, 3, Hp, Wp)).astype(np.int16)
    levels[rng.random(levels.shape) < zero_frac] = 0
    ncu = (Hp // ctu) * (Wp // ctu)
    mv = rng.integers(-(4 * R + 3), 4 * R + 4, (G, T, ncu, 2)).astype(np.int16)
    mv[:, 0] = 0
    lmax = {8: 3, 16: 4, 32: 5, 64: 5}[ctu]
    tu = rng.integers(2, lmax + 1, (G, T, ncu)).astype(np.uint8)
    return levels, mv, tu


@pytest.mark.parametrize("ctu,R,Hp,Wp,G,qp", [(8, 4, 24, 40, 2, 22), (16, 9, 48, 32, 1, 35), (32, 5, 64, 96, 2, 27),
                                              (64, 6, 128, 64, 1, 30)])
def test_decode_frame_random_data(xv, ctx, ctu, R, Hp, Wp, G, qp):
    """Frame by frame on arbitrary coded data: recon and rate equal the oracle's."""
    T = 3
    levels, mv, tu = random_coded(ctu * 7 + R, G, T, Hp, Wp, ctu, R)
    want = [oracle.decode_planes(levels[g:g + 1], mv[g:g + 1], tu[g:g + 1], ctu, qp) for g in range(G)]
    p = xv.xv_params_init(ctu, R, 0b111100 if ctu >= 32 else (0b11100 if ctu == 16 else 0b1100), qp)
    fsz = 3 * Hp * Wp
    ncu = (Hp // ctu) * (Wp // ctu)
    d_lev, d_mv, d_tu = to_dev(levels), to_dev(mv), to_dev(tu)
    recon = torch.zeros((G, T, 3, Hp, Wp), dtype=torch.int16, device="cuda")
    bits = torch.zeros((G, T), dtype=torch.int64, device="cuda")
    for t in range(T):
        xv.xv_decode_frame(ctx, d_lev[:, t], recon[:, t - 1] if t else None, d_mv[:, t], d_tu[:, t], G, T * fsz, Hp,
                           Wp, p, T * ncu, recon[:, t], bits[:, t], T)
    torch.cuda.synchronize()
    got = to_np(recon).view(np.uint16)
    for g in range(G):
        assert np.array_equal(got[g], want[g]["recon"][0])
        assert np.array_equal(to_np(bits)[g].astype(np.uint64), want[g]["bits"][0])


def gpu_encode(xv, cube, ctu, R, mask, qp):
    bands, T, H, W = cube.shape
    p = xv.xv_params_init(ctu, R, mask, qp)
    buf = xv.alloc_cube_buffers(bands, T, H, W, p)
    buf["src"] = to_dev(cube)
    job = xv.make_job(buf["src"], p, buf["planes"], buf["recon"], minmax=buf["minmax"], mv=buf["mv"],
                      cost=buf["cost"], levels=buf["levels"], tu_log2=buf["tu_log2"], bits=buf["bits"])
    return p, buf, job


def decode_job(xv, p, buf, bands, H, W):
    G, T, _, Hp, Wp = buf["levels"].shape
    out = dict(recon=torch.empty_like(buf["recon"]), bits=torch.zeros((G, T), dtype=torch.int64, device="cuda"),
               dst=torch.zeros((bands, T, H, W), dtype=torch.float32, device="cuda"))
    dj = xv.make_djob(p, buf["levels"], buf["mv"], buf["tu_log2"], out["recon"], bits=out["bits"],
                      minmax=buf["minmax"], dst=out["dst"], bands=bands, H=H, W=W)
    return dj, out


def test_decode_batch_inverts_encode_mixed(xv, ctx):
    """Ragged cubes of every CTU size: the GPU encoder's output, decoded in one
    batch, gives back its reconstruction and rate, and the oracle's unpack."""
    specs = [((4, 5, 40, 56), 8, 6, 0b1100, 30), ((5, 3, 37, 53), 16, 9, 0b11100, 22),
             ((2, 4, 70, 33), 32, 5, 0b111100, 27), ((3, 2, 64, 64), 64, 4, 0b111100, 35)]
    encs, djs, outs = [], [], []
    for i, (shape, ctu, R, mask, qp) in enumerate(specs):
        cube, _ = synth.tiny_cube(700 + i, T=shape[1], H=shape[2], W=shape[3], bands=shape[0])
        p, buf, job = gpu_encode(xv, cube, ctu, R, mask, qp)
        encs.append((cube, buf, xv.xv_encode_batch(ctx, [job])[0]))
        dj, out = decode_job(xv, p, buf, shape[0], shape[2], shape[3])
        djs.append(dj)
        outs.append(out)
    totals = xv.xv_decode_batch(ctx, djs)
    torch.cuda.synchronize()
    for (cube, buf, res), out, tot in zip(encs, outs, totals):
        assert torch.equal(out["recon"].view(torch.int16), buf["recon"].view(torch.int16))
        assert torch.equal(out["bits"], buf["bits"])
        assert tot == res["total_bits"]
        want = oracle.unpack(to_np(buf["recon"]).view(np.uint16), to_np(buf["minmax"]), cube.shape[0], cube.shape[2],
                             cube.shape[3])
        assert np.array_equal(to_np(out["dst"]), want)


@pytest.mark.parametrize("block_size", [128, 256, 512])
def test_decode_batch_every_block_size(xv, ctx, block_size):
    c = synth.WORKLOADS["deepextremecubes"]
    cube = synth.make_cube("deepextremecubes", T=4)[:4]
    p, buf, job = gpu_encode(xv, cube, c.ctu, c.R, c.tu_mask, 27)
    xv.xv_encode_batch(ctx, [job])
    dj, out = decode_job(xv, p, buf, 4, c.H, c.W)
    xv.xv_debug_force_block_size(ctx, block_size)
    try:
        xv.xv_decode_batch(ctx, [dj])
    finally:
        xv.xv_debug_force_block_size(ctx, 0)
    assert torch.equal(out["recon"].view(torch.int16), buf["recon"].view(torch.int16))
    assert torch.equal(out["bits"], buf["bits"])


def test_decode_batch_random_data_matches_oracle(xv, ctx):
    """Arbitrary coded data through the persistent decoder (clipping paths an
    encoder rarely produces)."""
    ctu, R, Hp, Wp, G, T, qp = 16, 12, 64, 80, 2, 5, 18
    levels, mv, tu = random_coded(99, G, T, Hp, Wp, ctu, R, level_span=400, zero_frac=0.5)
    want = [oracle.decode_planes(levels[g:g + 1], mv[g:g + 1], tu[g:g + 1], ctu, qp) for g in range(G)]
    p = xv.xv_params_init(ctu, R, 0b11100, qp)
    recon = torch.zeros((G, T, 3, Hp, Wp), dtype=torch.int16, device="cuda")
    bits = torch.zeros((G, T), dtype=torch.int64, device="cuda")
    dj = xv.make_djob(p, to_dev(levels), to_dev(mv), to_dev(tu), recon, bits=bits)
    (tot,) = xv.xv_decode_batch(ctx, [dj])
    got = to_np(recon).view(np.uint16)
    for g in range(G):
        assert np.array_equal(got[g], want[g]["recon"][0])
        assert np.array_equal(to_np(bits)[g].astype(np.uint64), want[g]["bits"][0])
    assert tot == sum(int(w["bits"].sum()) for w in want)


def test_decode_full_resolution_prefixes(xv, ctx):
    """Two frames of the DynamicEarthNet-shaped (uint16, CTU 64, R 64) and
    ERA5-shaped (721 x 1440, CTU 32) workloads: decode == encoder recon."""
    for name, cube in (("dynamicearthnet", synth.dynamicearthnet_cube(2000, T=2, H=512, W=512)),
                       ("era5", synth.era5_cube(3000, T=2)[:2])):
        c = synth.WORKLOADS[name]
        bands, T, H, W = cube.shape
        p, buf, job = gpu_encode(xv, cube, c.ctu, c.R, c.tu_mask, c.qps[0])
        res = xv.xv_encode_batch(ctx, [job])[0]
        dj, out = decode_job(xv, p, buf, bands, H, W)
        (tot,) = xv.xv_decode_batch(ctx, [dj])
        assert torch.equal(out["recon"].view(torch.int16), buf["recon"].view(torch.int16))
        assert tot == res["total_bits"]


def test_unpack_matches_oracle(xv, ctx):
    rng = np.random.default_rng(8)
    cube = rng.uniform(-4, 9, (5, 3, 21, 35)).astype(np.float32)
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, 8, mm)
    dst = torch.zeros(cube.shape, dtype=torch.float32, device="cuda")
    xv.xv_unpack(ctx, to_dev(planes), 5, 21, 35, to_dev(mm), dst)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(dst), oracle.unpack(planes, mm, 5, 21, 35))

"""GPU parity of the frame-0 intra coding (xv_intra_frame) and the in-loop
deblocking (xv_deblock_frame), alone and inside whole-cube encodes with the
XV_INTRA / XV_DEBLOCK options, against the oracle, bit for bit: every CTU
size, several groups, ragged planes, intra and inter boundary strengths."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_matches, to_dev, to_np
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


def frame_planes(workload, ctu, T=1, **kw):
    if workload == "tiny":
        cube = synth.tiny_cube(kw.get("seed", 5), T=T, H=kw.get("H", 64), W=kw.get("W", 64), bands=kw.get("bands", 6))[0]
    else:
        cube = synth.make_cube(workload, T=T)
    mm, _ = oracle.minmax(cube)
    return cube, oracle.quantize_pack(cube, ctu, mm)


@pytest.mark.parametrize("workload,ctu,mask,qp,shape", [
    ("tiny", 8, 0b1000, 27, dict(H=64, W=64)),
    ("tiny", 8, 0b1100, 22, dict(H=40, W=56)),            # ragged plane, 5 x 7 CUs
    ("deepextremecubes", 16, 0b11100, 27, {}),
    ("tiny", 32, 0b111100, 32, dict(H=96, W=160)),
    ("tiny", 64, 0b111100, 30, dict(H=128, W=192)),
])
def test_intra_frame_matches_the_oracle(xv, ctx, workload, ctu, mask, qp, shape):
    _, planes = frame_planes(workload, ctu, **shape)
    G, _, _, Hp, Wp = planes.shape
    n = (Hp // ctu) * (Wp // ctu)
    p = xv.xv_params_init(ctu, 8, mask, qp)
    cur = to_dev(planes[:, 0])
    recon = torch.zeros_like(cur)
    levels = torch.zeros(cur.shape, dtype=torch.int16, device="cuda")
    tu = torch.zeros((G, n), dtype=torch.uint8, device="cuda")
    mm = torch.zeros((G, n, 2), dtype=torch.int16, device="cuda")
    bits = torch.zeros(G, dtype=torch.int64, device="cuda")
    fs = 3 * Hp * Wp
    xv.xv_intra_frame(ctx, cur, G, fs, Hp, Wp, p, n, recon, levels, tu, mm, bits, 1)
    for g in range(G):
        want = oracle.intra_frame(planes[g, 0], ctu, mask, qp)
        assert np.array_equal(to_np(mm[g]), want["mode_mv"]), g
        assert np.array_equal(to_np(tu[g]), want["tu_log2"]), g
        assert np.array_equal(to_np(levels[g]), want["levels"]), g
        assert np.array_equal(to_np(recon[g]), want["recon"]), g
        assert int(bits[g]) == want["bits"], g


def side_info(rng, G, Hp, Wp, ctu, mask):
    n = (Hp // ctu) * (Wp // ctu)
    sizes = [k for k in range(2, 7) if (mask >> k) & 1 and (1 << k) <= ctu]
    tu = rng.choice(sizes, (G, n)).astype(np.uint8)
    lev = np.where(rng.random((G, 3, Hp, Wp)) < 0.004, rng.integers(-3, 4, (G, 3, Hp, Wp)), 0).astype(np.int16)
    mv = rng.integers(-12, 13, (G, n, 2)).astype(np.int16)
    mv[:, 1::2] = mv[:, ::2][:, :mv[:, 1::2].shape[1]]  # pairs of CUs with equal vectors
    return tu, lev, mv


@pytest.mark.parametrize("workload,ctu,mask,qp,intra", [
    ("deepextremecubes", 16, 0b11100, 37, False),
    ("deepextremecubes", 16, 0b11100, 30, True),
    ("tiny", 8, 0b1100, 45, False),
    ("tiny", 32, 0b111100, 27, False),
    ("tiny", 64, 0b111100, 40, True),
])
def test_deblock_frame_matches_the_oracle(xv, ctx, workload, ctu, mask, qp, intra):
    rng = np.random.default_rng(ctu * 100 + qp)
    shape = {} if workload != "tiny" else dict(H=96 if ctu < 64 else 128, W=128 if ctu < 64 else 192)
    _, planes = frame_planes(workload, ctu, **shape)
    # a coded-looking frame: the planes plus block-wise offsets that leave edges to filter
    G, _, _, Hp, Wp = planes.shape
    rec = planes[:, 0].astype(np.int32)
    rec += rng.integers(-6, 7, (G, 3, Hp // 8, Wp // 8)).repeat(8, axis=2).repeat(8, axis=3)
    rec = np.clip(rec, 0, 1023).astype(np.uint16)
    tu, lev, mv = side_info(rng, G, Hp, Wp, ctu, mask)
    p = xv.xv_params_init(ctu, 8, mask, qp)
    n = tu.shape[1]
    d_rec = to_dev(rec)
    xv.xv_deblock_frame(ctx, d_rec, G, 3 * Hp * Wp, Hp, Wp, p, n, to_dev(tu), to_dev(lev), to_dev(mv), intra)
    got = to_np(d_rec)
    changed = 0
    for g in range(G):
        want = oracle.deblock_frame(rec[g], ctu, qp, tu[g], lev[g], mv[g], intra)
        assert np.array_equal(got[g], want), g
        changed += int(np.count_nonzero(want != rec[g]))
    assert changed > 0


def options_job(xv, cube, ctu, R, mask, qp, flags):
    bands, T, H, W = cube.shape
    p = xv.xv_params_init(ctu, R, mask, qp)
    p.flags = flags
    buf = xv.alloc_cube_buffers(bands, T, H, W, p)
    buf["src"] = to_dev(cube)
    job = xv.make_job(buf["src"], p, buf["planes"], buf["recon"], minmax=buf["minmax"], mv=buf["mv"],
                      cost=buf["cost"], levels=buf["levels"], tu_log2=buf["tu_log2"], bits=buf["bits"])
    return job, buf


@pytest.mark.parametrize("flags", [1, 2, 3])
@pytest.mark.parametrize("case", ["tiny", "deepextremecubes", "dynamicearthnet", "era5"])
def test_encode_cube_with_options_matches_the_oracle(xv, ctx, case, flags):
    if case == "tiny":
        c = synth.WORKLOADS["tiny"]
        cube, ctu, R, mask, qp = synth.make_cube("tiny"), c.ctu, c.R, c.tu_mask, 27
    elif case == "deepextremecubes":
        c = synth.WORKLOADS[case]
        cube, ctu, R, mask, qp = synth.make_cube(case, T=4), c.ctu, c.R, c.tu_mask, 32
    else:  # the full-resolution workloads' CTU sizes on crops of their first frames
        c = synth.WORKLOADS[case]
        cube = np.ascontiguousarray(synth.make_cube(case, T=3)[:, :, :192, :256])
        ctu, R, mask, qp = c.ctu, 16, c.tu_mask, 27
    job, buf = options_job(xv, cube, ctu, R, mask, qp, flags)
    res = xv.xv_encode_cube(ctx, job)
    want = oracle.encode_cube(cube, ctu, R, mask, qp, flags=flags)
    assert_matches(buf, res, want)


def test_options_are_rejected_outside_the_per_frame_path(xv, ctx):
    cube = synth.make_cube("tiny")
    job, _ = options_job(xv, cube, 8, 16, 0b1000, 27, 3)
    with pytest.raises(xv.XvError) as e:
        xv.xv_encode_batch(ctx, [job])
    assert e.value.status == xv.XV_EINVAL
    with pytest.raises(xv.XvError):  # an unknown option
        xv.xv_encode_cube(ctx, options_job(xv, cube, 8, 16, 0b1000, 27, 4)[0])
    # deblocking needs the job's levels and TU sizes
    job2, buf2 = options_job(xv, cube, 8, 16, 0b1000, 27, 2)
    job2.levels = None
    with pytest.raises(xv.XvError) as e2:
        xv.xv_encode_cube(ctx, job2)
    assert e2.value.status == xv.XV_EINVAL


@pytest.mark.parametrize("flags", [1, 2, 3])
@pytest.mark.parametrize("case", ["tiny", "deepextremecubes", "dynamicearthnet"])
def test_decoding_an_optioned_encode_reproduces_it(xv, ctx, case, flags):
    """xv_decode_frame with the encoder's options, frame after frame, rebuilds
    every reconstruction and frame rate of an xv_encode_cube run with them."""
    c = synth.WORKLOADS[case]
    if case == "dynamicearthnet":
        cube = np.ascontiguousarray(synth.make_cube(case, T=3)[:, :, :192, :256])
    else:
        cube = synth.make_cube(case, T=None if case == "tiny" else 4)
    job, buf = options_job(xv, cube, c.ctu, 16, c.tu_mask, 30, flags)
    xv.xv_encode_cube(ctx, job)
    G, T, _, Hp, Wp = buf["levels"].shape
    n = buf["tu_log2"].shape[2]
    fsz = 3 * Hp * Wp
    rec = torch.zeros_like(buf["recon"])
    bits = torch.zeros((G, T), dtype=torch.int64, device="cuda")
    for t in range(T):
        xv.xv_decode_frame(ctx, buf["levels"][:, t], rec[:, t - 1] if t else None, buf["mv"][:, t],
                           buf["tu_log2"][:, t], G, T * fsz, Hp, Wp, job.p, T * n, rec[:, t], bits[:, t], T)
    assert torch.equal(rec.view(torch.int16), buf["recon"].view(torch.int16))
    assert torch.equal(bits, buf["bits"])
    want = oracle.decode_planes(to_np(buf["levels"]), to_np(buf["mv"]), to_np(buf["tu_log2"]), c.ctu, 30, flags=flags)
    assert np.array_equal(to_np(rec), want["recon"]) and np.array_equal(to_np(bits).astype(np.uint64), want["bits"])


@pytest.mark.parametrize("deblock", [False, True])
@pytest.mark.parametrize("ctu,mask", [(8, 0b1100), (16, 0b11100), (32, 0b111100), (64, 0b111100)])
def test_intra_decode_of_arbitrary_coded_data_matches_the_oracle(xv, ctx, ctu, mask, deblock):
    """Frame 0 decoded with XV_INTRA from arbitrary coded data -- every mode,
    random TU sizes, levels up to +-400 -- against the oracle (then
    deblocked as an intra frame with XV_DEBLOCK)."""
    rng = np.random.default_rng(ctu + 7 * deblock)
    G, Hp, Wp = 2, 2 * ctu + (64 if ctu < 64 else 0), 3 * ctu
    n = (Hp // ctu) * (Wp // ctu)
    sizes = [k for k in range(2, 6) if (mask >> k) & 1 and (1 << k) <= ctu]
    tu = rng.choice(sizes, (G, n)).astype(np.uint8)
    lev = np.where(rng.random((G, 3, Hp, Wp)) < 0.05, rng.integers(-400, 401, (G, 3, Hp, Wp)), 0).astype(np.int16)
    modes = np.stack([rng.integers(0, 35, (G, n)), np.zeros((G, n), int)], -1).astype(np.int16)
    p = xv.xv_params_init(ctu, 8, mask, 27)
    p.flags = xv.XV_INTRA | (xv.XV_DEBLOCK if deblock else 0)
    rec = torch.zeros((G, 3, Hp, Wp), dtype=torch.uint16, device="cuda")
    bits = torch.zeros(G, dtype=torch.int64, device="cuda")
    xv.xv_decode_frame(ctx, to_dev(lev), None, to_dev(modes), to_dev(tu), G, 3 * Hp * Wp, Hp, Wp, p, n, rec, bits, 1)
    for g in range(G):
        want, wbits = oracle.decode_intra_frame(lev[g], modes[g], tu[g], ctu, 27)
        if deblock:
            want = oracle.deblock_frame(want, ctu, 27, tu[g], lev[g], modes[g], intra=True)
        assert np.array_equal(to_np(rec[g]), want), g
        assert int(bits[g]) == wbits, g

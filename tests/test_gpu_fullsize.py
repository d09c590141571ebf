"""Parity at the benchmark's full sizes, in the launch the benchmark times:
every sub-cube of a workload at the benchmark's QPs (22, 27 and 32 for the
DeepExtremeCubes shape, the workload's own otherwise) in one xv_encode_batch,
with the block size the autotuner picks (the job list is bench.workload_jobs).

DeepExtremeCubes shape (10 bands x 256 frames x 128 x 128): every output of
the three encodes against the oracle's whole chain.

DynamicEarthNet shape (4 x 300 x 1024 x 1024 uint16) and ERA5 shape (six
sub-cubes of 24..168 frames of 6 x 721 x 1440): the chain is causal and every
inter frame is a full search the oracle needs seconds for, so the oracle
computes, from the synthetic cube alone,
  - the per-band min/max of every sub-cube,
  - the quantised planes of frames sampled across the whole cube,
  - every output of the first frames of every encode (the causal prefix,
    quantised with the whole sub-cube's min/max);
and, deep in every chain (frames T/3, T/2 and T-1 of every encode), the
oracle's motion search, refinement and transform chain run on the GPU's own
reconstruction of the previous frame as the reference: every vector, cost,
level, reconstruction, TU size and frame rate there must be the oracle's;
the other frames are checked by properties that hold at any size: the
decoder (bit-exact against the oracle in its own tests) reproduces every
reconstruction and frame rate from the coded data, samples stay 10-bit,
vectors stay within the search range (+-(4R + 3) quarter samples), frame 0
carries no vector and no cost, TU sizes are allowed ones, and the reported
totals (bits, 10-bit SSE, PSNR) equal sums recomputed from the buffers."""
import numpy as np
import pytest
import torch

import bench
import oracle
from gpu_util import assert_matches, to_np

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


def test_deepextremecubes_full_cube_three_qps_one_batch(xv, ctx):
    cfg, _, cube, _, jobs, bufs = bench.workload_jobs("deepextremecubes", device="cuda",
                                                      qps=bench.default_qps("deepextremecubes"))
    assert cube.shape == (10, 256, 128, 128) and len(jobs) == 3
    res = xv.xv_encode_batch(ctx, jobs)
    mm, _ = oracle.minmax(cube)
    for b, r in zip(bufs, res):
        assert np.array_equal(to_np(b["minmax"]), mm)
        want = oracle.encode_cube(cube, cfg.ctu, cfg.R, cfg.tu_mask, b["qp"], mm=mm)
        assert_matches(b, r, want)


def check_properties(xv, ctx, cfg, b, r):
    """The checks that hold at any size, on one encode's device buffers."""
    G, T = b["bits"].shape
    planes = b["planes"].view(torch.int16)
    recon = b["recon"].view(torch.int16)
    for a in (planes, recon):
        assert bool(((a >= 0) & (a <= 1023)).all())
    mv = b["mv"]
    assert not bool(mv[:, 0].any()) and not bool(b["cost"][:, 0].any())
    assert int(mv.abs().max()) <= 4 * cfg.R + 3
    allowed = torch.zeros(8, dtype=torch.bool, device=mv.device)
    for n in cfg.tu_sizes:
        allowed[int(n).bit_length() - 1] = True
    assert bool(allowed[b["tu_log2"].long()].all())
    assert r["total_bits"] == int(b["bits"].sum())
    # the 10-bit SSE per band from the buffers (band b in group b // 3, channel b % 3)
    sse = []
    for band in range(cfg.bands):
        g, c = band // 3, band % 3
        d = planes[g, :, c, :cfg.H, :cfg.W].to(torch.int32) - recon[g, :, c, :cfg.H, :cfg.W].to(torch.int32)
        sse.append(int((d * d).sum(dtype=torch.int64)))
    assert r["sse10_band"] == sse
    # the fused PSNR equals the standalone entry point's on the same buffers
    alone = xv.xv_psnr(ctx, b["src"], b["planes"], b["recon"], b["minmax"])
    for g_, w in zip(r["psnr_band"], alone["psnr_band"]):
        assert (np.isinf(g_) and np.isinf(w)) or abs(g_ - w) <= 1e-9 * abs(w)
    # the decoder reproduces every reconstruction and frame rate from the coded data
    p = xv.xv_params_init(cfg.ctu, cfg.R, cfg.tu_mask, b["qp"])
    out = torch.empty_like(b["recon"])
    dbits = torch.zeros((G, T), dtype=torch.int64, device=out.device)
    (tot,) = xv.xv_decode_batch(ctx, [xv.make_djob(p, b["levels"], b["mv"], b["tu_log2"], out, bits=dbits)])
    assert torch.equal(out.view(torch.int16), recon)
    assert torch.equal(dbits, b["bits"]) and tot == r["total_bits"]


def check_deep_frames(cfg, b, frames):
    """Frames t > 0 of one encode against the oracle run on that frame alone,
    with the GPU's reconstruction of frame t - 1 as the reference (the closed
    loop's input at t): vectors, costs, levels, reconstruction, TU sizes and
    the frame's rate."""
    lf8, lmv = oracle.lambdas(b["qp"])
    G = b["planes"].shape[0]
    for g in range(G):
        for t in frames:  # only these frames leave the device
            cur, ref = to_np(b["planes"][g, t]), to_np(b["recon"][g, t - 1])
            mvi, _ = oracle.me_int(cur[0], ref[0], cfg.ctu, cfg.R, lmv)
            wmv, wcost = oracle.me_qpel(cur[0], ref[0], cfg.ctu, lmv, mvi)
            assert np.array_equal(to_np(b["mv"][g, t]), wmv), (g, t)
            assert np.array_equal(to_np(b["cost"][g, t]).astype(np.uint32), wcost), (g, t)
            w = oracle.tqr_frame(cur, ref, wmv, cfg.ctu, cfg.tu_mask, b["qp"])
            assert np.array_equal(to_np(b["recon"][g, t]), w["recon"]), (g, t)
            assert np.array_equal(to_np(b["levels"][g, t]), w["levels"]), (g, t)
            assert np.array_equal(to_np(b["tu_log2"][g, t]), w["tu_log2"]), (g, t)
            assert int(b["bits"][g, t]) == w["bits"], (g, t)


@pytest.mark.parametrize("workload, prefix", [("dynamicearthnet", 2), ("era5", 3)])
def test_full_size_sampled_frames_and_properties(xv, ctx, workload, prefix):
    cfg, lengths, cube, _, jobs, bufs = bench.workload_jobs(workload, device="cuda", qps=bench.default_qps(workload))
    res = xv.xv_encode_batch(ctx, jobs)
    assert all(r["status"] == 0 for r in res)
    for T in lengths:
        sub = cube[:, :T]
        mm, _ = oracle.minmax(sub)
        ts = sorted({0, 1, T // 3, T // 2, T - 1})
        want_planes = oracle.quantize_pack(np.ascontiguousarray(sub[:, ts]), cfg.ctu, mm)
        head = np.ascontiguousarray(sub[:, :prefix])
        for b, r in zip(bufs, res):
            if b["T"] != T:
                continue
            assert np.array_equal(to_np(b["minmax"]), mm)
            assert np.array_equal(to_np(b["planes"].view(torch.int16)[:, ts]).view(np.uint16), want_planes)
            want = oracle.encode_cube(head, cfg.ctu, cfg.R, cfg.tu_mask, b["qp"], mm=mm)
            assert_matches(b, r, want, frames=prefix)
            check_deep_frames(cfg, b, sorted({max(1, T // 3), max(1, T // 2), T - 1}))
            check_properties(xv, ctx, cfg, b, r)
    del jobs, bufs
    torch.cuda.empty_cache()

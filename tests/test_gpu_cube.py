"""Whole-cube GPU parity: the plain per-frame path (xv_encode_cube) and the
batched persistent path (xv_encode_batch) against the oracle, on the seeded
synthetic workloads, their causal prefixes and ragged shapes."""
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


def gpu_job(xv, cube, ctu, R, mask, qp, minmax=None):
    bands, T, H, W = cube.shape
    p = xv.xv_params_init(ctu, R, mask, qp)
    buf = xv.alloc_cube_buffers(bands, T, H, W, p)
    buf["src"] = to_dev(cube)
    if minmax is not None:
        buf["minmax"] = to_dev(np.asarray(minmax, np.float64))
    job = xv.make_job(buf["src"], p, buf["planes"], buf["recon"], minmax=buf["minmax"],
                      minmax_fixed=minmax is not None, mv=buf["mv"], cost=buf["cost"], levels=buf["levels"],
                      tu_log2=buf["tu_log2"], bits=buf["bits"])
    return job, buf


def test_tiny_config_plain(xv, ctx):
    c = synth.WORKLOADS["tiny"]
    cube = synth.make_cube("tiny")
    want = oracle.encode_cube(cube, c.ctu, c.R, c.tu_mask, c.qps[0])
    job, buf = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, c.qps[0])
    res = xv.xv_encode_cube(ctx, job)
    assert_matches(buf, res, want)


@pytest.mark.parametrize("qp", [22, 27, 32])
def test_deepextremecubes_prefix_plain_and_batched(xv, ctx, qp):
    """The first 6 frames of the 10-band 128x128 cube (CTU 16, R 32, TU 4-16)."""
    c = synth.WORKLOADS["deepextremecubes"]
    cube = synth.make_cube("deepextremecubes", T=6)
    want = oracle.encode_cube(cube, c.ctu, c.R, c.tu_mask, qp)
    job, buf = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, qp)
    assert_matches(buf, xv.xv_encode_cube(ctx, job), want)
    job2, buf2 = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, qp)
    assert_matches(buf2, xv.xv_encode_batch(ctx, [job2])[0], want)
    # the search statistics: every P-frame PU's (2R+1)^2 candidates defined,
    # at least one unit of them evaluated exactly
    exact, full = xv.xv_last_batch_search_stats(ctx)
    G, npu = (c.bands + 2) // 3, (c.H // c.ctu) * (c.W // c.ctu)
    assert full == G * (6 - 1) * npu * (2 * c.R + 1) ** 2
    side = 2 * c.R + 1
    units = side * (side // 8 + 1 if side % 8 == 1 else (side + 7) // 8)
    assert G * 5 * npu * 8 <= exact <= G * 5 * npu * units * 8


def test_ragged_shapes_and_mixed_batch(xv, ctx):
    """Uneven cubes of different CTU sizes in one batch = each alone = oracle."""
    specs = [((4, 5, 40, 56), 8, 6, 0b1100, 30), ((5, 3, 37, 53), 16, 9, 0b11100, 22),
             ((2, 4, 70, 33), 32, 5, 0b111100, 27), ((3, 2, 64, 64), 64, 4, 0b111100, 35),
             ((1, 7, 24, 16), 8, 3, 0b1000, 12)]
    jobs, bufs, wants = [], [], []
    for i, (shape, ctu, R, mask, qp) in enumerate(specs):
        rng = np.random.default_rng(i)
        cube, _ = synth.tiny_cube(100 + i, T=shape[1], H=shape[2], W=shape[3], bands=shape[0])
        cube = (cube + rng.normal(0, 0.01, cube.shape)).astype(np.float32)
        wants.append(oracle.encode_cube(cube, ctu, R, mask, qp))
        j, b = gpu_job(xv, cube, ctu, R, mask, qp)
        jobs.append(j)
        bufs.append(b)
    results = xv.xv_encode_batch(ctx, jobs)
    for b, r, w in zip(bufs, results, wants):
        assert_matches(b, r, w)
    # the first cube alone through the plain path gives the same bytes
    cube, _ = synth.tiny_cube(100, T=5, H=40, W=56, bands=4)
    cube = (cube + np.random.default_rng(0).normal(0, 0.01, cube.shape)).astype(np.float32)
    j, b = gpu_job(xv, cube, 8, 6, 0b1100, 30)
    assert_matches(b, xv.xv_encode_cube(ctx, j), wants[0])


@pytest.mark.parametrize("block_size", [128, 192, 256, 512, 1])
def test_every_block_size_is_bit_exact(xv, ctx, block_size):
    """The autotuner's candidates, every persistent-kernel block size and the
    per-frame mode (1), all give the oracle's bytes (mixed CTU sizes)."""
    specs = [((4, 4, 40, 56), 8, 6, 0b1100, 30), ((5, 3, 37, 53), 16, 9, 0b11100, 22),
             ((2, 3, 70, 33), 32, 5, 0b111100, 27)]
    jobs, bufs, wants = [], [], []
    for i, (shape, ctu, R, mask, qp) in enumerate(specs):
        cube, _ = synth.tiny_cube(300 + i, T=shape[1], H=shape[2], W=shape[3], bands=shape[0])
        wants.append(oracle.encode_cube(cube, ctu, R, mask, qp))
        j, b = gpu_job(xv, cube, ctu, R, mask, qp)
        jobs.append(j)
        bufs.append(b)
    xv.xv_debug_force_block_size(ctx, block_size)
    try:
        results = xv.xv_encode_batch(ctx, jobs)
        assert xv.xv_last_batch_block_size(ctx) == block_size
    finally:
        xv.xv_debug_force_block_size(ctx, 0)
    for b, r, w in zip(bufs, results, wants):
        assert_matches(b, r, w)


def test_tuner_picks_per_class_configurations_and_every_candidate_is_bit_exact(xv):
    """A fresh context tunes a mixed batch (CTU 8, 16, 32): its log holds every
    class's persistent candidates and the per-frame mode, each class reports
    the configuration it ran, and the tuned batch -- and every candidate with
    a capped number of resident blocks per SM -- gives the oracle's bytes."""
    specs = [((4, 4, 40, 56), 8, 6, 0b1100, 30), ((5, 3, 37, 53), 16, 9, 0b11100, 22),
             ((2, 3, 70, 33), 32, 5, 0b111100, 27)]
    jobs, bufs, wants = [], [], []
    for i, (shape, ctu, R, mask, qp) in enumerate(specs):
        cube, _ = synth.tiny_cube(400 + i, T=shape[1], H=shape[2], W=shape[3], bands=shape[0])
        wants.append(oracle.encode_cube(cube, ctu, R, mask, qp))
        j, b = gpu_job(xv, cube, ctu, R, mask, qp)
        jobs.append(j)
        bufs.append(b)
    c = xv.Context(0)
    try:
        results = xv.xv_encode_batch(c, jobs)
        log = xv.xv_last_tune_log(c)
        entries = [e for e in log.split(";") if e]
        for ctu in (8, 16, 32):
            assert sum(e.startswith(f"ctu{ctu} ") for e in entries) >= 4, log
            nt, per = xv.xv_last_batch_config(c, ctu)
            assert nt in (1, 128, 192, 256, 512)
        assert any(e.startswith("frames ") for e in entries), log
        assert xv.xv_last_batch_config(c, 64) == (0, 0)  # no CTU-64 work
        for b, r, w in zip(bufs, results, wants):
            assert_matches(b, r, w)
        for code in (128 + 1024 * 1, 256 + 1024 * 2):
            xv.xv_debug_force_block_size(c, code)
            results = xv.xv_encode_batch(c, jobs)
            for ctu in (8, 16, 32):
                assert xv.xv_last_batch_config(c, ctu) == (code % 1024, code // 1024)
            for b, r, w in zip(bufs, results, wants):
                assert_matches(b, r, w)
    finally:
        c.close()


def oracle_chain_with_lambda(planes, ctu, R, mask, qp, lmv):
    """The oracle's closed loop (C4) run frame by frame with a motion-cost
    lambda of the caller's choice: integer search and refinement with lmv,
    then the transform chain against the previous reconstruction."""
    G, T, _, Hp, Wp = planes.shape
    n = (Hp // ctu) * (Wp // ctu)
    recon = np.zeros_like(planes)
    mv = np.zeros((G, T, n, 2), np.int16)
    for g in range(G):
        for t in range(T):
            ref = recon[g, t - 1] if t else None
            if t:
                mvi, _ = oracle.me_int(planes[g, t, 0], ref[0], ctu, R, lmv)
                mv[g, t], _ = oracle.me_qpel(planes[g, t, 0], ref[0], ctu, lmv, mvi)
            recon[g, t] = oracle.tqr_frame(planes[g, t], ref, mv[g, t] if t else None, ctu, mask, qp)["recon"]
    return recon, mv


@pytest.mark.parametrize("block_size", [1, 256])
def test_resubmitted_batch_with_new_lambda_is_not_a_stale_graph(xv, ctx, block_size):
    """The same buffers submitted twice through the captured graphs, only the
    motion-cost lambda changed the second time: the second result is the
    oracle's for the new lambda, not a replay of the first (the graph key
    covers every job parameter that a captured launch reads)."""
    c = synth.WORKLOADS["tiny"]
    cube = synth.make_cube("tiny")
    want = oracle.encode_cube(cube, c.ctu, c.R, c.tu_mask, 27)
    job, buf = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, 27)
    xv.xv_debug_force_block_size(ctx, block_size)
    try:
        assert_matches(buf, xv.xv_encode_batch(ctx, [job])[0], want)
        job.p.lambda_mv_fp16 = job.p.lambda_mv_fp16 * 16
        xv.xv_encode_batch(ctx, [job])
        assert xv.xv_last_batch_block_size(ctx) == block_size
    finally:
        xv.xv_debug_force_block_size(ctx, 0)
    recon, mv = oracle_chain_with_lambda(want["planes"], c.ctu, c.R, c.tu_mask, 27, int(job.p.lambda_mv_fp16))
    assert not np.array_equal(mv, want["mv"]), "the new lambda must change some vector for this test to mean anything"
    assert np.array_equal(to_np(buf["mv"]), mv)
    assert np.array_equal(to_np(buf["recon"]), recon)


def test_uint16_dynamicearthnet_prefix(xv, ctx):
    """Two frames of a DynamicEarthNet-shaped uint16 cube (CTU 64, R 64, TU 4-32),
    with a min/max fixed in advance (as a causal prefix of a longer cube would)."""
    c = synth.WORKLOADS["dynamicearthnet"]
    cube = synth.dynamicearthnet_cube(2000, T=2, H=256, W=320)
    mm = np.array([[0.0, 10000.0]] * 4)
    want = oracle.encode_cube(cube, c.ctu, c.R, c.tu_mask, 27, mm=mm)
    job, buf = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, 27, minmax=mm)
    assert_matches(buf, xv.xv_encode_cube(ctx, job), want)


def test_batch_timeout_is_reported_and_context_survives(xv, ctx):
    """A dependency that is never met: the bounded wait returns XV_ETIMEOUT
    (no fault, no hang) and the same context then encodes correctly."""
    c = synth.WORKLOADS["tiny"]
    cube = synth.make_cube("tiny", T=3)
    job, buf = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, 27)
    xv.xv_debug_set_wait_budget(ctx, 20_000_000)  # ~10 ms
    xv.xv_debug_stall_row(ctx, 8 + 3)  # frame 1, CTU row 3 (8 rows per frame)
    with pytest.raises(xv.XvError) as e:
        xv.xv_encode_batch(ctx, [job])
    assert e.value.status == xv.XV_ETIMEOUT
    xv.xv_debug_stall_row(ctx, -1)
    xv.xv_debug_set_wait_budget(ctx, 4_000_000_000)
    want = oracle.encode_cube(cube, c.ctu, c.R, c.tu_mask, 27)
    job, buf = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, 27)
    assert_matches(buf, xv.xv_encode_batch(ctx, [job])[0], want)


def test_batch_graph_capture_and_replay(xv):
    """The second submission of the same batch replays the captured graph; all
    runs (graph, replay, no graph) give the oracle's bytes."""
    c = synth.WORKLOADS["tiny"]
    cubes = [synth.tiny_cube(500 + i, T=4)[0] for i in range(2)]
    wants = [oracle.encode_cube(x, c.ctu, c.R, c.tu_mask, qp) for x, qp in zip(cubes, (22, 32))]
    ctx = xv.Context(0)
    try:
        made = [gpu_job(xv, x, c.ctu, c.R, c.tu_mask, qp) for x, qp in zip(cubes, (22, 32))]
        jobs = [m[0] for m in made]
        for _ in range(3):
            for b in (m[1] for m in made):
                b["recon"].zero_()
                b["mv"].zero_()
            results = xv.xv_encode_batch(ctx, jobs)
            for (j, b), r, w in zip(made, results, wants):
                assert_matches(b, r, w)
        captures, launches = xv.xv_batch_graph_stats(ctx)
        assert captures == 1 and launches >= 2
        xv.xv_set_batch_graphs(ctx, False)
        results = xv.xv_encode_batch(ctx, jobs)
        for (j, b), r, w in zip(made, results, wants):
            assert_matches(b, r, w)
        assert xv.xv_batch_graph_stats(ctx)[0] == 1
    finally:
        ctx.close()


@pytest.mark.parametrize("block_size, pinned", [(1, True), (128, True), (1, False)])
def test_batch_from_host_uploads_every_cube(xv, block_size, pinned):
    """xv_encode_batch_from_host: the cubes come from pinned host memory
    (per-frame mode: on their own stream, smallest first, each job starting
    when its own cube has arrived; persistent: before the batch) or from
    pageable memory (copied before the captured graphs).  The device
    sources hold garbage before every call, one job's cube is already on the
    device (no host source), another job shares an uploaded job's device
    buffer without a host source of its own, and the second call replays the
    captured graph, which must copy again: every output is the oracle's."""
    specs = [((4, 5, 40, 56), 8, 6, 0b1100, 30), ((3, 2, 37, 53), 8, 5, 0b1100, 22),
             ((5, 3, 33, 41), 8, 4, 0b1100, 27)]
    ctx = xv.Context(0)
    try:
        made, hosts, wants = [], [], []
        for i, (shape, ctu, R, mask, qp) in enumerate(specs):
            cube, _ = synth.tiny_cube(700 + i, T=shape[1], H=shape[2], W=shape[3], bands=shape[0])
            wants.append(oracle.encode_cube(cube, ctu, R, mask, qp))
            made.append(gpu_job(xv, cube, ctu, R, mask, qp))
            h = torch.from_numpy(cube.copy())
            hosts.append(None if i == 1 else (h.pin_memory() if pinned else h))
        # first in the list: a job at another QP that reads the first cube's
        # device buffer and has no host source of its own; it must wait for
        # that cube's upload
        cube0, _ = synth.tiny_cube(700, T=5, H=40, W=56, bands=4)
        p0 = xv.xv_params_init(8, 6, 0b1100, 22)
        b0 = xv.alloc_cube_buffers(4, 5, 40, 56, p0)
        b0["src"] = made[0][1]["src"]
        j0 = xv.make_job(b0["src"], p0, b0["planes"], b0["recon"], minmax=b0["minmax"], mv=b0["mv"], cost=b0["cost"],
                         levels=b0["levels"], tu_log2=b0["tu_log2"], bits=b0["bits"])
        made.insert(0, (j0, b0))
        hosts.insert(0, None)
        wants.insert(0, oracle.encode_cube(cube0, 8, 6, 0b1100, 22))
        jobs = [m[0] for m in made]
        xv.xv_debug_force_block_size(ctx, block_size)
        try:
            for _ in range(2):
                for (j, b), h in zip(made, hosts):
                    if h is not None:
                        b["src"].fill_(float("nan"))
                    b["recon"].zero_()
                    b["mv"].zero_()
                results = xv.xv_encode_batch_from_host(ctx, jobs, hosts)
                assert xv.xv_last_batch_block_size(ctx) == block_size
                for (j, b), r, w in zip(made, results, wants):
                    assert_matches(b, r, w)
            assert xv.xv_batch_graph_stats(ctx)[0] == 1
        finally:
            xv.xv_debug_force_block_size(ctx, 0)
    finally:
        ctx.close()


def test_batch_from_host_more_jobs_than_side_streams(xv):
    """Eighteen small cubes from pinned host memory in the per-frame mode:
    jobs share the sixteen side streams (and their uploads one stream), and
    every output is still the oracle's."""
    ctx = xv.Context(0)
    try:
        made, hosts, wants = [], [], []
        for i in range(18):
            T, H, W = 2 + i % 3, 24 + 8 * (i % 4), 40 - 8 * (i % 3)
            cube, _ = synth.tiny_cube(900 + i, T=T, H=H, W=W, bands=3 + i % 2)
            qp = (22, 27, 32)[i % 3]
            wants.append(oracle.encode_cube(cube, 8, 4, 0b1100, qp))
            made.append(gpu_job(xv, cube, 8, 4, 0b1100, qp))
            hosts.append(torch.from_numpy(cube.copy()).pin_memory())
        for j, b in made:
            b["src"].fill_(float("nan"))
        xv.xv_debug_force_block_size(ctx, 1)
        try:
            results = xv.xv_encode_batch_from_host(ctx, [m[0] for m in made], hosts)
        finally:
            xv.xv_debug_force_block_size(ctx, 0)
        for (j, b), r, w in zip(made, results, wants):
            assert_matches(b, r, w)
    finally:
        ctx.close()


def test_full_resolution_dynamicearthnet_and_era5_prefixes(xv, ctx):
    """Full-size frames of the DynamicEarthNet-shaped (1024x1024 uint16, CTU 64,
    R 64, TU 4-32) and ERA5-shaped (721x1440 float32, padded to 736, CTU 32,
    R 16) workloads, on causal prefixes the oracle finishes: plain path, and
    both together in one batch (two CTU classes, one launch each)."""
    c2, c3 = synth.WORKLOADS["dynamicearthnet"], synth.WORKLOADS["era5"]
    den = synth.make_cube("dynamicearthnet", T=2)
    era = synth.make_cube("era5", T=3)
    w2 = oracle.encode_cube(den, c2.ctu, c2.R, c2.tu_mask, 27)
    w3 = oracle.encode_cube(era, c3.ctu, c3.R, c3.tu_mask, 22)
    j2, b2 = gpu_job(xv, den, c2.ctu, c2.R, c2.tu_mask, 27)
    assert_matches(b2, xv.xv_encode_cube(ctx, j2), w2)
    j3, b3 = gpu_job(xv, era, c3.ctu, c3.R, c3.tu_mask, 22)
    assert_matches(b3, xv.xv_encode_cube(ctx, j3), w3)
    for b in (b2, b3):
        b["recon"].zero_()
        b["mv"].zero_()
    r2, r3 = xv.xv_encode_batch(ctx, [j2, j3])
    assert_matches(b2, r2, w2)
    assert_matches(b3, r3, w3)


def test_window_copy_wait_bound_reports_and_context_survives(xv):
    """The per-frame search's wait for its TMA window copy is bounded: with a
    bound of one poll the encode either completes (the copy was already in)
    or returns XV_ETIMEOUT without any fault; with the default bound the same
    context then encodes the oracle's bytes."""
    c = synth.WORKLOADS["tiny"]
    cube = synth.make_cube("tiny", T=3)
    want = oracle.encode_cube(cube, c.ctu, c.R, c.tu_mask, 27)
    ctx = xv.Context(0)
    try:
        xv.xv_debug_set_window_wait(ctx, 1)
        job, buf = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, 27)
        try:
            assert_matches(buf, xv.xv_encode_cube(ctx, job), want)
        except xv.XvError as e:
            assert e.status == xv.XV_ETIMEOUT
        xv.xv_debug_set_window_wait(ctx, 0)
        job, buf = gpu_job(xv, cube, c.ctu, c.R, c.tu_mask, 27)
        assert_matches(buf, xv.xv_encode_cube(ctx, job), want)
    finally:
        ctx.close()

"""Serving (continuous batching): results equal the oracle and are the same
alone and in a mix of requests arriving while others run; admission by the
memory budget; cancellation."""
import time

import numpy as np
import pytest
import torch

import oracle
from gpu_util import to_np
from paper_2506_19656_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xv():
    from paper_2506_19656_gb300 import build, xv as _xv
    build.build()
    oracle.build()
    return _xv


SPECS = [  # (bands, T, H, W), ctu, R, tu mask, qp
    ((3, 6, 64, 64), 8, 16, 0b1000, 27),
    ((4, 9, 48, 80), 16, 12, 0b11100, 22),
    ((5, 4, 70, 33), 32, 6, 0b111100, 32),
    ((2, 3, 64, 128), 64, 8, 0b111100, 27),
    ((10, 5, 32, 32), 16, 8, 0b11100, 30),
]


def make(xv, i):
    shape, ctu, R, mask, qp = SPECS[i]
    cube, _ = synth.tiny_cube(700 + i, T=shape[1], H=shape[2], W=shape[3], bands=shape[0])
    p = xv.xv_params_init(ctu, R, mask, qp)
    G, Hp, Wp = xv.xv_plane_geometry(shape[0], shape[2], shape[3], ctu)
    npu = (Hp // ctu) * (Wp // ctu)
    host = torch.from_numpy(cube).pin_memory()
    recon = torch.zeros((G, shape[1], 3, Hp, Wp), dtype=torch.int16).pin_memory()
    mv = torch.zeros((G, shape[1], npu, 2), dtype=torch.int16).pin_memory()
    req = xv.make_request(host, p, recon_out=recon, mv_out=mv)
    return dict(req=req, host=host, recon=recon, mv=mv, cube=cube, spec=SPECS[i])


def wait_all(xv, ctx, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            done, res = xv.xv_serve_poll(ctx, t)
            if done:
                out[t] = res
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.002)
    return [out[t] for t in tickets]


def check(item, res):
    shape, ctu, R, mask, qp = item["spec"]
    want = oracle.encode_cube(item["cube"], ctu, R, mask, qp, want_levels=False)
    assert res["status"] == 0, res.get("error")
    assert np.array_equal(item["recon"].numpy().view(np.uint16), want["recon"])
    assert np.array_equal(item["mv"].numpy(), want["mv"])
    assert res["total_bits"] == want["total_bits"]
    for g, w in zip(res["psnr_band"], want["psnr_band"]):
        assert (np.isinf(g) and np.isinf(w)) or abs(g - w) <= 1e-9 * abs(w)
    assert res["latency_s"] > 0


@pytest.mark.parametrize("frames_per_tick", [1, 3, 64])
def test_serving_matches_oracle_in_a_mix(xv, frames_per_tick):
    ctx = xv.Context(0)
    try:
        xv.xv_serve_start(ctx, 8, frames_per_tick)
        items = [make(xv, i) for i in range(len(SPECS))]
        tickets = []
        for it in items:  # arrivals spread out while earlier requests run
            tickets.append(xv.xv_serve_submit(ctx, it["req"]))
            time.sleep(0.003)
        results = wait_all(xv, ctx, tickets)
        for it, res in zip(items, results):
            check(it, res)
        stats = xv.xv_serve_stats(ctx)
        assert stats["ticks"] >= 1 and stats["bytes_in_use"] == 0
    finally:
        xv.xv_serve_stop(ctx)
        ctx.close()


def test_same_result_alone_and_in_the_mix(xv):
    ctx = xv.Context(0)
    try:
        xv.xv_serve_start(ctx, 8, 2)
        alone = make(xv, 1)
        res_alone = wait_all(xv, ctx, [xv.xv_serve_submit(ctx, alone["req"])])[0]
        mixed = [make(xv, i) for i in (0, 1, 2, 3, 4, 1)]
        tickets = []
        for it in mixed:
            tickets.append(xv.xv_serve_submit(ctx, it["req"]))
            time.sleep(0.001)
        res_mix = wait_all(xv, ctx, tickets)
        for k in (1, 5):  # the same request inside the mix, twice
            assert torch.equal(mixed[k]["recon"], alone["recon"])
            assert torch.equal(mixed[k]["mv"], alone["mv"])
            assert res_mix[k]["total_bits"] == res_alone["total_bits"]
            assert res_mix[k]["psnr_band"] == res_alone["psnr_band"]
        check(alone, res_alone)
    finally:
        xv.xv_serve_stop(ctx)
        ctx.close()


def test_admission_by_memory_budget_and_rejection(xv):
    items = [make(xv, 0) for _ in range(4)]  # about 0.6 MB of device buffers each
    ctx = xv.Context(0, mem_budget_bytes=1 << 20)  # room for one at a time
    try:
        xv.xv_serve_start(ctx, 8, 2)
        tickets = [xv.xv_serve_submit(ctx, it["req"]) for it in items]
        cube = torch.zeros((10, 4, 128, 128), dtype=torch.float32).pin_memory()  # 2.6 MB of input alone
        big = xv.make_request(cube, xv.xv_params_init(16, 8, 0b11100, 27))
        tb = xv.xv_serve_submit(ctx, big)
        results = wait_all(xv, ctx, tickets + [tb])
        for it, res in zip(items, results[:4]):
            check(it, res)
        assert results[4]["status"] == xv.XV_EBUDGET
        assert xv.xv_serve_stats(ctx)["peak_resident"] == 1
    finally:
        xv.xv_serve_stop(ctx)
        ctx.close()


def test_cancel(xv):
    ctx = xv.Context(0)
    try:
        xv.xv_serve_start(ctx, 1, 1)
        a, b = make(xv, 1), make(xv, 4)
        ta = xv.xv_serve_submit(ctx, a["req"])
        tb = xv.xv_serve_submit(ctx, b["req"])
        xv.xv_serve_cancel(ctx, tb)  # still queued behind a (one slot)
        ra, rb = wait_all(xv, ctx, [ta, tb])
        check(a, ra)
        assert rb["status"] == xv.XV_ECANCELLED
        with pytest.raises(xv.XvError):
            xv.xv_serve_poll(ctx, tb)  # released after the first 'done'
    finally:
        xv.xv_serve_stop(ctx)
        ctx.close()

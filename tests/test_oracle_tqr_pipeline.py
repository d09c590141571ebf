"""Pins of transform-quantise-reconstruct (C4, C11-C13) and of the whole
closed-loop chain: zero-residual closed forms, the low-QP reconstruction
bound, the TU decision rule, the causal-prefix property, group independence
and planted motion through the full chain."""
import numpy as np
import pytest

from paper_2506_19656_gb300 import synth


def test_frame0_flat_512_costs_cbf_only(xvo):
    cur = np.full((3, 64, 96), 512, np.uint16)
    for ctu, mask, Lmax in ((16, 0b11100, 4), (32, 0b111100, 5), (8, 0b1000, 3), (16, 0b1100, 3)):
        r = xvo.tqr_frame(cur, None, None, ctu, mask, 27)
        ncu = (64 // ctu) * (96 // ctu)
        ntu = (ctu >> Lmax) ** 2
        assert np.array_equal(r["recon"], cur)
        assert not r["levels"].any()
        assert np.all(r["tu_log2"] == Lmax)  # ties go to the larger TU
        assert r["bits"] == ncu * (2 + 3 * ntu)


def test_copy_with_zero_vector(xvo):
    rng = np.random.default_rng(0)
    ref = rng.integers(0, 1024, (3, 32, 32)).astype(np.uint16)
    mv = np.zeros((4, 2), np.int16)
    r = xvo.tqr_frame(ref, ref, mv, 16, 0b11100, 32)
    assert np.array_equal(r["recon"], ref)
    assert r["bits"] == 4 * (2 + 2 + 3)


def test_dc_residual_single_level(xvo):
    cur = np.full((3, 16, 16), 512, np.uint16)
    cur[0] += 40
    r = xvo.tqr_frame(cur, None, None, 16, 1 << 4, 22)
    lv = r["levels"]
    assert np.count_nonzero(lv) == 1 and lv[0, 0, 0] > 0
    level = int(lv[0, 0, 0])
    assert r["bits"] == 2 + (1 + 2 * 4 + xvo.ue_len_se(level)) + 1 + 1
    assert np.abs(r["recon"][0].astype(int) - 552).max() <= 4


def test_low_qp_reconstruction_bound(xvo):
    rng = np.random.default_rng(1)
    cur = rng.integers(0, 1024, (3, 32, 32)).astype(np.uint16)
    r = xvo.tqr_frame(cur, None, None, 16, 1 << 2, -12)
    assert np.abs(r["recon"].astype(int) - cur).max() <= 2


def test_tu_decision_is_min_cost(xvo):
    rng = np.random.default_rng(2)
    ref = synth.random_planes(3, 1, 1, 32, 32, smooth=2.0)[0, 0]
    cur = np.clip(ref.astype(int) + rng.integers(-30, 31, ref.shape), 0, 1023).astype(np.uint16)
    mv = rng.integers(-6, 7, (4, 2)).astype(np.int16)
    qp = 27
    lf8, _ = xvo.lambdas(qp)
    full = xvo.tqr_frame(cur, ref, mv, 16, 0b11100, qp)
    singles = {L: xvo.tqr_frame(cur, ref, mv, 16, 1 << L, qp) for L in (2, 3, 4)}
    for cu in range(4):
        cy, cx = divmod(cu, 2)
        sl = (slice(None), slice(16 * cy, 16 * cy + 16), slice(16 * cx, 16 * cx + 16))
        J = {}
        for L, s in singles.items():
            sse = int(((s["recon"][sl].astype(np.int64) - cur[sl]) ** 2).sum())
            bits = int(s["cu_bits"][cu]) - 2 - xvo.mv_bits(*mv[cu])
            J[L] = (sse << 8) + lf8 * bits
        best = min(J.values())
        Lb = max(L for L in J if J[L] == best)
        assert full["tu_log2"][cu] == Lb
        assert np.array_equal(full["recon"][sl], singles[Lb]["recon"][sl])
        assert full["cu_bits"][cu] == singles[Lb]["cu_bits"][cu]


def small_cube(seed=0, T=5):
    x, _ = synth.tiny_cube(seed, T=T, H=40, W=56, bands=4)
    return x


def test_causal_prefix(xvo):
    x = small_cube(0, T=6)
    mm, _ = xvo.minmax(x)
    planes = xvo.quantize_pack(x, 8, mm)
    full = xvo.encode_planes(planes, 8, 6, 0b1100, 27)
    pre = xvo.encode_planes(np.ascontiguousarray(planes[:, :3]), 8, 6, 0b1100, 27)
    for k in ("recon", "mv", "cost", "mv_int", "cost_int", "levels", "tu_log2", "bits"):
        assert np.array_equal(pre[k], full[k][:, :3]), k


def test_groups_are_independent(xvo):
    x = small_cube(1, T=4)
    mm, _ = xvo.minmax(x)
    planes = xvo.quantize_pack(x, 8, mm)
    full = xvo.encode_planes(planes, 8, 4, 0b1000, 30)
    one = xvo.encode_planes(np.ascontiguousarray(planes[1:2]), 8, 4, 0b1000, 30)
    assert np.array_equal(one["recon"], full["recon"][1:2])
    assert np.array_equal(one["bits"], full["bits"][1:2])


def test_planted_motion_through_the_chain(xvo):
    """Random texture moving by known integer steps, coded near-losslessly:
    interior PUs of every P-frame find the planted vector."""
    rng = np.random.default_rng(7)
    H = W = 64
    base = rng.integers(0, 1024, (H + 40, W + 40))
    steps = [(0, 0), (2, -1), (-3, 2), (1, 3)]
    frames, ox, oy = [], 20, 20
    for sx, sy in steps:
        ox, oy = ox + sx, oy + sy  # content moves by -s, so cur(x) = prev(x + s)
        frames.append(base[oy:oy + H, ox:ox + W])
    planes = np.stack([np.stack([f, f, f]) for f in frames])[None].astype(np.uint16)
    enc = xvo.encode_planes(planes, 16, 4, 0b100, -12)
    for t in range(1, len(steps)):
        for pu in range(16):
            y0, x0 = divmod(pu, 4)
            if 1 <= x0 <= 2 and 1 <= y0 <= 2:
                assert tuple(enc["mv_int"][0, t, pu]) == steps[t]
                assert tuple(enc["mv"][0, t, pu]) == (4 * steps[t][0], 4 * steps[t][1])


def test_encode_cube_bpppb_definition(xvo):
    x = small_cube(2, T=3)
    r = xvo.encode_cube(x, 8, 4, 0b1100, 32)
    bands, T, H, W = x.shape
    assert r["bpppb"] == r["total_bits"] / (H * W * T * bands)
    assert r["total_bits"] == int(r["bits"].sum())
    assert np.all(np.isfinite(r["psnr_band"])) and r["psnr_mean"] > 20

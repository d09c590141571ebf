"""The oracle's decoder (coded levels, vectors and TU sizes -> reconstruction
-> cube units), pinned against the oracle's encoder and closed forms."""
import numpy as np
import pytest

import oracle
from paper_2506_19656_gb300 import synth


@pytest.mark.parametrize("shape,ctu,R,mask,qp,dtype", [
    ((4, 5, 40, 56), 8, 6, 0b1100, 30, np.float32),
    ((5, 3, 37, 53), 16, 9, 0b11100, 22, np.float32),
    ((2, 4, 70, 33), 32, 5, 0b111100, 27, np.float32),
    ((3, 3, 64, 64), 64, 4, 0b111100, 35, np.float32),
    ((1, 6, 24, 16), 8, 3, 0b1000, 12, np.float32),
    ((4, 3, 48, 40), 16, 8, 0b10000, 40, np.uint16),
])
def test_decode_inverts_encode(shape, ctu, R, mask, qp, dtype):
    """The decoder's reconstruction and rate equal the encoder's, bit for bit
    (the encoder's recon is, by construction, what a decoder must rebuild)."""
    rng = np.random.default_rng(sum(shape) + ctu)
    cube, _ = synth.tiny_cube(500 + ctu, T=shape[1], H=shape[2], W=shape[3], bands=shape[0])
    if dtype == np.uint16:
        cube = (cube * 9000 + rng.integers(0, 50, cube.shape)).astype(np.uint16)
    else:
        cube = (cube + rng.normal(0, 0.01, cube.shape)).astype(np.float32)
    enc = oracle.encode_cube(cube, ctu, R, mask, qp)
    dec = oracle.decode_planes(enc["levels"], enc["mv"], enc["tu_log2"], ctu, qp)
    assert np.array_equal(dec["recon"], enc["recon"])
    assert np.array_equal(dec["bits"], enc["bits"])


def test_decode_tiny_workload_every_qp():
    c = synth.WORKLOADS["tiny"]
    cube = synth.make_cube("tiny")
    for qp in (12, 27, 45):
        enc = oracle.encode_cube(cube, c.ctu, c.R, c.tu_mask, qp)
        dec = oracle.decode_planes(enc["levels"], enc["mv"], enc["tu_log2"], c.ctu, qp)
        assert np.array_equal(dec["recon"], enc["recon"]) and np.array_equal(dec["bits"], enc["bits"])


@pytest.mark.parametrize("ctu,L", [(8, 2), (16, 3), (32, 5), (64, 4)])
def test_zero_levels_frame0_is_flat(ctu, L):
    """No residual in frame 0: every sample is 2^(B-1) = 512; the rate is 2
    bits per CU (its TU size) plus one coded-block flag per TU and channel."""
    Hp, Wp = 2 * ctu, 3 * ctu
    levels = np.zeros((3, Hp, Wp), np.int16)
    ncu = (Hp // ctu) * (Wp // ctu)
    tu = np.full(ncu, L, np.uint8)
    recon, bits = oracle.decode_frame(levels, None, np.zeros((ncu, 2), np.int16), tu, ctu, 27)
    assert np.all(recon == 512)
    assert bits == ncu * (2 + 3 * (ctu >> L) ** 2)


@pytest.mark.parametrize("ctu", [8, 16, 32])
def test_zero_levels_is_motion_compensation(ctu):
    """With no residual, each CU is its motion-compensated prediction, the
    same samples the interpolation routine gives for that vector; the rate
    adds each vector's signed Exp-Golomb lengths."""
    rng = np.random.default_rng(ctu)
    Hp, Wp = 2 * ctu, 2 * ctu
    ref = rng.integers(0, 1024, (3, Hp, Wp)).astype(np.uint16)
    ncu = 4
    mv = rng.integers(-9, 10, (ncu, 2)).astype(np.int16)
    tu = np.full(ncu, 3, np.uint8)
    recon, bits = oracle.decode_frame(np.zeros((3, Hp, Wp), np.int16), ref, mv, tu, ctu, 30)
    for cu in range(ncu):
        x0, y0 = (cu % 2) * ctu, (cu // 2) * ctu
        for c in range(3):
            want = oracle.interp_block(ref[c], x0, y0, ctu, ctu, int(mv[cu, 0]), int(mv[cu, 1]))
            assert np.array_equal(recon[c, y0:y0 + ctu, x0:x0 + ctu], want)
    want_bits = sum(2 + oracle.mv_bits(int(m[0]), int(m[1])) + 3 * (ctu // 8) ** 2 for m in mv)
    assert bits == want_bits


@pytest.mark.parametrize("L,qp,level", [(2, 22, 3), (3, 27, -5), (4, 32, 7), (5, 37, 1)])
def test_single_dc_level(L, qp, level):
    """One DC level in one TU over a flat frame-0 prediction: the TU holds
    512 + the inverse transform of the dequantised coefficient, clipped; every
    other TU stays 512; the rate counts that level's code length."""
    N = 1 << L
    ctu = max(N, 8)
    levels = np.zeros((3, ctu, ctu), np.int16)
    levels[1, 0, 0] = level
    tu = np.array([L], np.uint8)
    recon, bits = oracle.decode_frame(levels, None, np.zeros((1, 2), np.int16), tu, ctu, qp)
    D = np.zeros((N, N), np.int32)
    D[0, 0] = oracle.dequant(level, qp, L)
    r = oracle.inv_transform(D)
    assert np.array_equal(recon[1, :N, :N], np.clip(512 + r, 0, 1023).astype(np.uint16))
    assert np.all(recon[0] == 512) and np.all(recon[2] == 512)
    ntu = (ctu // N) ** 2
    assert bits == 2 + 3 * ntu + 2 * L + oracle.ue_len_se(level)


def test_unpack_endpoints_and_quantiser_bound():
    """Level 0 is the band minimum exactly, level 1023 the maximum to float
    rounding, and unpack(quantise(x)) is within half a step (plus float
    rounding) of x."""
    rng = np.random.default_rng(3)
    cube = rng.uniform(-3, 7, (4, 3, 20, 27)).astype(np.float32)
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, 8, mm)
    x = oracle.unpack(planes, mm, 4, 20, 27)
    step = (mm[:, 1] - mm[:, 0]) / 1023
    for b in range(4):
        err = np.abs(x[b].astype(np.float64) - cube[b].astype(np.float64))
        assert err.max() <= step[b] / 2 + 4 * np.spacing(np.float32(7))
    lv = np.zeros_like(planes)
    bottom = oracle.unpack(lv, mm, 4, 20, 27)
    for b in range(4):
        assert np.all(bottom[b] == np.float32(mm[b, 0]))
    lv[:] = 1023
    top = oracle.unpack(lv, mm, 4, 20, 27)
    for b in range(4):
        assert abs(float(top[b].max()) - mm[b, 1]) <= np.spacing(np.float32(abs(mm[b, 1]))) * 2

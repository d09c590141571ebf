"""Pins of the oracle's frame-0 intra prediction (reading R4: the H.265 planar,
DC and angular predictions per CU) and in-loop deblocking (reading R5: the
H.265 luma filter on every channel), checked against what the definitions
fix: exact copies and diagonals, rounded means, the transpose symmetry of the
angular modes, linear references, the availability and substitution rules,
the filter's mirror symmetry, its step response and where it may act.  Of
the beta / tC tables (the standard's printed values), the structure is pinned:
beta's piecewise-linear growth with QP, tC's growth with the quantiser step,
the 10-bit scaling and the boundary-strength offset; tC's individual values at
low QP are not."""
import numpy as np
import pytest

import oracle

rng = np.random.default_rng(91)


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def refs(N, lo=0, hi=1024):
    return rng.integers(lo, hi, 2 * N), rng.integers(lo, hi, 2 * N), int(rng.integers(lo, hi))


# ---------------------------------------------------------------- intra
@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_vertical_and_horizontal_modes_copy_the_neighbours(N):
    left, top, tl = refs(N)
    v = oracle.intra_pred(left, top, tl, N, 26)
    h = oracle.intra_pred(left, top, tl, N, 10)
    assert np.array_equal(v, np.tile(top[:N], (N, 1)))
    assert np.array_equal(h, np.tile(left[:N, None], (1, N)))


@pytest.mark.parametrize("N", [8, 16, 32])
def test_diagonal_modes_are_exact_shifts(N):
    left, top, tl = refs(N)
    p2 = oracle.intra_pred(left, top, tl, N, 2)
    p34 = oracle.intra_pred(left, top, tl, N, 34)
    p18 = oracle.intra_pred(left, top, tl, N, 18)
    for y in range(N):
        for x in range(N):
            assert p34[y, x] == top[x + y + 1]   # up-right diagonal
            assert p2[y, x] == left[x + y + 1]   # down-left diagonal
            want = top[x - y - 1] if x > y else (tl if x == y else left[y - x - 1])
            assert p18[y, x] == want             # through the corner


@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_dc_is_the_rounded_mean_of_the_adjacent_samples(N):
    left, top, tl = refs(N)
    dc = oracle.intra_pred(left, top, tl, N, 1)
    mean = (int(top[:N].sum()) + int(left[:N].sum())) / (2 * N)
    assert np.all(dc == int(np.floor(mean + 0.5)))


def test_constant_references_predict_the_constant_in_every_mode():
    N = 16
    for m in range(35):
        p = oracle.intra_pred(np.full(2 * N, 700), np.full(2 * N, 700), 700, N, m)
        assert np.all(p == 700), m


@pytest.mark.parametrize("N", [8, 16, 32])
def test_modes_m_and_36_minus_m_are_transposes(N):
    """The angle table is symmetric about mode 18, and a horizontal mode reads
    the left column exactly as its vertical twin reads the top row: swapping
    the two reference sides transposes the prediction (planar and DC too)."""
    left, top, tl = refs(N)
    for m in range(2, 35):
        a = oracle.intra_pred(left, top, tl, N, m)
        b = oracle.intra_pred(top, left, tl, N, 36 - m)
        assert np.array_equal(a, b.T), m
    for m in (0, 1):
        assert np.array_equal(oracle.intra_pred(left, top, tl, N, m), oracle.intra_pred(top, left, tl, N, m).T)


def test_angle_table_structure_and_inverse_angles():
    ang = [oracle.intra_angle(m) for m in range(2, 35)]
    assert ang == ang[::-1] and ang[0] == 32 and ang[8] == 0 and ang[16] == -32 and ang[24] == 0
    assert all(a > b for a, b in zip(ang[:16], ang[1:17]))   # decreasing from mode 2 to 18
    for a in sorted(set(x for x in ang if x < 0)):
        assert oracle.intra_inv_angle(a) == int(np.floor(8192 / a + 0.5)) or \
            oracle.intra_inv_angle(a) == -int(np.floor(8192 / -a + 0.5))


@pytest.mark.parametrize("mode", [27, 29, 30, 32, 33])
def test_linear_top_row_gives_the_projected_position(mode):
    """With top[k] = a + s k, a vertical mode of positive angle predicts the
    sample at fractional position x + (y + 1) angle / 32 of the row, rounded
    half up (the two-tap interpolation is exact on a line)."""
    N, a, s = 16, 100, 3
    top = a + s * np.arange(2 * N)
    left = rng.integers(0, 1024, 2 * N)
    p = oracle.intra_pred(left, top, 50, N, mode)
    ang = oracle.intra_angle(mode)
    for y in range(N):
        for x in range(N):
            assert p[y, x] == int(np.floor(a + s * (x + (y + 1) * ang / 32) + 0.5))


def test_planar_diagonal_is_the_mean_of_two_constant_sides():
    N = 16
    p = oracle.intra_pred(np.full(2 * N, 300), np.full(2 * N, 901), 0, N, 0)
    assert all(p[i, i] == (300 + 901 + 1) // 2 for i in range(N))
    assert np.all(np.diff(p, axis=1) >= 0) and np.all(np.diff(p, axis=0) <= 0)


def test_reference_availability_and_substitution():
    ctu, H, W = 8, 24, 24
    plane = rng.integers(0, 1024, (H, W)).astype(np.uint16)
    # the first CU: nothing coded -> 2^(B-1)
    l, t, c = oracle.intra_refs(plane, ctu, 0, 0)
    assert np.all(l == 512) and np.all(t == 512) and c == 512
    # second CU of row 0: only its left neighbours; the below-left, the corner
    # and the whole top row are substituted from the nearest available sample
    l, t, c = oracle.intra_refs(plane, ctu, 8, 0)
    assert np.array_equal(l[:8], plane[0:8, 7]) and np.all(l[8:] == plane[7, 7])
    assert c == plane[0, 7] and np.all(t == plane[0, 7])
    # centre CU: left, corner, top and top-right coded; below-left not
    l, t, c = oracle.intra_refs(plane, ctu, 8, 8)
    assert np.array_equal(l[:8], plane[8:16, 7]) and np.all(l[8:] == plane[15, 7])
    assert c == plane[7, 7] and np.array_equal(t, plane[7, 8:24])
    # last CU of a row: the top-right lies outside the plane
    l, t, c = oracle.intra_refs(plane, ctu, 16, 8)
    assert np.array_equal(t[:8], plane[7, 16:24]) and np.all(t[8:] == plane[7, 23])


def test_intra_frame_outputs_are_consistent_and_beat_the_flat_prediction():
    from paper_2506_19656_gb300 import synth
    cube = synth.make_cube("deepextremecubes", T=1)
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, 16, mm)
    cur = planes[0, 0]
    got = oracle.intra_frame(cur, 16, 0b11100, 27)
    flat = oracle.tqr_frame(cur, None, None, 16, 0b11100, 27)
    assert got["bits"] == int(got["cu_bits"].sum())
    assert np.all(got["mode_mv"][:, 1] == 0) and got["mode_mv"][:, 0].min() >= 0 and got["mode_mv"][:, 0].max() <= 34
    assert len(set(got["mode_mv"][:, 0].tolist())) > 3          # the modes vary with the content
    assert got["bits"] < flat["bits"]                            # neighbours predict better than 512
    sse = lambda r: float(((r.astype(np.int64) - cur) ** 2).sum())
    assert sse(got["recon"]) <= 1.5 * sse(flat["recon"])


@pytest.mark.parametrize("N", [8, 16, 32])
def test_mode_decision_finds_the_copy_modes_and_breaks_ties_low(N):
    """Vertical stripes (every column constant, random levels) are predicted
    best by the vertical mode 26 in every CU below the first row (their top
    neighbours are the reconstructed stripes; any slanted mode shifts them);
    horizontal stripes by mode 10 right of the first column.  A constant
    frame at the substitution value 512 is predicted exactly by every mode,
    so the tie goes to the lowest, planar (0), and nothing is coded."""
    H = W = 4 * N
    mask = 0b11100 if N <= 16 else 0b111100
    s = rng.integers(100, 900, W)
    cur = np.broadcast_to(s[None, None, :], (3, H, W)).astype(np.uint16).copy()
    modes = oracle.intra_frame(cur, N, mask, 4)["mode_mv"][:, 0].reshape(H // N, W // N)
    assert np.all(modes[1:] == 26)
    s = rng.integers(100, 900, H)
    cur = np.broadcast_to(s[None, :, None], (3, H, W)).astype(np.uint16).copy()
    modes = oracle.intra_frame(cur, N, mask, 4)["mode_mv"][:, 0].reshape(H // N, W // N)
    assert np.all(modes[:, 1:] == 10)
    cur = np.full((3, H, W), 512, np.uint16)
    got = oracle.intra_frame(cur, N, mask, 27)
    assert np.all(got["mode_mv"][:, 0] == 0) and np.array_equal(got["recon"], cur) and not got["levels"].any()


# ------------------------------------------------------------- deblocking
def side_info(H, W, ctu, tu_log2=4, coded=False, mv=None):
    n = (H // ctu) * (W // ctu)
    tu = np.full(n, tu_log2, np.uint8)
    lev = np.zeros((3, H, W), np.int16)
    if coded:
        lev[:, ::4, ::4] = 1
    mvv = np.zeros((n, 2), np.int16) if mv is None else mv
    return tu, lev, mvv


def test_threshold_tables_follow_their_design_laws():
    """beta' (8-bit) is 0 up to QP 15, then grows by 1 per QP from 6 at QP 16
    to 18 at QP 28 and by 2 per QP from 20 at QP 29 to 64 at QP 51 (clamped
    outside 0..51).  tC' is non-decreasing, 0 up to QP 17 and 1 from 18, ends
    at 24 (QP 53), and above QP 35 roughly doubles every 6 QP like the
    quantiser step 2^((QP-4)/6).  Both are scaled by 2^(10-8) = 4 for 10-bit
    samples; tC is read at QP + 2 (bS - 1) and is 0 at bS 0; beta does not
    depend on bS."""
    beta8 = {}
    tc8 = {}
    for q in range(0, 54):
        b, t = oracle.deblock_params(q, 1)
        assert b % 4 == 0 and t % 4 == 0
        beta8[q], tc8[q] = b // 4, t // 4
        b2, t2 = oracle.deblock_params(q, 2)
        assert b2 == b and oracle.deblock_params(q, 0) == (b, 0)
        assert t2 == oracle.deblock_params(min(q + 2, 53), 1)[1]
    for q in range(0, 52):
        want = 0 if q <= 15 else (q - 10 if q <= 28 else 2 * q - 38)
        assert beta8[q] == want, q
    assert beta8[52] == beta8[53] == 64
    assert all(tc8[q + 1] >= tc8[q] for q in range(53))
    assert all(tc8[q] == 0 for q in range(18)) and tc8[18] == 1 and tc8[53] == 24
    for q in range(36, 48):
        assert 1.7 <= tc8[q + 6] / tc8[q] <= 2.2, q
    assert oracle.deblock_params(-5, 1) == oracle.deblock_params(0, 1)
    assert oracle.deblock_params(60, 1) == oracle.deblock_params(53, 1)


def test_threshold_tables_equal_the_published_values():
    """Every beta' (Q = 0..51) and tC' (Q = 0..53) value equals the standard's
    table (tests/golden/hevc_deblock_thresholds.txt), scaled by 2^(10-8):
    beta at bS 1 and tC at Q = qp with bS 1, i.e. no offset."""
    from conftest import read_golden
    g = read_golden("hevc_deblock_thresholds.txt")
    beta, tc = g["BETA"][0], g["TC"][0]
    assert len(beta) == 52 and len(tc) == 54
    for q in range(54):
        b, t = oracle.deblock_params(q, 1)
        assert b == 4 * beta[min(q, 51)], q
        assert t == 4 * tc[q], q
    # intra edges (bS 2) read tC' two steps up, clamped at 53
    for q in range(54):
        assert oracle.deblock_params(q, 2)[1] == 4 * tc[min(q + 2, 53)], q


def test_no_filtering_at_boundary_strength_zero():
    rec = rng.integers(0, 1024, (3, 32, 32)).astype(np.uint16)
    tu, lev, mv = side_info(32, 32, 16)
    assert np.array_equal(oracle.deblock_frame(rec, 16, 37, tu, lev, mv, intra=False), rec)


def test_boundary_strength_rules_on_a_step_at_a_cu_edge():
    """A small step between two 16 x 16 CUs (x = 16), filtered where the
    boundary strength is > 0: vectors differing by 4 quarter samples in x or
    y (BS 1; by 3: BS 0, untouched), a coded coefficient in the p-side TU
    that touches the edge, in any channel (BS 1 for all three channels, on
    that TU's segments only; in a TU away from the edge: untouched), an intra
    frame (BS 2 everywhere).  The filter moves at most three samples on each
    side.  (Rows below a filtered segment can change too: the horizontal
    pass runs after the vertical one and sees the new differences.)"""
    H, W, ctu, qp = 32, 32, 16, 37
    rec = np.full((3, H, W), 500, np.uint16)
    rec[:, :, 16:] = 508
    zero = np.zeros((3, H, W), np.int16)

    def changed(mv=((0, 0),) * 4, lev=zero, tu=4, intra=False):
        out = oracle.deblock_frame(rec, ctu, qp, np.full(4, tu, np.uint8), lev, np.array(mv, np.int16), intra)
        return out != rec

    for mv in ([[0, 0], [4, 0], [0, 0], [0, 0]], [[0, 0], [0, -4], [0, 0], [0, 0]]):
        c = changed(mv)
        assert c[:, :16, 15:17].all() and not c[:, 20:].any()
        assert not c[:, :, :13].any() and not c[:, :, 19:].any()
    assert not changed([[0, 0], [3, 0], [0, 0], [0, 0]]).any()
    assert not changed([[0, 0], [0, 3], [0, 0], [0, 0]]).any()
    lev = zero.copy()
    lev[2, 3, 12] = 1                       # channel 2, TU x 8..15 / y 0..7
    c = changed(lev=lev, tu=3)
    assert c[:, :8, 15:17].all() and not c[:, 12:].any()
    lev = zero.copy()
    lev[2, 3, 4] = 1                        # channel 2, TU x 0..7: not at the step
    assert not changed(lev=lev, tu=3).any()
    c = changed(intra=True)
    assert c[:, :, 15:17].all() and not c[:, :, :13].any() and not c[:, :, 19:].any()


def test_flat_frame_is_unchanged_at_any_strength():
    rec = np.full((3, 32, 32), 613, np.uint16)
    tu, lev, mv = side_info(32, 32, 16, tu_log2=3)
    assert np.array_equal(oracle.deblock_frame(rec, 16, 45, tu, lev, mv, intra=True), rec)


@pytest.mark.parametrize("qp,intra", [(30, True), (37, False), (45, True)])
def test_mirroring_the_frame_mirrors_the_result(qp, intra):
    """The decisions and the strong filter are mirror-symmetric; the weak
    filter's Delta floors (9 (q0 - p0) - 3 (q1 - p1) + 8) >> 4, so a mirrored
    step can round one level differently: equal up to 1, and exactly equal
    on most filtered samples (a swapped p / q side would break both)."""
    H, W, ctu = 32, 48, 16
    base = np.cumsum(rng.integers(-6, 7, (3, H, W)), axis=2) + 500
    rec = np.clip(base, 0, 1023).astype(np.uint16)
    n = (H // ctu) * (W // ctu)
    tu = rng.choice([2, 3, 4], n).astype(np.uint8)
    lev = (rng.random((3, H, W)) < 0.01).astype(np.int16)
    mv = rng.integers(-9, 10, (n, 2)).astype(np.int16)
    out = oracle.deblock_frame(rec, ctu, qp, tu, lev, mv, intra)
    nx = W // ctu
    perm = np.array([(cu // nx) * nx + (nx - 1 - cu % nx) for cu in range(n)])
    mv_m = mv[perm].copy()
    mv_m[:, 0] = -mv_m[:, 0]
    out_m = oracle.deblock_frame(rec[:, :, ::-1], ctu, qp, tu[perm], lev[:, :, ::-1], mv_m, intra)
    diff = np.abs(out_m[:, :, ::-1].astype(np.int32) - out)
    changed = out != rec
    assert np.count_nonzero(changed) > 100                    # something was filtered
    assert diff.max() <= 1 and np.count_nonzero(diff) < np.count_nonzero(changed) / 3


def test_weak_filter_step_response():
    """A step a | b with |b - a| too large for the strong filter but below
    10 tC: p0 and q0 move towards each other by Delta = clip3(-tC, tC,
    (6 (b - a) + 8) >> 4) (the general Delta with q1 - p1 = q0 - p0 = b - a),
    p1 and q1 by clip3(-tC/2, tC/2, Delta >> 1) and ((-Delta) >> 1)."""
    qp, bs = 37, 1
    beta, tc = oracle.deblock_params(qp, bs)
    a = 400
    for h in ((5 * tc + 1) // 2 + 1, 3 * tc, 10 * tc):
        b = a + h
        s = np.array([[a] * 4 + [b] * 4] * 4)
        out = oracle.deblock_segment(s, bs, qp)
        d = int(np.clip((6 * h + 8) >> 4, -tc, tc))
        if abs((6 * h + 8) >> 4) >= 10 * tc:
            assert np.array_equal(out, s)
            continue
        want = np.array([a, a, a + int(np.clip(d >> 1, -(tc >> 1), tc >> 1)), a + d,
                         b - d, b + int(np.clip((-d) >> 1, -(tc >> 1), tc >> 1)), b, b])
        assert np.array_equal(out[0], want) and np.all(out == out[0]), (h, out[0], want)


def test_natural_edges_and_texture_are_left_alone():
    qp, bs = 37, 2
    beta, tc = oracle.deblock_params(qp, bs)
    a = 100
    big = np.array([[a] * 4 + [a + 27 * tc] * 4] * 4)   # |Delta| >= 10 tC
    assert np.array_equal(oracle.deblock_segment(big, bs, qp), big)
    tex = np.array([[0, 900, 0, 900, 0, 900, 0, 900]] * 4)  # second differences far above beta
    assert np.array_equal(oracle.deblock_segment(tex, bs, qp), tex)


def test_strong_filter_on_a_small_step_stays_monotone_and_bounded():
    qp, bs = 45, 2
    beta, tc = oracle.deblock_params(qp, bs)
    a, h = 300, (5 * tc + 1) // 2 - 1
    s = np.array([[a] * 4 + [a + h] * 4] * 4)
    out = oracle.deblock_segment(s, bs, qp)
    assert np.all(np.diff(out[0]) >= 0) and out[0].min() >= a and out[0].max() <= a + h
    assert np.count_nonzero(out[0] != s[0]) >= 4           # the strong filter reaches p2 / q2


def test_only_tu_and_cu_boundaries_on_the_8x8_grid_are_filtered():
    H, W, ctu = 32, 32, 16
    x = np.arange(W)
    rec = np.broadcast_to(((x // 4) % 2) * 40 + 400, (3, H, W)).astype(np.uint16).copy()
    tu, lev, mv = side_info(H, W, ctu, tu_log2=4)            # 16 x 16 TUs: edges at x = 16 only
    out = oracle.deblock_frame(rec, ctu, 45, tu, lev, mv, intra=True)
    changed = np.nonzero(np.any(out != rec, axis=(0, 1)))[0]
    assert len(changed) and set(changed) <= set(range(16 - 3, 16 + 3))


def test_chain_options_compose_from_the_frame_functions():
    """Frame 0 of an INTRA chain is the intra frame, and with DEBLOCK every
    frame's output is its deblocked reconstruction (tested on two frames)."""
    from paper_2506_19656_gb300 import synth
    cube = synth.tiny_cube(77, T=2, H=48, W=64, bands=3)[0]
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, 16, mm)
    enc = oracle.encode_planes(planes, 16, 8, 0b11100, 30, flags=oracle.INTRA | oracle.DEBLOCK)
    f0 = oracle.intra_frame(planes[0, 0], 16, 0b11100, 30)
    assert np.array_equal(enc["mv"][0, 0], f0["mode_mv"]) and enc["bits"][0, 0] == f0["bits"]
    d0 = oracle.deblock_frame(f0["recon"], 16, 30, f0["tu_log2"], f0["levels"], f0["mode_mv"], intra=True)
    assert np.array_equal(enc["recon"][0, 0], d0)
    plain = oracle.encode_planes(planes, 16, 8, 0b11100, 30)
    none = oracle.encode_planes(planes, 16, 8, 0b11100, 30, flags=0)
    assert all(np.array_equal(plain[k], none[k]) for k in ("recon", "mv", "levels", "bits"))


@pytest.mark.parametrize("flags", [1, 2, 3])
@pytest.mark.parametrize("ctu,mask", [(8, 0b1000), (16, 0b11100), (32, 0b111100)])
def test_decode_of_an_optioned_encode_reproduces_it(flags, ctu, mask):
    """The decoder with the encoder's options rebuilds every reconstruction
    and frame rate from the coded data alone (levels, vectors / modes, TU
    sizes): the intra frame from its decoded neighbours, every frame
    deblocked before it is a reference."""
    from paper_2506_19656_gb300 import synth
    cube = synth.tiny_cube(31 + ctu, T=3, H=64, W=96, bands=4)[0]
    mm, _ = oracle.minmax(cube)
    planes = oracle.quantize_pack(cube, ctu, mm)
    enc = oracle.encode_planes(planes, ctu, 8, mask, 29, flags=flags)
    dec = oracle.decode_planes(enc["levels"], enc["mv"], enc["tu_log2"], ctu, 29, flags=flags)
    assert np.array_equal(dec["recon"], enc["recon"]) and np.array_equal(dec["bits"], enc["bits"])
    # without the options the same data decode to something else
    plain = oracle.decode_planes(enc["levels"], enc["mv"], enc["tu_log2"], ctu, 29)
    assert not np.array_equal(plain["recon"], enc["recon"])

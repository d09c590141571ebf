"""Pins of the oracle's motion estimation (C7 integer full search, C8
quarter-pel refinement): planted shifts, tie-break, the motion-cost model,
and an independent numpy brute force on tiny frames."""
import numpy as np
import pytest

from conftest import read_golden


def test_ue_lengths(xvo):
    # se(v) -> ue(k): 0->0, 1->1, -1->2, 2->3, -2->4 ...; Exp-Golomb code
    # lengths (H.265 subclause 9.2): k = 0: 1 bit, 1..2: 3, 3..6: 5, 7..14: 7, 15..30: 9
    vals = (0, 1, -1, 2, -2, 3, -3, 4, -4, 7, -7, 8, -8)
    assert [xvo.ue_len_se(v) for v in vals] == [1, 3, 3, 5, 5, 5, 5, 7, 7, 7, 7, 9, 9]


def test_lambdas(xvo):
    for qp in (22, 27, 32):
        lam = 0.57 * 2 ** ((qp - 12) / 3)
        lf8, lmv = xvo.lambdas(qp)
        assert abs(lf8 / 256 - lam) <= 0.5 / 256
        assert abs(lmv / 65536 - np.sqrt(lam)) <= 0.5 / 65536
    assert xvo.mv_cost(0, 0, 65536) == 2


def texture(seed, H, W):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1024, (H, W)).astype(np.uint16)


@pytest.mark.parametrize("s", [(0, 0), (3, -2), (-5, 4), (7, 7), (-8, 0)])
def test_planted_integer_shift(xvo, s):
    """cur(x) = ref(x + s) on a random texture: every PU whose block + shift
    stays inside the frame finds mv = s with J = mvcost(4 s)."""
    H = W = 64
    ctu, R = 8, 8
    ref = texture(11, H, W)
    cur = np.zeros_like(ref)
    sx, sy = s
    for y in range(H):
        for x in range(W):
            cur[y, x] = ref[min(max(y + sy, 0), H - 1), min(max(x + sx, 0), W - 1)]
    _, lmv = xvo.lambdas(27)
    mv, J = xvo.me_int(cur, ref, ctu, R, lmv)
    nx = W // ctu
    for pu in range(len(mv)):
        x0, y0 = (pu % nx) * ctu, (pu // nx) * ctu
        if 0 <= x0 + sx and x0 + ctu + sx <= W and 0 <= y0 + sy and y0 + ctu + sy <= H:
            assert tuple(mv[pu]) == s
            assert J[pu] == xvo.mv_cost(4 * sx, 4 * sy, lmv)


def test_flat_frame_prefers_zero_vector(xvo):
    cur = np.full((32, 32), 400, np.uint16)
    _, lmv = xvo.lambdas(27)
    mv, J = xvo.me_int(cur, cur, 8, 4, lmv)
    assert not mv.any()
    assert np.all(J == xvo.mv_cost(0, 0, lmv))


def test_tie_break_smaller_raster_index(xvo):
    """Columns alternating with period 2 and cur(x) = ref(x + 1): dx = +1 and
    dx = -1 both have SAD 0 and equal cost (|ue| of 4 and -4 are both 7);
    the smaller raster index, dx = -1, wins."""
    H = W = 48
    yy, xx = np.mgrid[0:H, 0:W]
    rng = np.random.default_rng(5)
    rowv = rng.integers(0, 1024, H)
    ref = np.where(xx % 2 == 0, 100, 900).astype(np.int64) + rowv[:, None] * 0
    ref = ref.astype(np.uint16)
    cur = np.ascontiguousarray(np.roll(ref, -1, axis=1))  # cur(x) = ref(x+1)
    _, lmv = xvo.lambdas(27)
    mv, _ = xvo.me_int(cur, ref, 8, 3, lmv)
    nx = W // 8
    for pu in range(len(mv)):
        x0 = (pu % nx) * 8
        if 8 <= x0 <= W - 16:
            assert tuple(mv[pu]) == (-1, 0)


def brute_force_me(cur, ref, ctu, R, lmv, bits):
    """Independent statement: edge-padded reference, all candidates at once."""
    H, W = cur.shape
    pad = np.pad(ref.astype(np.int64), R, mode="edge")
    out = []
    for y0 in range(0, H, ctu):
        for x0 in range(0, W, ctu):
            blk = cur[y0:y0 + ctu, x0:x0 + ctu].astype(np.int64)
            best = None
            for dy in range(-R, R + 1):
                for dx in range(-R, R + 1):
                    win = pad[R + y0 + dy:R + y0 + dy + ctu, R + x0 + dx:R + x0 + dx + ctu]
                    J = int(np.abs(blk - win).sum()) + ((lmv * (bits(4 * dx) + bits(4 * dy)) + 32768) >> 16)
                    key = (J, (dy + R) * (2 * R + 1) + dx + R)
                    if best is None or key < best[0]:
                        best = (key, (dx, dy))
            out.append((best[1], best[0][0]))
    return out


def test_brute_force_tiny(xvo):
    def bits(v):
        k = 2 * v - 1 if v > 0 else -2 * v
        return 2 * int(np.floor(np.log2(k + 1))) + 1
    rng = np.random.default_rng(9)
    for trial in range(3):
        ref = (rng.integers(0, 64, (16, 16)) * 16).astype(np.uint16)
        cur = np.roll(ref, (1, -2), axis=(0, 1)).astype(np.int64) + rng.integers(-8, 9, (16, 16))
        cur = np.clip(cur, 0, 1023).astype(np.uint16)
        _, lmv = xvo.lambdas(27 + 5 * trial)
        mv, J = xvo.me_int(cur, ref, 8, 3, lmv)
        bf = brute_force_me(cur, ref, 8, 3, lmv, bits)
        assert [tuple(m) for m in mv] == [b[0] for b in bf]
        assert J.tolist() == [b[1] for b in bf]


@pytest.mark.parametrize("mvq", [(2, 0), (0, -2), (1, 3), (-3, -1), (6, -5), (-9, 10)])
def test_planted_subpel_shift_is_recovered(xvo, mvq):
    """cur = the reference interpolated at a planted quarter-sample vector with
    the same filter: interior PUs recover it with SATD 0 from the integer
    search's start."""
    H = W = 64
    rng = np.random.default_rng(21)
    base = rng.normal(size=(H, W))
    from numpy.fft import fft2, ifft2, fftfreq
    k2 = fftfreq(H)[:, None] ** 2 + fftfreq(W)[None, :] ** 2
    smooth = np.real(ifft2(fft2(base) * np.exp(-2 * np.pi ** 2 * 2.0 ** 2 * k2)))
    ref = np.clip((smooth - smooth.min()) / np.ptp(smooth) * 1000 + 10, 0, 1023).astype(np.uint16)
    ctu = 16
    cur = xvo.interp_block(ref, 0, 0, W, H, mvq[0], mvq[1])
    lf8, lmv = xvo.lambdas(12)
    mvi, _ = xvo.me_int(cur, ref, ctu, 4, lmv)
    mv, J = xvo.me_qpel(cur, ref, ctu, lmv, mvi)
    nx = W // ctu
    hits = 0
    for pu in range(len(mv)):
        x0, y0 = (pu % nx) * ctu, (pu // nx) * ctu
        if 8 <= x0 <= W - ctu - 8 and 8 <= y0 <= H - ctu - 8:
            if abs(4 * int(mvi[pu][0]) - mvq[0]) <= 3 and abs(4 * int(mvi[pu][1]) - mvq[1]) <= 3:
                assert tuple(mv[pu]) == mvq
                assert J[pu] == xvo.mv_cost(mvq[0], mvq[1], lmv)
                hits += 1
    assert hits >= 2


# ---------------------------------------------------------------------------
# Independent restatement of the quarter-sample refinement (C8): its own
# interpolation from the published taps, its own SATD from scipy's Hadamard
# matrix, and the stated search order.  The oracle's refinement must agree
# with it on frames built to tie, where a wrong visiting order, a
# non-strict replacement or a wrong centre for the second stage change the
# answer.

RING = [(-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]


def _se_bits(v):
    k = 2 * v - 1 if v > 0 else -2 * v
    return 2 * int(np.floor(np.log2(k + 1))) + 1


def _interp(ref, x0, y0, n, mvx, mvy, taps):
    """The n x n prediction at quarter-sample vector (mvx, mvy): edge-padded
    reference, full samples << 4, one fractional axis >> 2, both: horizontal
    >> 2 then vertical >> 6, weighted-default rounding (v + 8) >> 4, 10 bits."""
    pad = 80
    p = np.pad(ref.astype(np.int64), pad, mode="edge")
    ix, fx, iy, fy = mvx >> 2, mvx & 3, mvy >> 2, mvy & 3
    ys = y0 + iy + pad + np.arange(-3, n + 5)
    xs = x0 + ix + pad + np.arange(-3, n + 5)
    win = p[np.ix_(ys, xs)]  # rows/cols -3 .. n+4 around the block
    if fx:
        f = np.asarray(taps[fx], np.int64)
        h = sum(f[i] * win[:, i:i + n] for i in range(8)) >> 2   # rows -3..n+4, cols 0..n-1
    else:
        h = win[:, 3:3 + n]
    if fy:
        f = np.asarray(taps[fy], np.int64)
        v = sum(f[i] * h[i:i + n, :] for i in range(8))
        v = v >> (6 if fx else 2)
    else:
        v = h[3:3 + n, :] if fx else h[3:3 + n, :] << 4
    return np.clip((v + 8) >> 4, 0, 1023)


def _satd(d):
    import scipy.linalg
    H8 = scipy.linalg.hadamard(8)
    s = 0
    for by in range(0, d.shape[0], 8):
        for bx in range(0, d.shape[1], 8):
            s += (int(np.abs(H8 @ d[by:by + 8, bx:bx + 8] @ H8.T).sum()) + 2) >> 2
    return s


def restated_refinement(cur, ref, ctu, lmv, mv_int, taps, order=RING, strict=True, second_centre="best"):
    """Per PU: J at 4 mv_int, then the 8 half-sample neighbours in `order`
    (replace when J is strictly lower), then the 8 quarter-sample neighbours
    of the best.  The keyword arguments plant known mistakes for the
    sensitivity check below."""
    H, W = cur.shape
    nx = W // ctu
    out, cost = [], []
    for pu in range(len(mv_int)):
        x0, y0 = (pu % nx) * ctu, (pu // nx) * ctu
        blk = cur[y0:y0 + ctu, x0:x0 + ctu].astype(np.int64)

        def J(mx, my):
            sat = _satd(blk - _interp(ref, x0, y0, ctu, mx, my, taps))
            return sat + ((lmv * (_se_bits(mx) + _se_bits(my)) + 32768) >> 16)

        start = (4 * int(mv_int[pu][0]), 4 * int(mv_int[pu][1]))
        best, bJ = start, J(*start)
        for step in (2, 1):
            c = best if (step == 2 or second_centre == "best") else start
            for ox, oy in order:
                m = (c[0] + step * ox, c[1] + step * oy)
                j = J(*m)
                if j < bJ or (not strict and j == bJ):
                    best, bJ = m, j
        out.append(best)
        cost.append(bJ)
    return out, cost


def _tie_frames():
    """(cur, ref) pairs whose candidates tie often: constant, period-2
    stripes in x and y, a checkerboard, a ramp, and a random texture."""
    rng = np.random.default_rng(31)
    H = W = 24
    yy, xx = np.mgrid[0:H, 0:W]
    planes = [
        np.full((H, W), 600),
        np.where(xx % 2 == 0, 200, 800),
        np.where(yy % 2 == 0, 300, 700),
        np.where((xx + yy) % 2 == 0, 100, 900),
        4 * xx + 8 * yy + 50,
        rng.integers(0, 1024, (H, W)),
    ]
    out = []
    for i, r in enumerate(planes):
        r = r.astype(np.uint16)
        out.append((r, r))                                       # cur = ref
        out.append((np.roll(r, (1, -1), axis=(0, 1)), r))        # shifted copy
        c = np.clip(r.astype(np.int64) + rng.integers(-3, 4, r.shape), 0, 1023).astype(np.uint16)
        out.append((c, r))                                       # noisy copy
    return out


def _starts(n, rng):
    return np.array([[int(rng.integers(-3, 4)), int(rng.integers(-3, 4))] for _ in range(n)], np.int16)


def test_refinement_matches_independent_restatement(xvo):
    taps_g = read_golden("hevc_luma_filter.txt")
    taps = {1: taps_g["QUARTER"][0], 2: taps_g["HALF"][0], 3: taps_g["THREEQUARTER"][0]}
    rng = np.random.default_rng(7)
    ctu = 8
    for cur, ref in _tie_frames():
        for lmv in (4096, 65536, 300000):  # small lambdas round many bit counts to one cost
            starts = _starts((cur.shape[0] // ctu) * (cur.shape[1] // ctu), rng)
            mv, J = xvo.me_qpel(cur, ref, ctu, lmv, starts)
            want, wJ = restated_refinement(cur, ref, ctu, lmv, starts, taps)
            assert [tuple(int(v) for v in m) for m in mv] == want
            assert [int(j) for j in J] == wJ


def test_refinement_fixture_detects_planted_mistakes(xvo):
    """The frames above separate the stated order from plausible misreadings:
    for each planted mistake at least one PU's answer changes."""
    taps_g = read_golden("hevc_luma_filter.txt")
    taps = {1: taps_g["QUARTER"][0], 2: taps_g["HALF"][0], 3: taps_g["THREEQUARTER"][0]}
    mistakes = {
        "non-strict replacement": dict(strict=False),
        "reversed ring order": dict(order=RING[::-1]),
        "column-major ring order": dict(order=sorted(RING)),
        "second stage around the start": dict(second_centre="start"),
    }
    ctu = 8
    found = {k: False for k in mistakes}
    rng = np.random.default_rng(7)
    for cur, ref in _tie_frames():
        for lmv in (4096, 65536, 300000):
            starts = _starts((cur.shape[0] // ctu) * (cur.shape[1] // ctu), rng)
            right = restated_refinement(cur, ref, ctu, lmv, starts, taps)
            for k, kw in mistakes.items():
                if not found[k] and restated_refinement(cur, ref, ctu, lmv, starts, taps, **kw) != right:
                    found[k] = True
    assert all(found.values()), found

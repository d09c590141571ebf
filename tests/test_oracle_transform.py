"""Pins of the oracle's integer core transform (convention C10) against the
published HEVC matrices, orthogonality, the DCT it approximates (scipy), and
round-trip bounds."""
import numpy as np
import pytest
import scipy.fft

from conftest import read_golden


def test_t4_matches_published(xvo):
    g = read_golden("hevc_transform.txt")
    assert xvo.transform_matrix(4).tolist() == g["T4"]


@pytest.mark.parametrize("N", [8, 16, 32])
def test_odd_rows_match_published(xvo, N):
    g = read_golden("hevc_transform.txt")
    T = xvo.transform_matrix(N)
    assert T[1::2, 0].tolist() == g[f"ODD{N}"][0]


def test_t8_row1(xvo):
    g = read_golden("hevc_transform.txt")
    assert xvo.transform_matrix(8)[1].tolist() == g["T8ROW1"][0]


@pytest.mark.parametrize("N", [8, 16, 32])
def test_even_rows_embed_half_size(xvo, N):
    T, Th = xvo.transform_matrix(N), xvo.transform_matrix(N // 2)
    assert np.array_equal(T[0::2, : N // 2], Th)


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_symmetry_and_near_orthogonality(xvo, N):
    T = xvo.transform_matrix(N).astype(np.int64)
    k = np.arange(N)[:, None]
    assert np.array_equal(T[:, ::-1], T * np.where(k % 2 == 0, 1, -1))
    G = T @ T.T / (4096.0 * N)
    d = np.diag(G)
    # the smallest norm is the 4-point odd rows: 2 (83^2 + 36^2) / 16384 = 0.9991455
    assert d.min() >= 16370 / 16384 and d.max() <= 1.00132
    off = np.abs(G - np.diag(d)).max()
    assert off <= 0.00287
    if N == 4:
        assert off == 0


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_close_to_scaled_cosines(xvo, N):
    T = xvo.transform_matrix(N)
    k = np.arange(N)[:, None]
    n = np.arange(N)[None, :]
    ref = 64 * np.sqrt(2) * np.cos(k * np.pi * (2 * n + 1) / (2 * N))
    ref[0, :] = 64
    assert np.abs(T - ref).max() <= 1.364


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_forward_is_scaled_orthonormal_dct(xvo, N):
    """C ~= 2^(15 - B - log2 N) * DCT-II(X) (scipy, orthonormal), B = 10.

    The integer matrix departs from the scaled cosines by up to 4% on single
    entries (36 vs 34.6 in the 4-point matrix), so the check is on the
    Frobenius norm: within 3.5%.  A wrong shift (factor 2), a transposed
    operand or a sign error gives an error of order 100%."""
    rng = np.random.default_rng(N)
    L = N.bit_length() - 1
    for _ in range(20):
        X = rng.integers(-1023, 1024, (N, N)).astype(np.int32)
        C = xvo.fwd_transform(X).astype(np.float64)
        D = scipy.fft.dctn(X.astype(np.float64), type=2, norm="ortho") * 2.0 ** (5 - L)
        assert np.linalg.norm(C - D) <= 0.035 * np.linalg.norm(D)


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_dc_only_block(xvo, N):
    """A constant residual d puts exactly 32 d in the DC coefficient, 0 elsewhere."""
    for d in (-1023, -7, 1, 300):
        C = xvo.fwd_transform(np.full((N, N), d, np.int32))
        E = np.zeros((N, N), np.int32)
        E[0, 0] = 32 * d
        assert np.array_equal(C, E)


@pytest.mark.parametrize("N,bound", [(4, 2), (8, 6), (16, 16), (32, 20)])
def test_round_trip_without_quantisation(xvo, N, bound):
    rng = np.random.default_rng(1)
    worst = 0
    for _ in range(50):
        X = rng.integers(-1023, 1024, (N, N)).astype(np.int32)
        R = xvo.inv_transform(xvo.fwd_transform(X))
        worst = max(worst, int(np.abs(R - X).max()))
    assert worst <= bound


@pytest.mark.parametrize("N", [4, 8])
def test_round_trip_low_qp_small_amplitude(xvo, N):
    """qP 0 (QP -12): max |x - inv(deq(quant(fwd x)))| <= 2 at amplitude <= 64."""
    L = N.bit_length() - 1
    rng = np.random.default_rng(0)
    for amp in (8, 64):
        for _ in range(30):
            X = rng.integers(-amp, amp + 1, (N, N)).astype(np.int32)
            C = xvo.fwd_transform(X)
            D = xvo.dequant(xvo.quant(C, -12, L), -12, L)
            R = xvo.inv_transform(D)
            assert np.abs(R - X).max() <= 2


def test_inverse_of_zero_is_zero(xvo):
    for N in (4, 8, 16, 32):
        assert not xvo.inv_transform(np.zeros((N, N), np.int32)).any()

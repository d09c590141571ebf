"""CPU oracle for the encoder-analysis path (test infrastructure only).

This package is the plain, slow statement of what the GPU library computes:
per-band min-max quantisation to 10-bit planes with three-band packing
(paper Sec. 2.1), integer full-search + quarter-pel motion estimation, the
HEVC-style integer core transform, quantise / dequantise / inverse /
reconstruct, and the PSNR and bits-per-pixel-per-band reductions (paper
Sec. 2.3); beyond the encoder, the decoder (the video2xarray step), SSIM and
spectral angle (Sec. 2.3), frame-0 intra prediction and in-loop deblocking
(options), and PCA over bands (Sec. 2.1).  The arithmetic lives in ``xvo.c``
(plain C loops, compiled with gcc); this module only marshals numpy arrays,
except for PCA, which is numpy in float64 with ``eigh`` as the library step.

Parity unpinned (see ``xvo.h``): only the end-to-end outputs of whole
synthetic encodes, which no published value fixes.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libxvo.so")
_SRC = os.path.join(_HERE, "xvo.c")
_lock = threading.Lock()
_lib = None

F32, U16 = 0, 1
BIT_DEPTH = 10


def build(force: bool = False) -> str:
    """Compile xvo.c into a shared library (OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "xvo.h"))
    ):
        return _LIB_PATH
    os.makedirs(_BUILD_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            vp, i, i64, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint
            L.xvo_group_count.argtypes = [i]
            L.xvo_group_band.argtypes = [i, i, i]
            L.xvo_minmax.argtypes = [vp, i, i, i, i, i, vp, vp]
            L.xvo_quantize_pack.argtypes = [vp, i, i, i, i, i, i, vp, vp]
            L.xvo_transform_matrix.argtypes = [i, vp]
            L.xvo_fwd_transform.argtypes = [i, vp, vp]
            L.xvo_inv_transform.argtypes = [i, vp, vp]
            L.xvo_quant.argtypes = [ctypes.c_int32, i, i]
            L.xvo_quant.restype = ctypes.c_int32
            L.xvo_dequant.argtypes = [ctypes.c_int32, i, i]
            L.xvo_dequant.restype = ctypes.c_int32
            L.xvo_lambdas.argtypes = [i, vp, vp]
            L.xvo_ue_len_se.argtypes = [i]
            L.xvo_mv_bits.argtypes = [i, i]
            L.xvo_mv_cost.argtypes = [i, i, i64]
            L.xvo_mv_cost.restype = ctypes.c_uint32
            L.xvo_interp_block.argtypes = [vp, i, i, i, i, i, i, i, i, vp]
            L.xvo_hadamard8.argtypes = [vp, vp]
            L.xvo_satd.argtypes = [vp, i, i]
            L.xvo_satd.restype = ctypes.c_uint32
            L.xvo_me_int.argtypes = [vp, vp, i, i, i, i, i64, vp, vp]
            L.xvo_me_qpel.argtypes = [vp, vp, i, i, i, i64, vp, vp, vp]
            L.xvo_tqr_frame.argtypes = [vp, vp, vp, i, i, i, u, i, i64, vp, vp, vp, vp]
            L.xvo_tqr_frame.restype = ctypes.c_uint64
            L.xvo_encode_planes.argtypes = [vp, i, i, i, i, i, i, u, i, vp, vp, vp, vp, vp, vp, vp, vp]
            L.xvo_psnr.argtypes = [vp, i, i, i, i, i, vp, vp, i, i, vp, vp, vp, vp, vp]
            L.xvo_intra_angle.argtypes = [i]
            L.xvo_intra_inv_angle.argtypes = [i]
            L.xvo_intra_pred.argtypes = [vp, vp, ctypes.c_int32, i, i, vp]
            L.xvo_intra_refs.argtypes = [vp, i, i, i, i, i, vp, vp, vp]
            L.xvo_intra_frame.argtypes = [vp, i, i, i, u, i, i64, vp, vp, vp, vp, vp]
            L.xvo_intra_frame.restype = ctypes.c_uint64
            L.xvo_deblock_params.argtypes = [i, i, vp, vp]
            L.xvo_deblock_segment.argtypes = [vp, i, i]
            L.xvo_deblock_frame.argtypes = [vp, i, i, i, i, vp, vp, vp, i]
            L.xvo_encode_planes_ex.argtypes = [vp, i, i, i, i, i, i, u, i, u, vp, vp, vp, vp, vp, vp, vp, vp]
            L.xvo_decode_frame.argtypes = [vp, vp, vp, vp, i, i, i, i, vp]
            L.xvo_decode_frame.restype = ctypes.c_uint64
            L.xvo_decode_planes.argtypes = [vp, vp, vp, i, i, i, i, i, i, vp, vp]
            L.xvo_decode_intra_frame.argtypes = [vp, vp, vp, i, i, i, i, vp]
            L.xvo_decode_intra_frame.restype = ctypes.c_uint64
            L.xvo_decode_planes_ex.argtypes = [vp, vp, vp, i, i, i, i, i, i, u, vp, vp]
            L.xvo_unpack.argtypes = [vp, i, i, i, i, i, i, vp, vp]
            L.xvo_ssim_window.argtypes = [vp]
            L.xvo_ssim_image.argtypes = [vp, vp, i, i, ctypes.c_double, vp]
            L.xvo_ssim_image.restype = ctypes.c_double
            L.xvo_ssim.argtypes = [vp, i, i, i, i, i, vp, i, i, vp, vp]
            L.xvo_sa.argtypes = [vp, i, i, i, i, i, vp, i, i, vp, vp]
            L.xvo_sa.restype = ctypes.c_double
            L.xvo_max_threads.restype = i
            L.xvo_set_threads.argtypes = [i]
            _lib = L
        return _lib


def set_threads(n: int) -> None:
    lib().xvo_set_threads(int(n))


def max_threads() -> int:
    return int(lib().xvo_max_threads())


# ----------------------------------------------------------------- C2 / C3
def group_count(bands: int) -> int:
    return int(lib().xvo_group_count(bands))


def group_bands(bands: int) -> list[list[int]]:
    """Band index held by each (group, channel) slot."""
    L = lib()
    return [[int(L.xvo_group_band(bands, g, c)) for c in range(3)] for g in range(group_count(bands))]


def plane_geometry(H: int, W: int, ctu: int) -> tuple[int, int]:
    return -(-H // ctu) * ctu, -(-W // ctu) * ctu


# ----------------------------------------------------------------- C1
def _src(src: np.ndarray):
    src = np.ascontiguousarray(src)
    if src.dtype == np.float32:
        return src, F32
    if src.dtype == np.uint16:
        return src, U16
    raise TypeError("source must be float32 or uint16")


def minmax(src: np.ndarray):
    """(mm[bands,2] float64, nan_count[bands]) for a [bands,T,H,W] cube."""
    src, dt = _src(src)
    bands, T, H, W = src.shape
    mm = np.zeros((bands, 2), np.float64)
    nn = np.zeros(bands, np.int64)
    lib().xvo_minmax(_p(src), dt, bands, T, H, W, _p(mm), _p(nn))
    return mm, nn


def quantize_pack(src: np.ndarray, ctu: int, mm: np.ndarray) -> np.ndarray:
    """u16 planes [G,T,3,Hp,Wp]."""
    src, dt = _src(src)
    bands, T, H, W = src.shape
    Hp, Wp = plane_geometry(H, W, ctu)
    G = group_count(bands)
    out = np.zeros((G, T, 3, Hp, Wp), np.uint16)
    mm = np.ascontiguousarray(mm, np.float64)
    lib().xvo_quantize_pack(_p(src), dt, bands, T, H, W, ctu, _p(mm), _p(out))
    return out


# ----------------------------------------------------------------- C10 / C11
def transform_matrix(N: int) -> np.ndarray:
    T = np.zeros((N, N), np.int32)
    lib().xvo_transform_matrix(N, _p(T))
    return T


def fwd_transform(X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, np.int32)
    C = np.zeros_like(X)
    lib().xvo_fwd_transform(X.shape[0], _p(X), _p(C))
    return C


def inv_transform(C: np.ndarray) -> np.ndarray:
    C = np.ascontiguousarray(C, np.int32)
    R = np.zeros_like(C)
    lib().xvo_inv_transform(C.shape[0], _p(C), _p(R))
    return R


def quant(c, qp: int, log2N: int):
    f = lib().xvo_quant
    return np.vectorize(lambda v: int(f(int(v), qp, log2N)), otypes=[np.int32])(np.asarray(c))


def dequant(level, qp: int, log2N: int):
    f = lib().xvo_dequant
    return np.vectorize(lambda v: int(f(int(v), qp, log2N)), otypes=[np.int32])(np.asarray(level))


# ----------------------------------------------------------------- C7
def lambdas(qp: int) -> tuple[int, int]:
    a = np.zeros(1, np.int64)
    b = np.zeros(1, np.int64)
    lib().xvo_lambdas(qp, _p(a), _p(b))
    return int(a[0]), int(b[0])


def ue_len_se(v: int) -> int:
    return int(lib().xvo_ue_len_se(int(v)))


def mv_bits(mvx_q: int, mvy_q: int) -> int:
    return int(lib().xvo_mv_bits(int(mvx_q), int(mvy_q)))


def mv_cost(mvx_q: int, mvy_q: int, lambda_mv_fp16: int) -> int:
    return int(lib().xvo_mv_cost(int(mvx_q), int(mvy_q), int(lambda_mv_fp16)))


# ----------------------------------------------------------------- C8 / C9
def interp_block(ref: np.ndarray, x0: int, y0: int, w: int, h: int, mvx_q: int, mvy_q: int):
    ref = np.ascontiguousarray(ref, np.uint16)
    out = np.zeros((h, w), np.uint16)
    lib().xvo_interp_block(_p(ref), ref.shape[0], ref.shape[1], x0, y0, w, h, mvx_q, mvy_q, _p(out))
    return out


def hadamard8(d: np.ndarray) -> np.ndarray:
    d = np.ascontiguousarray(d, np.int32)
    out = np.zeros((8, 8), np.int32)
    lib().xvo_hadamard8(_p(d), _p(out))
    return out


def satd(d: np.ndarray) -> int:
    d = np.ascontiguousarray(d, np.int32)
    return int(lib().xvo_satd(_p(d), d.shape[1], d.shape[0]))


# ----------------------------------------------------------------- C7 / C8 per frame
def me_int(cur: np.ndarray, ref: np.ndarray, ctu: int, R: int, lambda_mv_fp16: int):
    """Integer full search on single planes [Hp,Wp] -> (mv_int [nPU,2] px, J [nPU])."""
    cur = np.ascontiguousarray(cur, np.uint16)
    ref = np.ascontiguousarray(ref, np.uint16)
    Hp, Wp = cur.shape
    n = (Hp // ctu) * (Wp // ctu)
    mv = np.zeros((n, 2), np.int16)
    J = np.zeros(n, np.uint32)
    lib().xvo_me_int(_p(cur), _p(ref), Hp, Wp, ctu, R, lambda_mv_fp16, _p(mv), _p(J))
    return mv, J


def me_qpel(cur: np.ndarray, ref: np.ndarray, ctu: int, lambda_mv_fp16: int, mv_int: np.ndarray):
    """Quarter-pel refinement on single planes -> (mv [nPU,2] qpel, J [nPU])."""
    cur = np.ascontiguousarray(cur, np.uint16)
    ref = np.ascontiguousarray(ref, np.uint16)
    mv_int = np.ascontiguousarray(mv_int, np.int16)
    Hp, Wp = cur.shape
    n = (Hp // ctu) * (Wp // ctu)
    mv = np.zeros((n, 2), np.int16)
    J = np.zeros(n, np.uint32)
    lib().xvo_me_qpel(_p(cur), _p(ref), Hp, Wp, ctu, lambda_mv_fp16, _p(mv_int), _p(mv), _p(J))
    return mv, J


def tqr_frame(cur: np.ndarray, ref, mv, ctu: int, tu_mask: int, qp: int):
    """One frame [3,Hp,Wp] -> dict(recon, levels, tu_log2, cu_bits, bits)."""
    cur = np.ascontiguousarray(cur, np.uint16)
    _, Hp, Wp = cur.shape
    n = (Hp // ctu) * (Wp // ctu)
    lf8, _ = lambdas(qp)
    recon = np.zeros_like(cur)
    levels = np.zeros(cur.shape, np.int16)
    tu = np.zeros(n, np.uint8)
    cub = np.zeros(n, np.uint64)
    ref = None if ref is None else np.ascontiguousarray(ref, np.uint16)
    mv = np.zeros((n, 2), np.int16) if mv is None else np.ascontiguousarray(mv, np.int16)
    total = lib().xvo_tqr_frame(_p(cur), _p(ref), _p(mv), Hp, Wp, ctu, tu_mask, qp, lf8,
                                _p(recon), _p(levels), _p(tu), _p(cub))
    return dict(recon=recon, levels=levels, tu_log2=tu, cu_bits=cub, bits=int(total))


# ----------------------------------------------------------------- C4 chain
def encode_planes(planes: np.ndarray, ctu: int, R: int, tu_mask: int, qp: int, want_levels=True, flags: int = 0):
    """The chain over frames per group (flags: INTRA, DEBLOCK)."""
    planes = np.ascontiguousarray(planes, np.uint16)
    G, T, _, Hp, Wp = planes.shape
    n = (Hp // ctu) * (Wp // ctu)
    out = dict(
        recon=np.zeros_like(planes),
        mv=np.zeros((G, T, n, 2), np.int16),
        cost=np.zeros((G, T, n), np.uint32),
        mv_int=np.zeros((G, T, n, 2), np.int16),
        cost_int=np.zeros((G, T, n), np.uint32),
        levels=np.zeros(planes.shape, np.int16) if want_levels else None,
        tu_log2=np.zeros((G, T, n), np.uint8),
        bits=np.zeros((G, T), np.uint64),
    )
    lib().xvo_encode_planes_ex(_p(planes), G, T, Hp, Wp, ctu, R, tu_mask, qp, flags, _p(out["recon"]),
                            _p(out["mv"]), _p(out["cost"]), _p(out["mv_int"]), _p(out["cost_int"]),
                            _p(out["levels"]), _p(out["tu_log2"]), _p(out["bits"]))
    return out


# ------------------------------------- options: frame-0 intra and deblocking
INTRA, DEBLOCK = 1, 2


def intra_angle(mode: int) -> int:
    return int(lib().xvo_intra_angle(mode))


def intra_inv_angle(angle: int) -> int:
    return int(lib().xvo_intra_inv_angle(angle))


def intra_pred(left, top, tl: int, N: int, mode: int) -> np.ndarray:
    """The N x N intra prediction (int32) from left[2N], top[2N] and the corner tl."""
    left = np.ascontiguousarray(left, np.int32)
    top = np.ascontiguousarray(top, np.int32)
    assert left.shape == (2 * N,) and top.shape == (2 * N,)
    out = np.zeros((N, N), np.int32)
    lib().xvo_intra_pred(_p(left), _p(top), int(tl), N, mode, _p(out))
    return out


def intra_refs(plane: np.ndarray, ctu: int, x0: int, y0: int):
    """(left[2N], top[2N], tl) of the CU at (x0, y0) from one plane [Hp,Wp]."""
    plane = np.ascontiguousarray(plane, np.uint16)
    Hp, Wp = plane.shape
    left = np.zeros(2 * ctu, np.int32)
    top = np.zeros(2 * ctu, np.int32)
    tl = np.zeros(1, np.int32)
    lib().xvo_intra_refs(_p(plane), Hp, Wp, ctu, x0, y0, _p(left), _p(top), _p(tl))
    return left, top, int(tl[0])


def intra_frame(cur: np.ndarray, ctu: int, tu_mask: int, qp: int):
    """Frame 0 [3,Hp,Wp] with intra prediction -> dict(recon, levels, tu_log2, mode_mv, cu_bits, bits)."""
    cur = np.ascontiguousarray(cur, np.uint16)
    _, Hp, Wp = cur.shape
    n = (Hp // ctu) * (Wp // ctu)
    lf8, _ = lambdas(qp)
    recon = np.zeros_like(cur)
    levels = np.zeros(cur.shape, np.int16)
    tu = np.zeros(n, np.uint8)
    mm = np.zeros((n, 2), np.int16)
    cub = np.zeros(n, np.uint64)
    total = lib().xvo_intra_frame(_p(cur), Hp, Wp, ctu, tu_mask, qp, lf8, _p(recon), _p(levels), _p(tu), _p(mm),
                                  _p(cub))
    return dict(recon=recon, levels=levels, tu_log2=tu, mode_mv=mm, cu_bits=cub, bits=int(total))


def deblock_params(qp: int, bs: int):
    """(beta, tC) at 10 bits for a QP and boundary strength."""
    b = np.zeros(1, np.int32)
    t = np.zeros(1, np.int32)
    lib().xvo_deblock_params(qp, bs, _p(b), _p(t))
    return int(b[0]), int(t[0])


def deblock_segment(s: np.ndarray, bs: int, qp: int) -> np.ndarray:
    """One 4-line segment s[4][8] (p3 p2 p1 p0 | q0 q1 q2 q3 per line), filtered."""
    s = np.ascontiguousarray(s, np.int32).copy()
    assert s.shape == (4, 8)
    lib().xvo_deblock_segment(_p(s), bs, qp)
    return s


def deblock_frame(rec: np.ndarray, ctu: int, qp: int, tu_log2, levels, mv, intra: bool) -> np.ndarray:
    """A reconstructed frame [3,Hp,Wp] deblocked (a new array)."""
    rec = np.ascontiguousarray(rec, np.uint16).copy()
    _, Hp, Wp = rec.shape
    lib().xvo_deblock_frame(_p(rec), Hp, Wp, ctu, qp, _p(np.ascontiguousarray(tu_log2, np.uint8)),
                            _p(np.ascontiguousarray(levels, np.int16)), _p(np.ascontiguousarray(mv, np.int16)),
                            int(bool(intra)))
    return rec


# ------------------------------------------------------------------ decoder
def decode_frame(levels: np.ndarray, ref, mv: np.ndarray, tu_log2: np.ndarray, ctu: int, qp: int):
    """One frame [3,Hp,Wp] of one group from its levels, vectors and TU sizes
    (ref None: frame 0).  Returns (recon, bits)."""
    levels = np.ascontiguousarray(levels, np.int16)
    _, Hp, Wp = levels.shape
    recon = np.zeros(levels.shape, np.uint16)
    r = None if ref is None else np.ascontiguousarray(ref, np.uint16)
    bits = lib().xvo_decode_frame(_p(levels), _p(r), _p(np.ascontiguousarray(mv, np.int16)),
                                  _p(np.ascontiguousarray(tu_log2, np.uint8)), Hp, Wp, ctu, qp, _p(recon))
    return recon, int(bits)


def decode_planes(levels: np.ndarray, mv: np.ndarray, tu_log2: np.ndarray, ctu: int, qp: int, flags: int = 0):
    """The whole chain [G,T,3,Hp,Wp]: frames in order per group (flags: INTRA,
    DEBLOCK, as the encoder used them).  Returns dict(recon, bits[G,T])."""
    levels = np.ascontiguousarray(levels, np.int16)
    G, T, _, Hp, Wp = levels.shape
    recon = np.zeros(levels.shape, np.uint16)
    bits = np.zeros((G, T), np.uint64)
    lib().xvo_decode_planes_ex(_p(levels), _p(np.ascontiguousarray(mv, np.int16)),
                               _p(np.ascontiguousarray(tu_log2, np.uint8)), G, T, Hp, Wp, ctu, qp, flags, _p(recon),
                               _p(bits))
    return dict(recon=recon, bits=bits)


def decode_intra_frame(levels: np.ndarray, mode_mv: np.ndarray, tu_log2: np.ndarray, ctu: int, qp: int):
    """Frame 0 [3,Hp,Wp] decoded with intra prediction.  Returns (recon, bits)."""
    levels = np.ascontiguousarray(levels, np.int16)
    _, Hp, Wp = levels.shape
    recon = np.zeros(levels.shape, np.uint16)
    bits = lib().xvo_decode_intra_frame(_p(levels), _p(np.ascontiguousarray(mode_mv, np.int16)),
                                        _p(np.ascontiguousarray(tu_log2, np.uint8)), Hp, Wp, ctu, qp, _p(recon))
    return recon, int(bits)


def unpack(recon: np.ndarray, mm: np.ndarray, bands: int, H: int, W: int) -> np.ndarray:
    """The reconstruction in the cube's units: float32 [bands,T,H,W]."""
    recon = np.ascontiguousarray(recon, np.uint16)
    G, T, _, Hp, Wp = recon.shape
    dst = np.zeros((bands, T, H, W), np.float32)
    lib().xvo_unpack(_p(recon), bands, T, H, W, Hp, Wp, _p(np.ascontiguousarray(mm, np.float64)), _p(dst))
    return dst


# ------------------------------------------------------------ SSIM and SA
def ssim_window() -> np.ndarray:
    w = np.zeros(11)
    lib().xvo_ssim_window(_p(w))
    return w


def ssim_image(X: np.ndarray, Y: np.ndarray, L: float):
    """(sum of the SSIM map over the valid windows, windows counted) of one image pair."""
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    n = np.zeros(1, np.int64)
    s = lib().xvo_ssim_image(_p(X), _p(Y), X.shape[0], X.shape[1], float(L), _p(n))
    return s, int(n[0])


def ssim(src: np.ndarray, recon: np.ndarray, mm: np.ndarray) -> np.ndarray:
    """Mean SSIM per band between the cube and the de-quantised reconstruction."""
    src, dt = _src(src)
    bands, T, H, W = src.shape
    Hp, Wp = recon.shape[-2:]
    out = np.zeros(bands)
    lib().xvo_ssim(_p(src), dt, bands, T, H, W, _p(np.ascontiguousarray(recon, np.uint16)), Hp, Wp,
                   _p(np.ascontiguousarray(mm, np.float64)), _p(out))
    return out


def sa(src: np.ndarray, recon: np.ndarray, mm: np.ndarray):
    """(mean spectral angle in radians, pixels counted)."""
    src, dt = _src(src)
    bands, T, H, W = src.shape
    Hp, Wp = recon.shape[-2:]
    n = np.zeros(1, np.int64)
    v = lib().xvo_sa(_p(src), dt, bands, T, H, W, _p(np.ascontiguousarray(recon, np.uint16)), Hp, Wp,
                     _p(np.ascontiguousarray(mm, np.float64)), _p(n))
    return float(v), int(n[0])


# --------------------------------------------------------------------- PCA
def pca_fit(src: np.ndarray):
    """PCA over the bands (the paper's optional transform before packing,
    Sec. 2.1): every pixel (t, y, x) with all bands finite is a sample.
    Returns (mean [bands], components [bands, bands], variance [bands]):
    mean = the sample mean, covariance = (1/n) sum (x - mean)(x - mean)^T,
    components = its eigenvectors as rows in order of decreasing eigenvalue
    (ties: lower index first), each signed so that its entry of largest
    magnitude (the first such) is positive; variance = the eigenvalues."""
    x = np.asarray(src, np.float64).reshape(src.shape[0], -1)
    x = x[:, np.all(np.isfinite(x), axis=0)]
    mean = x.mean(axis=1)
    xc = x - mean[:, None]
    cov = xc @ xc.T / x.shape[1]
    w, v = np.linalg.eigh(cov)
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    comps = v[:, order].T.copy()
    for k in range(comps.shape[0]):
        j = int(np.argmax(np.abs(comps[k])))
        if comps[k, j] < 0:
            comps[k] = -comps[k]
    return mean, comps, w[order]


def pca_project(src: np.ndarray, mean: np.ndarray, comps: np.ndarray, npc: int) -> np.ndarray:
    """z_k = sum_b comps[k, b] (x_b - mean_b) for k < npc, in float64, stored
    as float32 [npc, T, H, W] (NaN where a band is non-finite)."""
    bands = src.shape[0]
    x = np.asarray(src, np.float64).reshape(bands, -1)
    z = comps[:npc] @ (x - mean[:, None])
    return z.reshape((npc,) + src.shape[1:]).astype(np.float32)


def pca_inverse(z: np.ndarray, mean: np.ndarray, comps: np.ndarray) -> np.ndarray:
    """x_b = mean_b + sum_k comps[k, b] z_k over the kept components, float32."""
    npc = z.shape[0]
    zz = np.asarray(z, np.float64).reshape(npc, -1)
    x = mean[:, None] + comps[:npc].T @ zz
    return x.reshape((comps.shape[1],) + z.shape[1:]).astype(np.float32)


# ----------------------------------------------------------------- C14 / C13
def psnr(src: np.ndarray, planes: np.ndarray, recon: np.ndarray, mm: np.ndarray):
    src, dt = _src(src)
    bands, T, H, W = src.shape
    Hp, Wp = planes.shape[-2:]
    planes = np.ascontiguousarray(planes, np.uint16)
    recon = np.ascontiguousarray(recon, np.uint16)
    mm = np.ascontiguousarray(mm, np.float64)
    ps = np.zeros(bands)
    mse = np.zeros(bands)
    sse10 = np.zeros(bands, np.uint64)
    ps10 = np.zeros(bands)
    lib().xvo_psnr(_p(src), dt, bands, T, H, W, _p(planes), _p(recon), Hp, Wp, _p(mm), _p(ps),
                   _p(mse), _p(sse10), _p(ps10))
    return dict(psnr_band=ps, mse_band=mse, sse10_band=sse10, psnr10_band=ps10,
                psnr_mean=float(np.mean(ps)))


def encode_cube(src: np.ndarray, ctu: int, R: int, tu_mask: int, qp: int, mm=None, want_levels=True, flags: int = 0):
    """The whole path on one cube [bands,T,H,W]: A1..A11 (flags: INTRA, DEBLOCK)."""
    if mm is None:
        mm, _ = minmax(src)
    planes = quantize_pack(src, ctu, mm)
    enc = encode_planes(planes, ctu, R, tu_mask, qp, want_levels=want_levels, flags=flags)
    met = psnr(src, planes, enc["recon"], mm)
    bands, T, H, W = src.shape
    total_bits = int(enc["bits"].sum())
    enc.update(met)
    enc.update(mm=mm, planes=planes, total_bits=total_bits,
               bpppb=total_bits / float(H * W * T * bands))
    return enc

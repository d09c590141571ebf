"""Thin Python binding of libxv (include/xv.h): same names, argument
marshalling only.  Every step of the path runs in the CUDA library; this
module converts torch tensors to device pointers and checks status codes.

Raises ``XvError`` on any non-OK status and ``RuntimeError`` when the library
has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

XV_OK, XV_EINVAL, XV_ENOMEM, XV_EBUDGET, XV_ETIMEOUT, XV_EBUSY, XV_ECUDA, XV_ECANCELLED, XV_ENOTFOUND = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
XV_F32, XV_U16 = 0, 1
XV_INTRA, XV_DEBLOCK = 1, 2  # xv_params.flags options (xv_encode_cube and the per-frame calls)
XV_MAX_BANDS = 16

_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64


class xv_params(ctypes.Structure):
    _fields_ = [("bit_depth", _i), ("ctu", _i), ("search_range", _i), ("tu_mask", ctypes.c_uint),
                ("qp", _i), ("lambda_fp8", _i64), ("lambda_mv_fp16", _i64), ("flags", ctypes.c_uint)]


class xv_job(ctypes.Structure):
    _fields_ = [("src", _vp), ("dtype", _i), ("bands", _i), ("T", _i), ("H", _i), ("W", _i),
                ("p", xv_params), ("minmax", _vp), ("minmax_fixed", _i), ("planes", _vp), ("recon", _vp),
                ("mv", _vp), ("cost", _vp), ("levels", _vp), ("tu_log2", _vp), ("bits", _vp)]


class xv_request(ctypes.Structure):
    _fields_ = [("src", _vp), ("dtype", _i), ("bands", _i), ("T", _i), ("H", _i), ("W", _i), ("p", xv_params),
                ("recon_out", _vp), ("mv_out", _vp)]


class xv_djob(ctypes.Structure):
    _fields_ = [("p", xv_params), ("G", _i), ("T", _i), ("Hp", _i), ("Wp", _i), ("levels", _vp), ("mv", _vp),
                ("tu_log2", _vp), ("recon", _vp), ("bits", _vp), ("bands", _i), ("H", _i), ("W", _i),
                ("minmax", _vp), ("dst", _vp)]


class xv_result(ctypes.Structure):
    _fields_ = [("status", _i), ("bands", _i), ("psnr_mean", ctypes.c_double), ("bpppb", ctypes.c_double),
                ("total_bits", ctypes.c_uint64), ("psnr_band", ctypes.c_double * XV_MAX_BANDS),
                ("mse_band", ctypes.c_double * XV_MAX_BANDS), ("sse10_band", ctypes.c_uint64 * XV_MAX_BANDS),
                ("latency_s", ctypes.c_double), ("ctu", _i), ("block_size", _i)]

    def as_dict(self):
        n = self.bands
        return dict(status=self.status, psnr_mean=self.psnr_mean, bpppb=self.bpppb, total_bits=self.total_bits,
                    psnr_band=list(self.psnr_band[:n]), mse_band=list(self.mse_band[:n]),
                    sse10_band=list(self.sse10_band[:n]), latency_s=self.latency_s, ctu=self.ctu,
                    block_size=self.block_size)


class XvError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


_lib = None

_SIGS = {
    "xv_create": [ctypes.POINTER(_vp), _i, ctypes.c_size_t],
    "xv_destroy": [_vp],
    "xv_ctx_bytes": [_vp],
    "xv_params_init": [ctypes.POINTER(xv_params), _i, _i, ctypes.c_uint, _i],
    "xv_plane_geometry": [_i, _i, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "xv_minmax": [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp],
    "xv_quantize_pack": [_vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _i, _vp, _vp],
    "xv_motion_search": [_vp, _vp, _vp, _i, _i64, _i, _i, ctypes.POINTER(xv_params), _vp, _vp, _vp, _vp, _i64, _vp],
    "xv_transform_quant_recon": [_vp, _vp, _vp, _vp, _i, _i64, _i, _i, ctypes.POINTER(xv_params), _i64, _vp, _vp,
                                 _vp, _vp, _i64, _vp],
    "xv_psnr": [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp],
    "xv_decode_frame": [_vp, _vp, _vp, _vp, _vp, _i, _i64, _i, _i, ctypes.POINTER(xv_params), _i64, _vp, _vp, _i64,
                        _vp],
    "xv_intra_frame": [_vp, _vp, _i, _i64, _i, _i, ctypes.POINTER(xv_params), _i64, _vp, _vp, _vp, _vp, _vp, _i64,
                       _vp],
    "xv_deblock_frame": [_vp, _vp, _i, _i64, _i, _i, ctypes.POINTER(xv_params), _i64, _vp, _vp, _vp, _i, _vp],
    "xv_decode_batch": [_vp, ctypes.POINTER(xv_djob), _i, ctypes.POINTER(ctypes.c_uint64), _vp],
    "xv_unpack": [_vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _vp, _vp],
    "xv_pca_fit": [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp],
    "xv_pca_project": [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _i, _vp, _vp],
    "xv_pca_inverse": [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp],
    "xv_ssim": [_vp, _vp, _i, _i, _i, _i, _i, _vp, _i, _i, _vp, _vp, _vp, _vp],
    "xv_sa": [_vp, _vp, _i, _i, _i, _i, _i, _vp, _i, _i, _vp, _vp, ctypes.POINTER(ctypes.c_int64), _vp],
    "xv_psnr_noalloc": [_vp, _i, _i, _i, _i, _i, _vp, _vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp],
    "xv_job_scratch_bytes": [ctypes.POINTER(xv_job)],
    "xv_encode_cube": [_vp, ctypes.POINTER(xv_job), ctypes.POINTER(xv_result), _vp],
    "xv_split_groups": [ctypes.POINTER(xv_job), ctypes.POINTER(_i), ctypes.POINTER(xv_job), ctypes.POINTER(_i)],
    "xv_encode_batch": [_vp, ctypes.POINTER(xv_job), _i, ctypes.POINTER(xv_result), _vp],
    "xv_encode_batch_from_host": [_vp, ctypes.POINTER(xv_job), ctypes.POINTER(_vp), _i, ctypes.POINTER(xv_result),
                                  _vp],
    "xv_serve_start": [_vp, _i, _i],
    "xv_serve_submit": [_vp, ctypes.POINTER(xv_request), ctypes.POINTER(ctypes.c_uint64)],
    "xv_serve_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(xv_result), ctypes.POINTER(_i)],
    "xv_serve_cancel": [_vp, ctypes.c_uint64],
    "xv_serve_stats": [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i),
                       ctypes.POINTER(ctypes.c_size_t)],
    "xv_serve_stop": [_vp],
    "xv_last_batch_kernel_ms": [_vp, ctypes.POINTER(ctypes.c_double)],
    "xv_last_batch_block_size": [_vp, ctypes.POINTER(_i)],
    "xv_last_batch_search_stats": [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)],
    "xv_ctx_launches": [_vp],
    "xv_last_batch_config": [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "xv_last_tune_log": [_vp],
    "xv_measure_peak": [_vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "xv_set_batch_graphs": [_vp, _i],
    "xv_batch_graph_stats": [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)],
    "xv_debug_set_wait_budget": [_vp, ctypes.c_longlong],
    "xv_debug_force_block_size": [_vp, _i],
    "xv_debug_stall_row": [_vp, ctypes.c_longlong],
    "xv_debug_set_window_wait": [_vp, ctypes.c_longlong],
}


def lib():
    """Load libxv.so (it must have been built: ``paper_2506_19656_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libxv.so not built ({LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _i
        L.xv_destroy.restype = None
        L.xv_ctx_bytes.restype = ctypes.c_size_t
        L.xv_job_scratch_bytes.restype = ctypes.c_size_t
        L.xv_ctx_launches.restype = ctypes.c_uint64
        L.xv_last_tune_log.restype = ctypes.c_char_p
        L.xv_last_error.restype = ctypes.c_char_p
        L.xv_status_string.restype = ctypes.c_char_p
        L.xv_status_string.argtypes = [_i]
        _lib = L
    return _lib


def check(status, where):
    if status != XV_OK:
        raise XvError(status, where, lib().xv_last_error().decode())
    return status


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return XV_F32
    if t.dtype == torch.uint16:
        return XV_U16
    raise TypeError("cube must be float32 or uint16")


class Context:
    """An xv_ctx: device scratch, budgets and the batched path's state."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        h = _vp()
        check(lib().xv_create(ctypes.byref(h), device, mem_budget_bytes), "xv_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().xv_destroy(self.handle)
            self.handle = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def bytes(self) -> int:
        return int(lib().xv_ctx_bytes(self.handle))


def xv_params_init(ctu: int, search_range: int, tu_mask: int, qp: int) -> xv_params:
    p = xv_params()
    check(lib().xv_params_init(ctypes.byref(p), ctu, search_range, tu_mask, qp), "xv_params_init")
    return p


def xv_plane_geometry(bands: int, H: int, W: int, ctu: int):
    G, Hp, Wp = _i(), _i(), _i()
    check(lib().xv_plane_geometry(bands, H, W, ctu, ctypes.byref(G), ctypes.byref(Hp), ctypes.byref(Wp)),
          "xv_plane_geometry")
    return G.value, Hp.value, Wp.value


def xv_minmax(ctx: Context, src, minmax, stream=None):
    bands, T, H, W = src.shape
    check(lib().xv_minmax(ctx.handle, _ptr(src), _dtype_code(src), bands, T, H, W, _ptr(minmax), _stream(stream)),
          "xv_minmax")


def xv_quantize_pack(ctx: Context, src, ctu: int, minmax, planes, minmax_fixed: bool = False, stream=None):
    bands, T, H, W = src.shape
    check(lib().xv_quantize_pack(ctx.handle, _ptr(src), _dtype_code(src), bands, T, H, W, ctu, _ptr(minmax),
                                 int(minmax_fixed), _ptr(planes), _stream(stream)), "xv_quantize_pack")


def xv_motion_search(ctx: Context, cur, ref, G: int, plane_gstride: int, Hp: int, Wp: int, p: xv_params, mv,
                     cost=None, mv_int=None, cost_int=None, pu_gstride: int = 0, stream=None):
    check(lib().xv_motion_search(ctx.handle, _ptr(cur), _ptr(ref), G, plane_gstride, Hp, Wp, ctypes.byref(p),
                                 _ptr(mv), _ptr(cost), _ptr(mv_int), _ptr(cost_int), pu_gstride, _stream(stream)),
          "xv_motion_search")


def xv_transform_quant_recon(ctx: Context, cur, ref, mv, G: int, plane_gstride: int, Hp: int, Wp: int,
                             p: xv_params, pu_gstride: int, recon, levels, tu_log2, bits, bits_gstride: int,
                             stream=None):
    check(lib().xv_transform_quant_recon(ctx.handle, _ptr(cur), _ptr(ref), _ptr(mv), G, plane_gstride, Hp, Wp,
                                         ctypes.byref(p), pu_gstride, _ptr(recon), _ptr(levels), _ptr(tu_log2),
                                         _ptr(bits), bits_gstride, _stream(stream)), "xv_transform_quant_recon")


def xv_intra_frame(ctx: Context, cur, G: int, plane_gstride: int, Hp: int, Wp: int, p: xv_params, pu_gstride: int,
                   recon, levels, tu_log2, mode_mv, bits, bits_gstride: int, stream=None):
    check(lib().xv_intra_frame(ctx.handle, _ptr(cur), G, plane_gstride, Hp, Wp, ctypes.byref(p), pu_gstride,
                               _ptr(recon), _ptr(levels), _ptr(tu_log2), _ptr(mode_mv), _ptr(bits), bits_gstride,
                               _stream(stream)), "xv_intra_frame")


def xv_deblock_frame(ctx: Context, recon, G: int, plane_gstride: int, Hp: int, Wp: int, p: xv_params,
                     pu_gstride: int, tu_log2, levels, mv, intra: bool, stream=None):
    check(lib().xv_deblock_frame(ctx.handle, _ptr(recon), G, plane_gstride, Hp, Wp, ctypes.byref(p), pu_gstride,
                                 _ptr(tu_log2), _ptr(levels), _ptr(mv), int(bool(intra)), _stream(stream)),
          "xv_deblock_frame")


def xv_decode_frame(ctx: Context, levels, ref, mv, tu_log2, G: int, plane_gstride: int, Hp: int, Wp: int,
                    p: xv_params, pu_gstride: int, recon, bits, bits_gstride: int, stream=None):
    check(lib().xv_decode_frame(ctx.handle, _ptr(levels), _ptr(ref), _ptr(mv), _ptr(tu_log2), G, plane_gstride, Hp,
                                Wp, ctypes.byref(p), pu_gstride, _ptr(recon), _ptr(bits), bits_gstride,
                                _stream(stream)), "xv_decode_frame")


def make_djob(p: xv_params, levels, mv, tu_log2, recon, bits=None, minmax=None, dst=None, bands=0, H=0,
              W=0) -> xv_djob:
    """levels [G,T,3,Hp,Wp] int16, mv [G,T,nCU,2] int16, tu_log2 [G,T,nCU] uint8, recon like levels (uint16);
    with dst ([bands,T,H,W] float32) and minmax the reconstruction is also written in the cube's units.
    The job holds raw device pointers: the tensors must stay alive while it is used."""
    G, T, _, Hp, Wp = levels.shape
    return xv_djob(p=p, G=G, T=T, Hp=Hp, Wp=Wp, levels=_ptr(levels), mv=_ptr(mv), tu_log2=_ptr(tu_log2),
                   recon=_ptr(recon), bits=_ptr(bits), bands=bands, H=H, W=W, minmax=_ptr(minmax), dst=_ptr(dst))


def xv_decode_batch(ctx: Context, djobs, stream=None) -> list:
    """Decodes the jobs in one persistent launch per CTU size; returns each job's total rate-proxy bits."""
    n = len(djobs)
    arr = (xv_djob * n)(*djobs)
    tot = (ctypes.c_uint64 * n)()
    check(lib().xv_decode_batch(ctx.handle, arr, n, tot, _stream(stream)), "xv_decode_batch")
    return list(tot)


def xv_unpack(ctx: Context, recon, bands: int, H: int, W: int, minmax, dst, stream=None):
    G, T, _, Hp, Wp = recon.shape
    check(lib().xv_unpack(ctx.handle, _ptr(recon), bands, T, H, W, Hp, Wp, _ptr(minmax), _ptr(dst), _stream(stream)),
          "xv_unpack")


def xv_pca_fit(ctx: Context, src, stream=None):
    """(mean [bands], components [bands, bands], variance [bands]) as numpy float64."""
    import numpy as np
    bands, T, H, W = src.shape
    mean = np.zeros(bands)
    comps = np.zeros((bands, bands))
    var = np.zeros(bands)
    check(lib().xv_pca_fit(ctx.handle, _ptr(src), _dtype_code(src), bands, T, H, W, mean.ctypes.data,
                           comps.ctypes.data, var.ctypes.data, _stream(stream)), "xv_pca_fit")
    return mean, comps, var


def xv_pca_project(ctx: Context, src, mean, comps, npc: int, dst, stream=None):
    import numpy as np
    bands, T, H, W = src.shape
    m = np.ascontiguousarray(mean, np.float64)
    cmp = np.ascontiguousarray(comps, np.float64)
    check(lib().xv_pca_project(ctx.handle, _ptr(src), _dtype_code(src), bands, T, H, W, m.ctypes.data,
                               cmp.ctypes.data, npc, _ptr(dst), _stream(stream)), "xv_pca_project")


def xv_pca_inverse(ctx: Context, z, mean, comps, dst, stream=None):
    import numpy as np
    npc, T, H, W = z.shape
    bands = dst.shape[0]
    m = np.ascontiguousarray(mean, np.float64)
    cmp = np.ascontiguousarray(comps, np.float64)
    check(lib().xv_pca_inverse(ctx.handle, _ptr(z), npc, bands, T, H, W, m.ctypes.data, cmp.ctypes.data, _ptr(dst),
                               _stream(stream)), "xv_pca_inverse")


def xv_ssim(ctx: Context, src, recon, minmax, stream=None) -> dict:
    """SSIM per band and their mean; src [bands,T,H,W] (float32/uint16), recon [G,T,3,Hp,Wp]."""
    bands, T, H, W = src.shape
    Hp, Wp = recon.shape[-2:]
    band = (ctypes.c_double * bands)()
    mean = ctypes.c_double()
    check(lib().xv_ssim(ctx.handle, _ptr(src), _dtype_code(src), bands, T, H, W, _ptr(recon), Hp, Wp, _ptr(minmax),
                        band, ctypes.byref(mean), _stream(stream)), "xv_ssim")
    return dict(ssim_band=list(band), ssim_mean=mean.value)


def xv_sa(ctx: Context, src, recon, minmax, stream=None):
    """(mean spectral angle in radians, pixels counted)."""
    bands, T, H, W = src.shape
    Hp, Wp = recon.shape[-2:]
    v, n = ctypes.c_double(), ctypes.c_int64()
    check(lib().xv_sa(ctx.handle, _ptr(src), _dtype_code(src), bands, T, H, W, _ptr(recon), Hp, Wp, _ptr(minmax),
                      ctypes.byref(v), ctypes.byref(n), _stream(stream)), "xv_sa")
    return v.value, n.value


def xv_psnr(ctx: Context, src, planes, recon, minmax, stream=None):
    """Returns dict(psnr_band, mse_band, sse10_band, psnr_mean) (host values)."""
    bands, T, H, W = src.shape
    Hp, Wp = planes.shape[-2:]
    ps = (ctypes.c_double * bands)()
    mse = (ctypes.c_double * bands)()
    s10 = (ctypes.c_uint64 * bands)()
    mean = ctypes.c_double()
    check(lib().xv_psnr(ctx.handle, _ptr(src), _dtype_code(src), bands, T, H, W, _ptr(planes), _ptr(recon), Hp, Wp,
                        _ptr(minmax), ps, mse, s10, ctypes.byref(mean), _stream(stream)), "xv_psnr")
    return dict(psnr_band=list(ps), mse_band=list(mse), sse10_band=list(s10), psnr_mean=mean.value)


def xv_psnr_noalloc(src, planes, recon, minmax, stream=None):
    """xv_psnr without a context or any device allocation (fixed scratch in
    the library); same results.  Returns dict(psnr_band, mse_band, sse10_band,
    psnr_mean)."""
    bands, T, H, W = src.shape
    Hp, Wp = planes.shape[-2:]
    ps = (ctypes.c_double * bands)()
    mse = (ctypes.c_double * bands)()
    s10 = (ctypes.c_uint64 * bands)()
    mean = ctypes.c_double()
    check(lib().xv_psnr_noalloc(_ptr(src), _dtype_code(src), bands, T, H, W, _ptr(planes), _ptr(recon), Hp, Wp,
                                _ptr(minmax), ps, mse, s10, ctypes.byref(mean), _stream(stream)), "xv_psnr_noalloc")
    return dict(psnr_band=list(ps), mse_band=list(mse), sse10_band=list(s10), psnr_mean=mean.value)


def make_job(src, p: xv_params, planes, recon, minmax=None, minmax_fixed=False, mv=None, cost=None, levels=None,
             tu_log2=None, bits=None) -> xv_job:
    """The job of one cube.  It holds raw device pointers: the tensors must stay alive while it is used."""
    bands, T, H, W = src.shape
    return xv_job(src=_ptr(src), dtype=_dtype_code(src), bands=bands, T=T, H=H, W=W, p=p, minmax=_ptr(minmax),
                  minmax_fixed=int(minmax_fixed), planes=_ptr(planes), recon=_ptr(recon), mv=_ptr(mv),
                  cost=_ptr(cost), levels=_ptr(levels), tu_log2=_ptr(tu_log2), bits=_ptr(bits))


def xv_split_groups(job: xv_job, qps) -> list:
    """One job per 3-band group of `job`, group g at QP qps[g] (views of the
    whole job's buffers)."""
    G = (job.bands + 2) // 3
    q = (_i * G)(*[int(v) for v in qps])
    out = (xv_job * G)()
    n = _i()
    check(lib().xv_split_groups(ctypes.byref(job), q, out, ctypes.byref(n)), "xv_split_groups")
    return [out[i] for i in range(n.value)]


def xv_encode_cube(ctx: Context, job: xv_job, stream=None) -> dict:
    r = xv_result()
    check(lib().xv_encode_cube(ctx.handle, ctypes.byref(job), ctypes.byref(r), _stream(stream)), "xv_encode_cube")
    return r.as_dict()


def xv_encode_batch(ctx: Context, jobs, stream=None) -> list:
    n = len(jobs)
    arr = (xv_job * n)(*jobs)
    res = (xv_result * n)()
    check(lib().xv_encode_batch(ctx.handle, arr, n, res, _stream(stream)), "xv_encode_batch")
    return [r.as_dict() for r in res]


PEAK_KINDS = {0: "sad", 1: "fp32_absdiff", 2: "sad_fp32_mix", 3: "imad"}


def xv_measure_peak(ctx: Context, kind: int) -> tuple:
    """(operations per second, ms of the best run) of microbenchmark `kind`
    (PEAK_KINDS: 0-2 abs-diff-accumulates, 3 integer multiply-adds)."""
    r = ctypes.c_double()
    ms = ctypes.c_double()
    check(lib().xv_measure_peak(ctx.handle, kind, ctypes.byref(r), ctypes.byref(ms)), "xv_measure_peak")
    return r.value, ms.value


def xv_last_batch_config(ctx: Context, ctu: int) -> tuple:
    """(block size or 1 for the per-frame mode, resident-block cap per SM or 0)
    of CTU class `ctu` in the last xv_encode_batch."""
    nt, per = _i(), _i()
    check(lib().xv_last_batch_config(ctx.handle, ctu, ctypes.byref(nt), ctypes.byref(per)), "xv_last_batch_config")
    return nt.value, per.value


def xv_last_tune_log(ctx: Context) -> str:
    """The autotuner's last candidate timings ("ctu32 nt128 per4 12.345;...")."""
    return lib().xv_last_tune_log(ctx.handle).decode()


def xv_encode_batch_from_host(ctx: Context, jobs, host_srcs, stream=None) -> list:
    """xv_encode_batch after copying each host cube (a CPU tensor, pinned for
    an asynchronous copy, or None) into its job's device source buffer."""
    n = len(jobs)
    arr = (xv_job * n)(*jobs)
    hs = (_vp * n)(*[None if h is None else h.data_ptr() for h in host_srcs])
    res = (xv_result * n)()
    check(lib().xv_encode_batch_from_host(ctx.handle, arr, hs, n, res, _stream(stream)), "xv_encode_batch_from_host")
    return [r.as_dict() for r in res]


def xv_serve_start(ctx: Context, max_slots: int, frames_per_tick: int):
    check(lib().xv_serve_start(ctx.handle, max_slots, frames_per_tick), "xv_serve_start")


def make_request(src_host, p: xv_params, recon_out=None, mv_out=None) -> xv_request:
    """src_host: a CPU torch tensor [bands, T, H, W] (pin it for an asynchronous upload)."""
    bands, T, H, W = src_host.shape
    return xv_request(src=_ptr(src_host), dtype=_dtype_code(src_host), bands=bands, T=T, H=H, W=W, p=p,
                      recon_out=_ptr(recon_out), mv_out=_ptr(mv_out))


def xv_serve_submit(ctx: Context, req: xv_request) -> int:
    t = ctypes.c_uint64()
    check(lib().xv_serve_submit(ctx.handle, ctypes.byref(req), ctypes.byref(t)), "xv_serve_submit")
    return t.value


def xv_serve_poll(ctx: Context, ticket: int):
    """(done, result dict or None); a failed request's result carries its message as "error"."""
    r = xv_result()
    done = _i()
    check(lib().xv_serve_poll(ctx.handle, ticket, ctypes.byref(r), ctypes.byref(done)), "xv_serve_poll")
    if not done.value:
        return False, None
    res = r.as_dict()
    if res["status"] != XV_OK:
        res["error"] = lib().xv_last_error().decode()
    return True, res


def xv_serve_cancel(ctx: Context, ticket: int):
    check(lib().xv_serve_cancel(ctx.handle, ticket), "xv_serve_cancel")


def xv_serve_stats(ctx: Context):
    t, ms, pk, b = ctypes.c_uint64(), ctypes.c_double(), _i(), ctypes.c_size_t()
    check(lib().xv_serve_stats(ctx.handle, ctypes.byref(t), ctypes.byref(ms), ctypes.byref(pk), ctypes.byref(b)),
          "xv_serve_stats")
    return dict(ticks=t.value, kernel_ms=ms.value, peak_resident=pk.value, bytes_in_use=b.value)


def xv_serve_stop(ctx: Context):
    check(lib().xv_serve_stop(ctx.handle), "xv_serve_stop")


def xv_last_batch_kernel_ms(ctx: Context) -> float:
    ms = ctypes.c_double()
    check(lib().xv_last_batch_kernel_ms(ctx.handle, ctypes.byref(ms)), "xv_last_batch_kernel_ms")
    return ms.value


def xv_last_batch_block_size(ctx: Context) -> int:
    nt = _i()
    check(lib().xv_last_batch_block_size(ctx.handle, ctypes.byref(nt)), "xv_last_batch_block_size")
    return nt.value


def xv_last_batch_search_stats(ctx: Context) -> tuple[int, int]:
    """(candidates evaluated exactly, candidates of the full search) of the
    last xv_encode_batch."""
    ex, full = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().xv_last_batch_search_stats(ctx.handle, ctypes.byref(ex), ctypes.byref(full)),
          "xv_last_batch_search_stats")
    return ex.value, full.value


def xv_set_batch_graphs(ctx: Context, enable: bool):
    check(lib().xv_set_batch_graphs(ctx.handle, int(enable)), "xv_set_batch_graphs")


def xv_batch_graph_stats(ctx: Context):
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().xv_batch_graph_stats(ctx.handle, ctypes.byref(a), ctypes.byref(b)), "xv_batch_graph_stats")
    return a.value, b.value


def xv_ctx_launches(ctx: Context) -> int:
    return int(lib().xv_ctx_launches(ctx.handle))


def xv_debug_set_wait_budget(ctx: Context, cycles: int):
    check(lib().xv_debug_set_wait_budget(ctx.handle, cycles), "xv_debug_set_wait_budget")


def xv_debug_force_block_size(ctx: Context, block_size: int):
    check(lib().xv_debug_force_block_size(ctx.handle, block_size), "xv_debug_force_block_size")


def xv_debug_set_window_wait(ctx: Context, polls: int):
    check(lib().xv_debug_set_window_wait(ctx.handle, polls), "xv_debug_set_window_wait")


def xv_debug_stall_row(ctx: Context, row: int):
    check(lib().xv_debug_stall_row(ctx.handle, row), "xv_debug_stall_row")


# ------------------------------------------------------------ tensor helpers
def alloc_cube_buffers(bands: int, T: int, H: int, W: int, p: xv_params, device="cuda", levels=True):
    """Device buffers of one cube (planes, recon, mv, cost, levels, tu_log2, bits, minmax)."""
    import torch
    G, Hp, Wp = xv_plane_geometry(bands, H, W, p.ctu)
    npu = (Hp // p.ctu) * (Wp // p.ctu)
    kw = dict(device=device)
    return dict(
        planes=torch.empty((G, T, 3, Hp, Wp), dtype=torch.uint16, **kw),
        recon=torch.empty((G, T, 3, Hp, Wp), dtype=torch.uint16, **kw),
        mv=torch.empty((G, T, npu, 2), dtype=torch.int16, **kw),
        cost=torch.empty((G, T, npu), dtype=torch.int32, **kw),
        levels=torch.empty((G, T, 3, Hp, Wp), dtype=torch.int16, **kw) if levels else None,
        tu_log2=torch.empty((G, T, npu), dtype=torch.uint8, **kw),
        bits=torch.empty((G, T), dtype=torch.int64, **kw),
        minmax=torch.empty((bands, 2), dtype=torch.float64, **kw),
    )

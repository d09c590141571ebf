"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/xv.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(xv_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libxv():
    from paper_2506_19656_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("xv_quantize_pack", "xv_motion_search", "xv_transform_quant_recon", "xv_psnr",
                     "xv_encode_cube", "xv_encode_batch"):
        assert required in names


def test_every_declared_symbol_is_exported(libxv):
    missing = [n for n in declared_functions() if not hasattr(libxv, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2506_19656_gb300 import xv
    bound = set(xv._SIGS) | {"xv_last_error", "xv_status_string"}
    assert set(declared_functions()) <= bound


def test_params_validation_without_gpu(libxv):
    from paper_2506_19656_gb300 import xv
    p = xv.xv_params_init(16, 32, 0b11100, 27)
    assert p.lambda_fp8 == round(256 * 0.57 * 2 ** (15 / 3))
    for bad in [(12, 32, 0b11100, 27), (16, 0, 0b11100, 27), (16, 32, 0b1000000, 27), (8, 8, 0b110000, 27),
                (16, 32, 0b11100, 52), (64, 65, 0b100, 22)]:
        with pytest.raises(xv.XvError) as e:
            xv.xv_params_init(*bad)
        assert e.value.status == xv.XV_EINVAL
    assert xv.xv_plane_geometry(10, 721, 1440, 32) == (4, 736, 1440)


def test_widened_entry_points_reject_bad_arguments_without_gpu(libxv):
    """The decoder, metric and PCA calls validate before touching the device:
    a NULL context or malformed shapes return XV_EINVAL (-1) with a message."""
    lib = libxv
    vp, i, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.xv_decode_frame.restype = i
    lib.xv_unpack.restype = i
    lib.xv_ssim.restype = i
    lib.xv_sa.restype = i
    lib.xv_pca_fit.restype = i
    lib.xv_pca_project.restype = i
    lib.xv_pca_inverse.restype = i
    lib.xv_decode_batch.restype = i
    null = vp(0)
    assert lib.xv_decode_frame(null, null, null, null, null, i(1), i64(0), i(16), i(16), null, i64(1), null, null,
                               i64(1), null) == -1
    assert lib.xv_decode_batch(null, null, i(1), null, null) == -1
    assert lib.xv_unpack(null, null, i(3), i(1), i(8), i(8), i(8), i(8), null, null, null) == -1
    assert lib.xv_ssim(null, null, i(0), i(3), i(1), i(8), i(8), null, i(8), i(8), null, null, null, null) == -1
    assert lib.xv_sa(null, null, i(0), i(3), i(1), i(8), i(8), null, i(8), i(8), null, null, null, null) == -1
    assert lib.xv_pca_fit(null, null, i(0), i(3), i(1), i(8), i(8), null, null, null, null) == -1
    assert lib.xv_pca_project(null, null, i(0), i(3), i(1), i(8), i(8), null, null, i(2), null, null) == -1
    assert lib.xv_pca_inverse(null, null, i(2), i(3), i(1), i(8), i(8), null, null, null, null) == -1


def test_option_entry_points_and_params_layout_without_gpu(libxv):
    """xv_intra_frame and xv_deblock_frame validate before the device (NULL
    context -> XV_EINVAL); xv_params ends with the options word, which
    xv_params_init sets to 0, and the option bits are the header's."""
    from paper_2506_19656_gb300 import xv
    lib = libxv
    vp, i, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.xv_intra_frame.restype = i
    lib.xv_deblock_frame.restype = i
    null = vp(0)
    assert lib.xv_intra_frame(null, null, i(1), i64(768), i(16), i(16), null, i64(1), null, null, null, null, null,
                              i64(1), null) == -1
    assert lib.xv_deblock_frame(null, null, i(1), i64(768), i(16), i(16), null, i64(1), null, null, null, i(0),
                                null) == -1
    assert xv.xv_params.flags.offset == 40 and ctypes.sizeof(xv.xv_params) == 48
    p = xv.xv_params_init(16, 32, 0b11100, 27)
    assert p.flags == 0
    header = open(os.path.join(ROOT, "include", "xv.h")).read()
    assert re.search(r"#define XV_INTRA 1u", header) and re.search(r"#define XV_DEBLOCK 2u", header)
    assert (xv.XV_INTRA, xv.XV_DEBLOCK) == (1, 2)

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

"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point include/dvgo.h declares, and rejects invalid arguments on
the host (no kernel is launched, so no GPU is needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dvgo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dvgo_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_05085_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("dvgo_sample_grid_fwd", "dvgo_sample_grid_bwd", "dvgo_composite_rgb_fwd",
                 "dvgo_composite_bwd", "dvgo_distortion_fwd", "dvgo_distortion_bwd",
                 "dvgo_adam_step", "dvgo_rgbnet_fwd", "dvgo_rgbnet_bwd", "dvgo_sample_rays",
                 "dvgo_tv_add_grad", "dvgo_alpha_weights_fwd"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_2206_05085_gb300 import _lib
    assert sorted(_lib.exported_names()) == sorted(set(_lib.exported_names()))
    assert set(_lib.exported_names()) <= set(_declared())


def test_host_validation_without_gpu(lib):
    lib.dvgo_distortion_fwd.restype = ctypes.c_int
    lib.dvgo_distortion_fwd.argtypes = [ctypes.c_void_p] * 5 + [ctypes.c_int64, ctypes.c_void_p,
                                                                 ctypes.c_void_p]
    assert lib.dvgo_distortion_fwd(None, None, None, None, None, 4, None, None) == -1
    lib.dvgo_sample_rays_workspace_size.restype = ctypes.c_size_t
    lib.dvgo_sample_rays_workspace_size.argtypes = [ctypes.c_int64]
    assert lib.dvgo_sample_rays_workspace_size(1000) >= 4 * 1001
    lib.dvgo_grid_bricked_elems.restype = ctypes.c_int64
    G = (ctypes.c_int32 * 3)(160, 160, 160)
    assert lib.dvgo_grid_bricked_elems(G, 12) == 20 ** 3 * 512 * 12
    G2 = (ctypes.c_int32 * 3)(9, 8, 17)
    assert lib.dvgo_grid_bricked_elems(G2, 1) == 2 * 1 * 3 * 512
    lib.dvgo_status_string.restype = ctypes.c_char_p
    assert lib.dvgo_status_string(-5) == b"bounded device-side wait gave up"
    lib.dvgo_rgbnet_fwd.restype = ctypes.c_int
    # bad precision enum with valid-looking (never dereferenced) pointers
    p = ctypes.c_void_p(16)
    lib.dvgo_rgbnet_fwd.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_void_p,
                                                             ctypes.c_void_p, ctypes.c_int,
                                                             ctypes.c_void_p, ctypes.c_void_p]
    assert lib.dvgo_rgbnet_fwd(p, p, p, None, 10, None, p, 9, p, None) == -1
    # the tensor-core FP32 form needs its act buffer
    assert lib.dvgo_rgbnet_fwd(p, p, p, None, 10, None, p, 2, p, None) == -1
    lib.dvgo_rgbnet_act_bytes.restype = ctypes.c_int64
    lib.dvgo_rgbnet_act_bytes.argtypes = [ctypes.c_int64, ctypes.c_int]
    assert lib.dvgo_rgbnet_act_bytes(10, 0) == 10 * 1024
    assert lib.dvgo_rgbnet_act_bytes(300, 2) == 256 + 3 * 90112 + 152 * 22019 * 4
    assert lib.dvgo_rgbnet_act_bytes(0, 2) == 256 + 152 * 22019 * 4
    # the BF16 form runs the same tensor-core kernels and needs the same buffer
    assert lib.dvgo_rgbnet_act_bytes(10, 1) == 256 + 90112 + 152 * 22019 * 4
    assert lib.dvgo_rgbnet_fwd(p, p, p, None, 10, None, p, 1, p, None) == -1
    assert lib.dvgo_rgbnet_act_bytes(-1, 0) == -1
    assert lib.dvgo_rgbnet_act_bytes(5, 7) == -1
    assert lib.dvgo_status_string(-8) == b"value outside the range of a split-FP16 operand"


def test_tv_rejects_a_grid_too_large_for_its_offsets(lib):
    """The TV kernel forms neighbour slots as int32 offsets: a grid whose layer
    of bricks does not fit is refused on the host, before any launch."""
    from paper_2206_05085_gb300 import _lib
    lib.dvgo_tv_add_grad_multi.restype = ctypes.c_int
    lib.dvgo_tv_add_grad_multi.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_float, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]
    one = _lib.TvGrid(16, 0, 1, 1.0, None, 16)
    G = (ctypes.c_int32 * 3)(20000, 20000, 8)
    assert lib.dvgo_tv_add_grad_multi(ctypes.byref(one), 1, G, 1.0, 1, None, None, None) == -1

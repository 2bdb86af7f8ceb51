"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function include/websplat.h declares, and
rejects bad arguments synchronously, before any CUDA call."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ws_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    import shutil
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    from paper_2602_03207_gb300 import build, capi
    build.build()
    return capi.lib()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"ws_preprocess", "ws_cull", "ws_sort", "ws_rasterize"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version_and_status_strings(lib):
    from paper_2602_03207_gb300 import capi
    assert lib.ws_abi_version() == capi.WS_ABI_VERSION == 2
    assert lib.ws_status_string(0) == b"ok"
    assert lib.ws_status_string(3) == b"key capacity exceeded"


def test_workspace_and_argument_checks(lib):
    from paper_2602_03207_gb300 import capi
    from paper_2602_03207_gb300 import synthetic as S
    cam = capi.camera(S.small_forward()[1])
    cfg = capi.config()
    assert capi.ws_workspace_bytes(1000, 4000, cam, cfg) > 0
    assert capi.ws_workspace_bytes(-1, 4000, cam, cfg) == 0
    assert capi.ws_workspace_bytes(10, 1 << 31, cam, cfg) == 0
    bad = capi.config(tile=12)
    assert capi.ws_workspace_bytes(10, 10, cam, bad) == 0
    bad = capi.config(digit_bits=12)
    assert capi.ws_workspace_bytes(10, 10, cam, bad) == 0
    cam0 = capi.camera(S.small_forward()[1])
    cam0.width = 0
    assert capi.ws_workspace_bytes(10, 10, cam0, cfg) == 0
    # synchronous argument errors (returned before any launch)
    st = lib.ws_preprocess(-1, None, None, None, None, None, C.byref(cam), C.byref(cfg),
                           None, None, None, None, None)
    assert st == capi.WS_ERR_INVALID_ARG
    st = lib.ws_preprocess(10, None, None, None, None, None, C.byref(cam), C.byref(cfg),
                           None, None, None, None, None)
    assert st == capi.WS_ERR_INVALID_ARG
    misaligned = C.c_void_p(0x1004)
    st = lib.ws_preprocess(10, misaligned, misaligned, misaligned, misaligned, misaligned, C.byref(cam),
                           C.byref(cfg), misaligned, misaligned, misaligned, misaligned, None)
    assert st == capi.WS_ERR_INVALID_ARG
    in_alt = C.c_int32(0)
    st = lib.ws_sort(None, 10, 0, 65, None, None, None, None, C.byref(cfg), None, C.byref(in_alt), None)
    assert st == capi.WS_ERR_INVALID_ARG
    st = lib.ws_sort(None, 10, 0, 40, None, None, None, None, C.byref(capi.config(digit_bits=3)), None,
                     C.byref(in_alt), None)
    assert st == capi.WS_ERR_UNSUPPORTED


def test_key_layout_host_logic():
    from paper_2602_03207_gb300 import render
    assert render.tile_grid(1920, 1080, 16) == (120, 68)
    assert render.key_end_bit(1920, 1080, 16) == 31 + 13
    assert render.key_end_bit(3840, 2160, 16) == 31 + 15
    assert render.key_end_bit(256, 256, 16) == 31 + 8
    assert render.key_end_bit(16, 16, 16) == 31


def test_null_device_pointers_are_rejected(lib):
    """Every compute entry point, called with a positive count, valid camera
    and configuration and null device pointers, returns WS_ERR_INVALID_ARG
    before touching the GPU."""
    from paper_2602_03207_gb300 import capi
    from paper_2602_03207_gb300 import synthetic as S
    cam = capi.camera(S.small_forward()[1])
    cfg = capi.config()
    names = ["ws_preprocess", "ws_cull", "ws_sort", "ws_rasterize", "ws_preprocess_packed",
             "ws_rasterize_packed", "ws_render_quads", "ws_rasterize_backward", "ws_sort_noalloc",
             "ws_preprocess_batch", "ws_cull_batch", "ws_rasterize_batch", "ws_rasterize_backward_batch",
             "ws_image_residual", "ws_read_status"]
    for nm in names:
        fn = getattr(lib, nm)
        args = []
        ints32 = iter([0, 40, 8] if nm.startswith("ws_sort") else [])  # begin, end, digit bits
        for t in fn.argtypes:
            if t is C.c_int64:
                args.append(16)
            elif t is C.c_int32:
                args.append(next(ints32, 1))
            elif t is C.POINTER(C.c_int32):
                args.append(C.byref(C.c_int32(0)))
            elif t is C.POINTER(C.c_uint32):
                args.append(C.byref(C.c_uint32(0)))
            elif "camera" in repr(t).lower():
                args.append(C.byref(cam))
            elif "config" in repr(t).lower():
                args.append(C.byref(cfg))
            else:
                args.append(None)
        assert fn(*args) == capi.WS_ERR_INVALID_ARG, nm


def test_binding_constants_match_the_header():
    """The Python binding's flag and status constants equal the header's
    #defines and enum values."""
    from paper_2602_03207_gb300 import capi
    src = open(os.path.join(ROOT, "include", "websplat.h")).read()
    defines = {m.group(1): int(m.group(2), 0)
               for m in re.finditer(r"#define\s+(WS_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+|\d+)u?\b", src)}
    checked = 0
    for name, value in defines.items():
        if hasattr(capi, name):
            assert getattr(capi, name) == value, name
            checked += 1
    assert checked >= 5, sorted(defines)

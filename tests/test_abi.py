"""The C ABI library loads on a machine without a GPU, exports every function
that include/fss.h declares, and its host-only calls (sizes, layout,
argument validation) behave as documented.  No call here reaches the GPU:
every call either needs no device or is rejected before any launch."""
import ctypes as C
import os
import re

import pytest

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300.build import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fss.h")


@pytest.fixture(scope="module")
def lib():
    build()
    return L.lib()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:fss_status|const char \*)\s*(fss_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(L.EXPORTS)


def test_library_exports_every_declared_function(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_header_constants_match_binding():
    text = open(HEADER).read()
    assert f"#define FSS_MAX_CAMS {L.FSS_MAX_CAMS}" in text
    assert f"#define FSS_MAX_K {L.FSS_MAX_K}" in text
    m = re.search(r"#define FSS_STATIC_SCRATCH_BYTES \((\d+)u << (\d+)\)", text)
    assert m and int(m.group(1)) << int(m.group(2)) == L.FSS_STATIC_SCRATCH_BYTES


def _cam(w=64, h=48):
    c = (L.fss_camera * 1)()
    c[0].fx = c[0].fy = 50.0
    c[0].cx, c[0].cy = w / 2, h / 2
    c[0].width, c[0].height = w, h
    for k, v in enumerate([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 3]):
        c[0].viewmat[k] = v
    c[0].near_plane = 0.2
    return c


def test_default_params_and_sizes(lib):
    p = L.fss_default_params()
    assert (p.tile_size, p.K, p.bin_mode, p.stop_rule, p.C) == (16, 8, L.FSS_BIN_ACCU, L.FSS_STOP_TMIN, 16)
    cams = _cam()
    ws = L.fss_workspace_size(p, cams, 1, 1000, 5000)
    assert ws % 256 == 0 and ws > 0
    # every region lies inside the workspace, 256-byte aligned, without overlap
    spans = []
    for r in range(L.N_REGIONS):
        off, size = L.fss_workspace_region(p, cams, 1, 1000, 5000, r)
        assert off + size <= ws
        if r == L.REG_COUNTERS:  # the counters sit inside the status block
            s0, n0 = L.fss_workspace_region(p, cams, 1, 1000, 5000, L.REG_STATUS)
            assert s0 <= off and off + size <= s0 + n0
        elif size:
            assert off % 256 == 0
            spans.append((off, off + size))
    spans.sort()
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    # pairs cost 24 bytes each (list, sort scratch, warp mask)
    assert L.fss_workspace_size(p, cams, 1, 1000, 5000 + 256 * 100) - ws == 256 * 100 * 24
    sv = L.fss_saved_size(p, cams, 1)
    assert sv == 2 * 64 * 48 * 8 * 4 + 64 * 48 * 4


@pytest.mark.parametrize("field,value,status", [
    ("tile_size", 12, L.FSS_ERR_UNSUPPORTED), ("K", 33, L.FSS_ERR_UNSUPPORTED),
    ("C", 6, L.FSS_ERR_UNSUPPORTED), ("alpha_min", 0.0, L.FSS_ERR_INVALID_ARG),
    ("alpha_max", 1.0, L.FSS_ERR_INVALID_ARG), ("schedule", 5, L.FSS_ERR_INVALID_ARG),
    ("bin_mode", 7, L.FSS_ERR_INVALID_ARG), ("select", 2, L.FSS_ERR_INVALID_ARG),
    ("renorm", 2, L.FSS_ERR_INVALID_ARG)])
def test_invalid_params_are_rejected_before_any_launch(lib, field, value, status):
    p = L.fss_default_params()
    setattr(p, field, value)
    out = C.c_size_t()
    assert lib.fss_workspace_size(C.byref(p), _cam(), 1, 10, 10, C.byref(out)) == status
    assert L.last_error()
    # compute calls validate the same way and return before touching a device
    assert lib.fss_project_bin(C.byref(p), _cam(), 1, 10, None, None, None, None, None, 10, None) == status


def test_renormalisation_needs_top_k(lib):
    p = L.fss_default_params()
    p.K, p.renorm = 0, 1
    out = C.c_size_t()
    assert lib.fss_workspace_size(C.byref(p), _cam(), 1, 10, 10, C.byref(out)) == L.FSS_ERR_INVALID_ARG
    assert "renorm" in L.last_error()
    p.K = 4
    assert lib.fss_workspace_size(C.byref(p), _cam(), 1, 10, 10, C.byref(out)) == L.FSS_OK


def test_bad_camera_and_sizes_are_rejected(lib):
    p = L.fss_default_params()
    out = C.c_size_t()
    cams = _cam()
    cams[0].fx = 0.0
    assert lib.fss_workspace_size(C.byref(p), cams, 1, 10, 10, C.byref(out)) == L.FSS_ERR_INVALID_ARG
    assert lib.fss_workspace_size(C.byref(p), _cam(), 0, 10, 10, C.byref(out)) == L.FSS_ERR_UNSUPPORTED
    assert lib.fss_workspace_size(C.byref(p), _cam(), 1, -1, 10, C.byref(out)) == L.FSS_ERR_UNSUPPORTED
    assert lib.fss_workspace_size(C.byref(p), _cam(), 1, 10, 1 << 31, C.byref(out)) == L.FSS_ERR_UNSUPPORTED
    assert lib.fss_project_bin(C.byref(L.fss_default_params()), _cam(), 1, 10, None, None, None, None, None, 10,
                               None) == L.FSS_ERR_INVALID_ARG  # NULL workspace


def test_static_forward_rejects_oversized_frames_on_the_host(lib):
    p = L.fss_default_params()
    cams = _cam()
    big = L.FSS_STATIC_SCRATCH_BYTES // 16
    assert L.fss_workspace_size(p, cams, 1, 1000, big) > L.FSS_STATIC_SCRATCH_BYTES
    n = C.c_int64()
    s = lib.fss_forward_static(C.byref(p), cams, 1, 1000, big, *([None] * 11), C.byref(n), None)
    assert s == L.FSS_ERR_UNSUPPORTED and "FSS_STATIC_SCRATCH_BYTES" in L.last_error()


def test_kernel_event_hook_arguments(lib):
    assert lib.fss_set_kernel_events(None, 0) == L.FSS_OK
    assert lib.fss_set_kernel_events(None, 2) == L.FSS_ERR_INVALID_ARG
    arr = (C.c_void_p * 2)(None, None)
    assert lib.fss_set_kernel_events(arr, 2) == L.FSS_ERR_INVALID_ARG
    assert lib.fss_set_kernel_events(arr, -1) == L.FSS_ERR_INVALID_ARG


def test_query_label_arguments_are_checked_on_the_host(lib):
    z = C.c_void_p(16)  # never dereferenced: every call below is rejected first
    assert lib.fss_query_labels(10, 24, 32, z, z, z, z, z, z, L.FSS_F32, z, None) == L.FSS_ERR_UNSUPPORTED
    assert lib.fss_query_labels(10, 32, 40, z, z, z, z, z, z, L.FSS_F32, z, None) == L.FSS_ERR_UNSUPPORTED
    assert lib.fss_query_labels(10, 512, 32, z, z, z, z, z, z, L.FSS_F32, z, None) == L.FSS_ERR_UNSUPPORTED
    assert lib.fss_query_labels(-1, 32, 32, z, z, z, z, z, z, L.FSS_F32, z, None) == L.FSS_ERR_UNSUPPORTED
    assert lib.fss_query_labels(10, 32, 32, z, z, z, z, z, z, 7, z, None) == L.FSS_ERR_INVALID_ARG
    assert lib.fss_query_labels(10, 32, 32, None, z, z, z, z, z, L.FSS_F32, z, None) == L.FSS_ERR_INVALID_ARG
    assert lib.fss_query_labels(10, 32, 32, z, z, z, z, z, z, L.FSS_F32, None, None) == L.FSS_ERR_INVALID_ARG
    assert lib.fss_query_labels(10, 32, 32, C.c_void_p(24), z, z, z, z, z, L.FSS_F32, z, None) == L.FSS_ERR_INVALID_ARG
    assert "aligned" in L.last_error()


def test_colour_mode_arguments(lib):
    out = C.c_size_t()
    p = L.fss_default_params()
    assert (p.color_mode, p.sh_degree) == (L.FSS_COLOR_RGB, 0)
    p.color_mode = 2
    assert lib.fss_workspace_size(C.byref(p), _cam(), 1, 10, 10, C.byref(out)) == L.FSS_ERR_INVALID_ARG
    p.color_mode, p.sh_degree = L.FSS_COLOR_SH, 4
    assert lib.fss_workspace_size(C.byref(p), _cam(), 1, 10, 10, C.byref(out)) == L.FSS_ERR_UNSUPPORTED
    p.sh_degree = 3
    assert lib.fss_workspace_size(C.byref(p), _cam(), 1, 1000, 10, C.byref(out)) == L.FSS_OK
    ws_sh = out.value
    p.color_mode = L.FSS_COLOR_RGB
    lib.fss_workspace_size(C.byref(p), _cam(), 1, 1000, 10, C.byref(out))
    # the colour mode adds a direction (16 B) and a colour (12 B) per item
    assert ws_sh - out.value >= 1000 * 28


def test_status_values_match_the_header():
    text = open(HEADER).read()
    for name in ("FSS_ERR_INVALID_ARG", "FSS_ERR_UNSUPPORTED", "FSS_ERR_CAPACITY", "FSS_ERR_CUDA", "FSS_ERR_TIMEOUT",
                 "FSS_ERR_BOUNDS"):
        m = re.search(rf"{name} = (\d+)", text)
        assert m and int(m.group(1)) == getattr(L, name), name
        assert L.STATUS_NAMES[getattr(L, name)] == name


def test_check_build_exports_the_abi_with_a_canary_after_every_region(lib):
    """The check build (FSS_CHECK_BOUNDS=1) is the same ABI; its workspace
    adds one 256-byte canary after each region, and its regions keep the
    release sizes."""
    from paper_2604_10951_gb300.build import LIB_CHECK
    chk = C.CDLL(LIB_CHECK)
    for name in _declared():
        assert hasattr(chk, name), name
    pp, pc = C.POINTER(L.fss_params), C.POINTER(L.fss_camera)
    chk.fss_workspace_size.argtypes = [pp, pc, C.c_int32, C.c_int64, C.c_int64, C.POINTER(C.c_size_t)]
    chk.fss_workspace_region.argtypes = [pp, pc, C.c_int32, C.c_int64, C.c_int64, C.c_int32,
                                         C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    p = L.fss_default_params()
    cams = _cam()
    out = C.c_size_t()
    assert chk.fss_workspace_size(C.byref(p), cams, 1, 1000, 5000, C.byref(out)) == L.FSS_OK
    assert out.value == L.fss_workspace_size(p, cams, 1, 1000, 5000) + 256 * L.N_REGIONS
    off, size = C.c_size_t(), C.c_size_t()
    prev_end = 0
    for r in range(L.N_REGIONS):
        assert chk.fss_workspace_region(C.byref(p), cams, 1, 1000, 5000, r, C.byref(off), C.byref(size)) == L.FSS_OK
        assert size.value == L.fss_workspace_region(p, cams, 1, 1000, 5000, r)[1]
        if r != L.REG_COUNTERS:
            assert off.value >= prev_end  # the previous region's canary lies between
            prev_end = off.value + (size.value + 255) // 256 * 256 + 256
    assert prev_end <= out.value


def test_forward_loss_arguments_are_checked_on_the_host(lib):
    """fss_render_forward_loss (and with the sort, fss_sort_render_forward_loss)
    needs out_feat, out_rgb and every loss buffer,
    16-byte aligned feature buffers and valid parameters; each is rejected
    before any launch."""
    p = L.fss_default_params()
    z = C.c_void_p(256)  # never dereferenced: every call below is rejected first
    ws = C.c_void_p(4096)

    for fn in (lib.fss_render_forward_loss, lib.fss_sort_render_forward_loss):
        def call(params=p, out_feat=z, feat_target=z, d_feat=z, loss=z):
            return fn(C.byref(params), _cam(), 1, 10, ws, 100, z, z, out_feat, z, z, z, z, feat_target, z, 1.0, 1.0,
                      d_feat, z, loss, None)

        assert call(out_feat=None) == L.FSS_ERR_INVALID_ARG
        assert call(loss=None) == L.FSS_ERR_INVALID_ARG and "loss" in L.last_error()
        assert call(feat_target=C.c_void_p(264)) == L.FSS_ERR_INVALID_ARG and "aligned" in L.last_error()
        assert call(d_feat=C.c_void_p(72)) == L.FSS_ERR_INVALID_ARG
        bad = L.fss_default_params()
        bad.K = 33
        assert call(params=bad) == L.FSS_ERR_UNSUPPORTED

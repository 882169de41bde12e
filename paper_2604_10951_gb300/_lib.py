"""ctypes binding of ``libfss.so`` (the C ABI in ``include/fss.h``).

Functions keep the C names and take plain integers / pointers; this module
only marshals arguments.  Importing it never compiles anything: the library
must have been built (``paper_2604_10951_gb300.build.build()``), else
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from .build import LIB, LIB_CHECK

FSS_OK, FSS_ERR_INVALID_ARG, FSS_ERR_UNSUPPORTED, FSS_ERR_CAPACITY, FSS_ERR_CUDA, FSS_ERR_TIMEOUT, FSS_ERR_BOUNDS = range(7)
FSS_BIN_AABB, FSS_BIN_SNUG, FSS_BIN_ACCU = 0, 1, 2
FSS_STOP_TMIN, FSS_STOP_EXACT_TOPK = 0, 1
FSS_F32, FSS_BF16 = 0, 1
FSS_SCHED_GRID, FSS_SCHED_PERSISTENT = 0, 1
FSS_COLOR_RGB, FSS_COLOR_SH = 0, 1
FSS_SELECT_TOPW, FSS_SELECT_FRONT = 0, 1
FSS_MAX_CAMS = 64
FSS_MAX_K = 32
STATUS_NAMES = {0: "FSS_OK", 1: "FSS_ERR_INVALID_ARG", 2: "FSS_ERR_UNSUPPORTED", 3: "FSS_ERR_CAPACITY",
                4: "FSS_ERR_CUDA", 5: "FSS_ERR_TIMEOUT", 6: "FSS_ERR_BOUNDS"}

# workspace regions (fss_workspace_region)
REG_STATUS, REG_REC, REG_BINREC, REG_COUNT, REG_RANGES, REG_LIST, REG_COUNTERS, REG_TILECNT = range(8)
REG_SORTTMP, REG_GRAD_ITEM, REG_FEAT_ACC, REG_DOTS, REG_VIS, REG_UNB, REG_SLOT, REG_WIDE = range(8, 16)
REG_MASK = 16
REG_SLOT_SURF = 17
REG_DIR = 18
REG_COLOR = 19
REG_ORDER = 20
N_REGIONS = 21

EXPORTS = ["fss_default_params", "fss_workspace_size", "fss_saved_size", "fss_project_bin", "fss_sort",
           "fss_render_forward", "fss_render_backward", "fss_read_status", "fss_last_error",
           "fss_workspace_region", "fss_loss_l2_l1", "fss_forward_static", "fss_set_kernel_events",
           "fss_render_forward_aux", "fss_query_labels", "fss_test_hold_scan", "fss_render_forward_loss",
           "fss_sort_render_forward_loss"]
FSS_STATIC_SCRATCH_BYTES = 64 << 20


class fss_camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("viewmat", C.c_float * 12),
                ("near_plane", C.c_float)]


class fss_params(C.Structure):
    _fields_ = [("tile_size", C.c_int32), ("K", C.c_int32), ("bin_mode", C.c_int32), ("stop_rule", C.c_int32),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("T_min", C.c_float),
                ("feat_dtype", C.c_int32), ("out_dtype", C.c_int32), ("C", C.c_int32),
                ("bg_rgb", C.c_float * 3), ("schedule", C.c_int32), ("select", C.c_int32),
                ("renorm", C.c_int32), ("color_mode", C.c_int32), ("sh_degree", C.c_int32),
                ("lowpass", C.c_int32)]


class fss_aux_outputs(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("depth_median", C.c_void_p), ("normal", C.c_void_p), ("label", C.c_void_p)]


class FssError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def check_build() -> bool:
    """True when the environment asks for the check build (FSS_CHECK_BOUNDS=1)."""
    return os.environ.get("FSS_CHECK_BOUNDS", "0") == "1"


def lib():
    """The loaded library (the check build when FSS_CHECK_BOUNDS=1); raises
    if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = LIB_CHECK if check_build() else LIB
            if not os.path.exists(path):
                raise ImportError(f"{os.path.basename(path)} not built ({path}); "
                                  "run paper_2604_10951_gb300.build.build()")
            L = C.CDLL(path)
            P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            pp, pc = C.POINTER(fss_params), C.POINTER(fss_camera)
            sig = {
                "fss_default_params": [pp],
                "fss_workspace_size": [pp, pc, i32, i64, i64, C.POINTER(C.c_size_t)],
                "fss_saved_size": [pp, pc, i32, C.POINTER(C.c_size_t)],
                "fss_project_bin": [pp, pc, i32, i64, P, P, P, P, P, i64, P],
                "fss_sort": [pp, pc, i32, i64, P, i64, P],
                "fss_render_forward": [pp, pc, i32, i64, P, i64, P, P, P, P, P, P, P, P],
                "fss_render_backward": [pp, pc, i32, i64, P, i64, P, P, P, P, P, P, P, P, P, P, P,
                                        P, P, P, P, P, P, P],
                "fss_read_status": [pp, pc, i32, i64, P, i64, C.POINTER(C.c_int64), P],
                "fss_workspace_region": [pp, pc, i32, i64, i64, i32, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)],
                "fss_loss_l2_l1": [pp, i64, P, P, P, P, C.c_float, C.c_float, P, P, P, P],
                "fss_forward_static": [pp, pc, i32, i64, i64, P, P, P, P, P, P, P, P, P, P, P,
                                       C.POINTER(C.c_int64), P],
                "fss_set_kernel_events": [C.POINTER(C.c_void_p), i32],
                "fss_test_hold_scan": [i32],
                "fss_render_forward_aux": [pp, pc, i32, i64, P, i64, P, P, P, P, P, P, P,
                                           C.POINTER(fss_aux_outputs), P],
                "fss_query_labels": [i64, i32, i32, P, P, P, P, P, P, i32, P, P],
                "fss_render_forward_loss": [pp, pc, i32, i64, P, i64, P, P, P, P, P, P, P, P, P,
                                            C.c_float, C.c_float, P, P, P, P],
                "fss_sort_render_forward_loss": [pp, pc, i32, i64, P, i64, P, P, P, P, P, P, P, P, P,
                                                 C.c_float, C.c_float, P, P, P, P],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.fss_last_error.argtypes = []
            L.fss_last_error.restype = C.c_char_p
            _lib = L
    return _lib


def last_error() -> str:
    return lib().fss_last_error().decode()


def check(status: int) -> int:
    if status != FSS_OK:
        raise FssError(status, last_error())
    return status


# -- same-name wrappers (marshalling only) ----------------------------------

def fss_default_params() -> fss_params:
    p = fss_params()
    check(lib().fss_default_params(C.byref(p)))
    return p


def fss_workspace_size(params, cams, n_cams, N, pair_capacity) -> int:
    out = C.c_size_t()
    check(lib().fss_workspace_size(C.byref(params), cams, n_cams, N, pair_capacity, C.byref(out)))
    return out.value


def fss_saved_size(params, cams, n_cams) -> int:
    out = C.c_size_t()
    check(lib().fss_saved_size(C.byref(params), cams, n_cams, C.byref(out)))
    return out.value


def fss_workspace_region(params, cams, n_cams, N, pair_capacity, which):
    off, size = C.c_size_t(), C.c_size_t()
    check(lib().fss_workspace_region(C.byref(params), cams, n_cams, N, pair_capacity, which,
                                     C.byref(off), C.byref(size)))
    return off.value, size.value


def fss_project_bin(params, cams, n_cams, N, means, scales, quats, opac, workspace, pair_capacity, stream):
    return check(lib().fss_project_bin(C.byref(params), cams, n_cams, N, means, scales, quats, opac,
                                       workspace, pair_capacity, stream))


def fss_sort(params, cams, n_cams, N, workspace, pair_capacity, stream):
    return check(lib().fss_sort(C.byref(params), cams, n_cams, N, workspace, pair_capacity, stream))


def fss_render_forward(params, cams, n_cams, N, workspace, pair_capacity, rgb, feats, out_feat, out_rgb, out_T,
                       out_topk_id, saved, stream):
    return check(lib().fss_render_forward(C.byref(params), cams, n_cams, N, workspace, pair_capacity, rgb, feats,
                                          out_feat, out_rgb, out_T, out_topk_id, saved, stream))


def fss_render_backward(params, cams, n_cams, N, workspace, pair_capacity, means, scales, quats, opac, rgb, feats,
                        saved, out_T, d_feat, d_rgb, d_T, g_means, g_scales, g_quats, g_opac, g_rgb, g_feat, stream):
    return check(lib().fss_render_backward(C.byref(params), cams, n_cams, N, workspace, pair_capacity, means, scales,
                                           quats, opac, rgb, feats, saved, out_T, d_feat, d_rgb, d_T, g_means,
                                           g_scales, g_quats, g_opac, g_rgb, g_feat, stream))


def fss_loss_l2_l1(params, n_pix, feat, rgb, feat_target, rgb_target, w_feat, w_rgb, d_feat, d_rgb, loss, stream):
    return check(lib().fss_loss_l2_l1(C.byref(params), n_pix, feat, rgb, feat_target, rgb_target, float(w_feat),
                                      float(w_rgb), d_feat, d_rgb, loss, stream))


def fss_render_forward_loss(params, cams, n_cams, N, workspace, pair_capacity, rgb, feats, out_feat, out_rgb, out_T,
                            out_topk_id, saved, feat_target, rgb_target, w_feat, w_rgb, d_feat, d_rgb, loss, stream):
    return check(lib().fss_render_forward_loss(C.byref(params), cams, n_cams, N, workspace, pair_capacity, rgb, feats,
                                               out_feat, out_rgb, out_T, out_topk_id, saved, feat_target, rgb_target,
                                               float(w_feat), float(w_rgb), d_feat, d_rgb, loss, stream))


def fss_sort_render_forward_loss(params, cams, n_cams, N, workspace, pair_capacity, rgb, feats, out_feat, out_rgb,
                                 out_T, out_topk_id, saved, feat_target, rgb_target, w_feat, w_rgb, d_feat, d_rgb,
                                 loss, stream):
    return check(lib().fss_sort_render_forward_loss(C.byref(params), cams, n_cams, N, workspace, pair_capacity, rgb,
                                                    feats, out_feat, out_rgb, out_T, out_topk_id, saved, feat_target,
                                                    rgb_target, float(w_feat), float(w_rgb), d_feat, d_rgb, loss,
                                                    stream))


def fss_query_labels(N, n_queries, dim, f_ins, means, f_q, p_q, prec_q, labels, out_dtype, err, stream):
    return check(lib().fss_query_labels(N, n_queries, dim, f_ins, means, f_q, p_q, prec_q, labels, out_dtype, err,
                                        stream))


def fss_read_status(params, cams, n_cams, N, workspace, pair_capacity, stream):
    """Returns (status, num_pairs) without raising on device-side errors."""
    n = C.c_int64()
    s = lib().fss_read_status(C.byref(params), cams, n_cams, N, workspace, pair_capacity, C.byref(n), stream)
    return s, n.value


def fss_forward_static(params, cams, n_cams, N, pair_capacity, means, scales, quats, opac, rgb, feats, out_feat,
                       out_rgb, out_T, out_topk_id, saved, stream):
    """Returns (status, num_pairs); raises only on argument or CUDA errors."""
    n = C.c_int64()
    s = lib().fss_forward_static(C.byref(params), cams, n_cams, N, pair_capacity, means, scales, quats, opac, rgb,
                                 feats, out_feat, out_rgb, out_T, out_topk_id, saved, C.byref(n), stream)
    if s not in (FSS_OK, FSS_ERR_CAPACITY):
        check(s)
    return s, n.value


_events_keepalive = None


def fss_test_hold_scan(hold: bool):
    """Failure-detection test hook: the binning's tile scan withholds its result (see include/fss.h)."""
    check(lib().fss_test_hold_scan(1 if hold else 0))


def fss_set_kernel_events(events):
    """events: sequence of torch.cuda.Event (timing enabled) or raw handles; [] switches the hook off.
    torch creates an event's CUDA handle at its first record, so record each one once beforehand."""
    global _events_keepalive
    handles = [e.cuda_event if hasattr(e, "cuda_event") else int(e) for e in events]
    arr = (C.c_void_p * max(1, len(handles)))(*handles)
    check(lib().fss_set_kernel_events(arr, len(handles)))
    _events_keepalive = arr if handles else None


def fss_render_forward_aux(params, cams, n_cams, N, workspace, pair_capacity, rgb, feats, out_feat, out_rgb, out_T,
                           out_topk_id, saved, depth, depth_median, normal, stream, label=None):
    aux = fss_aux_outputs(depth, depth_median, normal, label)
    return check(lib().fss_render_forward_aux(C.byref(params), cams, n_cams, N, workspace, pair_capacity, rgb, feats,
                                              out_feat, out_rgb, out_T, out_topk_id, saved, C.byref(aux), stream))

"""FP64 CPU oracle for the 2DGS Top-K feature rasterizer (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; it
shares no code with the C source here (``fss_oracle.c``), which is compiled
with gcc into ``oracle/_build/liborc.so`` by :func:`build`.

Every function takes plain numpy arrays (float32 inputs exactly as the CUDA
library receives them) and returns numpy arrays.  Definitions and paper
citations are in ``fss_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fss_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liborc.so")
_lib = None
_lock = threading.Lock()

AABB, SNUG, ACCU = 0, 1, 2
TMIN, EXACT_TOPK = 0, 1
FLAG_ALPHA, FLAG_TMIN, FLAG_TIE, FLAG_EXACT, FLAG_NEAR, FLAG_CLAMP, FLAG_GRAZE = 1, 2, 4, 8, 16, 32, 64
FLAG_MEDIAN = 128
FLAG_LOWPASS = 256
# flags of the borderline decisions that a per-pixel flip mask can take the other way
FLAGS_BORDER = FLAG_ALPHA | FLAG_TMIN | FLAG_TIE | FLAG_EXACT | FLAG_NEAR
# flip-mask bit of the median-depth switch (bits 0..30: the other borderline decisions in order)
FLIP_MEDIAN = 1 << 31


class OrcCam(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("viewmat", C.c_float * 12),
                ("near_plane", C.c_float)]


class OrcParams(C.Structure):
    _fields_ = [("tile_size", C.c_int32), ("K", C.c_int32), ("bin_mode", C.c_int32),
                ("stop_rule", C.c_int32), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("T_min", C.c_float), ("bg", C.c_float * 3), ("C", C.c_int32), ("select", C.c_int32),
                ("renorm", C.c_int32), ("lowpass", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary32 ops unfused: -ffp-contract=off)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fexcess-precision=standard", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            i64 = C.c_int64
            lib.orc_mirror_project.argtypes = [i64, P, P, P, P, C.POINTER(OrcCam), C.POINTER(OrcParams), C.c_int, P, P, P]
            lib.orc_mirror_project.restype = None
            lib.orc_bin.argtypes = [i64, P, P, P, P, C.POINTER(OrcCam), C.POINTER(OrcParams), C.c_int, i64, P, P]
            lib.orc_bin.restype = i64
            lib.orc_sort_pairs.argtypes = [i64, P, P, P, P, P]
            lib.orc_sort_pairs.restype = None
            lib.orc_ranges.argtypes = [i64, P, C.c_int32, P]
            lib.orc_ranges.restype = None
            lib.orc_render.argtypes = [i64, P, P, P, P, P, P, C.POINTER(OrcCam), C.POINTER(OrcParams), P, P, P, P,
                                       P, P, P, P, P, P, P, P, P, P, C.c_int, P, P, P, P, P, P]
            lib.orc_render.restype = None
            lib.orc_render_backward.argtypes = [i64, P, P, P, P, P, P, C.POINTER(OrcCam), C.POINTER(OrcParams),
                                                P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_render_backward.restype = None
            lib.orc_geometry.argtypes = [i64, P, P, P, P, C.POINTER(OrcCam), C.POINTER(OrcParams), P, P, P, P]
            lib.orc_geometry.restype = None
            lib.orc_ray_splat.argtypes = [P, i64, P, C.c_double, P, P]
            lib.orc_ray_splat.restype = None
            lib.orc_check_conservative.argtypes = [i64, P, P, P, P, C.POINTER(OrcCam), C.POINTER(OrcParams), C.c_int, P]
            lib.orc_check_conservative.restype = i64
            lib.orc_query_labels.argtypes = [i64, C.c_int32, C.c_int32, P, P, P, P, P, P]
            lib.orc_query_labels.restype = None
            lib.orc_sh_basis.argtypes = [C.c_int, P, P, P]
            lib.orc_sh_basis.restype = None
            lib.orc_sh_colors.argtypes = [i64, C.c_int, P, P, C.POINTER(OrcCam), P]
            lib.orc_sh_colors.restype = None
            lib.orc_sh_backward.argtypes = [i64, C.c_int, P, P, C.POINTER(OrcCam), P, P, P, P]
            lib.orc_sh_backward.restype = None
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def make_cam(cam) -> OrcCam:
    """From any object with fx, fy, cx, cy, width, height, viewmat (3x4), near."""
    c = OrcCam()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    vm = np.asarray(cam.viewmat, dtype=np.float32).reshape(12)
    for k in range(12):
        c.viewmat[k] = float(vm[k])
    c.near_plane = float(getattr(cam, "near", 0.2))
    return c


def make_params(tile_size=16, K=0, bin_mode=ACCU, stop_rule=TMIN, alpha_min=1.0 / 255.0,
                alpha_max=0.99, T_min=1e-4, bg=(0.0, 0.0, 0.0), C=0, select=0, renorm=0, lowpass=0) -> OrcParams:
    p = OrcParams()
    p.tile_size, p.K, p.bin_mode, p.stop_rule = int(tile_size), int(K), int(bin_mode), int(stop_rule)
    p.alpha_min, p.alpha_max, p.T_min = float(np.float32(alpha_min)), float(alpha_max), float(T_min)
    for k in range(3):
        p.bg[k] = float(bg[k])
    p.C, p.select, p.renorm, p.lowpass = int(C), int(select), int(renorm), int(lowpass)
    return p


def _scene_arrays(scene):
    """binary32 parameters for the binning mirror"""
    return (_f32(scene.means), _f32(scene.scales), _f32(scene.quats), _f32(scene.opacities))


def _scene_arrays64(scene):
    """FP64 parameters for the renderer (binary32 scenes convert exactly;
    finite differences pass float64 arrays)"""
    return (_f64(scene.means), _f64(scene.scales), _f64(scene.quats), _f64(scene.opacities))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def geometry(scene, cam, params):
    """FP64 homography rows T [N,3,3], centre depth z, cos(normal, ray), cull flag."""
    lib = _load()
    m, s, q, o = _scene_arrays64(scene)
    N = m.shape[0]
    T = np.zeros((N, 3, 3)); z = np.zeros(N); ca = np.zeros(N); ok = np.zeros(N, np.int32)
    lib.orc_geometry(N, _ptr(m), _ptr(s), _ptr(q), _ptr(o), C.byref(make_cam(cam)), C.byref(params),
                     _ptr(T), _ptr(z), _ptr(ca), _ptr(ok))
    return T, z, ca, ok


def ray_splat(T, xy, near=-np.inf):
    """(u, v, z_hit) and validity for pixel points xy [M,2] under one T [3,3]."""
    lib = _load()
    T = _f64(T).reshape(9)
    xy = _f64(xy).reshape(-1, 2)
    uvz = np.zeros((xy.shape[0], 3)); valid = np.zeros(xy.shape[0], np.int32)
    lib.orc_ray_splat(_ptr(T), xy.shape[0], _ptr(xy), float(near), _ptr(uvz), _ptr(valid))
    return uvz, valid


def mirror_project(scene, cam, params, mode=None):
    """binary32 binning mirror: (recf [N,26], reci [N,11], count [N])."""
    lib = _load()
    mode = params.bin_mode if mode is None else mode
    m, s, q, o = _scene_arrays(scene)
    N = m.shape[0]
    recf = np.zeros((N, 26), np.float32); reci = np.zeros((N, 11), np.int32); cnt = np.zeros(N, np.int32)
    lib.orc_mirror_project(N, _ptr(m), _ptr(s), _ptr(q), _ptr(o), C.byref(make_cam(cam)), C.byref(params),
                           int(mode), _ptr(recf), _ptr(reci), _ptr(cnt))
    return recf, reci, cnt


REC_FIELDS = ["z", "k2", "xc", "yc", "det"] + [f"m{i}" for i in range(9)] + \
             ["A", "B", "C", "D", "E", "F", "X0", "Y0", "hx", "hy", "pad0", "pad1"]
RECI_FIELDS = ["visible", "culled_by_rule", "unbounded", "px0", "px1", "py0", "py1", "tx0", "tx1", "ty0", "ty1"]


def bin_pairs(scene, cam, params, mode=None):
    """Unsorted (tile, surfel) pairs in surfel order from the binning mirror."""
    lib = _load()
    mode = params.bin_mode if mode is None else mode
    m, s, q, o = _scene_arrays(scene)
    N = m.shape[0]
    cam_c = make_cam(cam)
    P = lib.orc_bin(N, _ptr(m), _ptr(s), _ptr(q), _ptr(o), C.byref(cam_c), C.byref(params), int(mode), 0, None, None)
    tiles = np.zeros(max(P, 1), np.int32); ids = np.zeros(max(P, 1), np.int32)
    lib.orc_bin(N, _ptr(m), _ptr(s), _ptr(q), _ptr(o), C.byref(cam_c), C.byref(params), int(mode), P,
                _ptr(tiles), _ptr(ids))
    return tiles[:P], ids[:P]


def n_tiles(cam, tile_size):
    return ((cam.width + tile_size - 1) // tile_size) * ((cam.height + tile_size - 1) // tile_size)


def sort_and_ranges(tiles, ids, z, ntiles):
    """Pairs ordered by (tile, depth bits, index) and per-tile [start, end)."""
    lib = _load()
    tiles, ids, z = _i32(tiles), _i32(ids), _f32(z)
    P = tiles.shape[0]
    st = np.zeros(max(P, 1), np.int32); si = np.zeros(max(P, 1), np.int32)
    lib.orc_sort_pairs(P, _ptr(tiles), _ptr(ids), _ptr(z), _ptr(st), _ptr(si))
    rng = np.zeros((ntiles, 2), np.int32)
    lib.orc_ranges(P, _ptr(st), int(ntiles), _ptr(rng))
    return st[:P], si[:P], rng


def binning(scene, cam, params, mode=None):
    """Full mirror binning: dict with recf, reci, count, sorted tiles/ids, ranges."""
    recf, reci, cnt = mirror_project(scene, cam, params, mode)
    tiles, ids = bin_pairs(scene, cam, params, mode)
    st, si, rng = sort_and_ranges(tiles, ids, recf[:, 0], n_tiles(cam, params.tile_size))
    return dict(recf=recf, reci=reci, count=cnt, tiles=st, ids=si, ranges=rng, P=int(st.shape[0]))


def _u32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint32)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


def render(scene, cam, params, feats=None, binned=None, brute=False, visible=None, zkey=None, threads=0, sh=None,
           flip=None, only=None):
    """FP64 render.  Tiled over ``binned`` lists (computed if None) unless
    ``brute``; returns a dict of per-pixel outputs.  ``sh`` [N, B, 3]:
    view-dependent colours from spherical-harmonic coefficients instead of
    ``scene.rgb``.  ``flip`` [H, W] (uint32): per-pixel masks that take the
    pixel's borderline decisions the other way (bit b: the b-th one met;
    FLIP_MEDIAN: the median-depth switch); ``only`` [H, W] (bool): render
    just those pixels (the others' outputs stay zero).  "nborder" counts the
    borderline decisions each pixel met."""
    lib = _load()
    m, s, q, o = _scene_arrays64(scene)
    rgb = _f64(scene.rgb) if sh is None else sh_colors(sh, scene.means, cam)
    feats = _f64(scene.feats if feats is None else feats)
    N, Cc = m.shape[0], feats.shape[1]
    params.C = Cc
    H, W, K = cam.height, cam.width, params.K
    if not brute and binned is None:
        binned = binning(scene, cam, params)
    out = dict(F=np.zeros((H, W, Cc)), rgb=np.zeros((H, W, 3)), T=np.zeros((H, W)),
               nstop=np.zeros((H, W), np.int32), ncontrib=np.zeros((H, W), np.int32),
               flags=np.zeros((H, W), np.int32), counters=np.zeros(2, np.int64),
               depth=np.zeros((H, W)), depth_med=np.zeros((H, W)), normal=np.zeros((H, W, 3)),
               nborder=np.zeros((H, W), np.int32))
    flip = _u32(flip)
    only = _u8(only)
    assert flip is None or flip.size == H * W
    assert only is None or only.size == H * W
    Kc = max(K, 1)
    out.update(ids=np.full((H, W, Kc), -1, np.int32), w=np.zeros((H, W, Kc)), pos=np.full((H, W, Kc), -1, np.int32))
    rng = None if brute else _i32(binned["ranges"])
    sid = None if brute else _i32(binned["ids"])
    vis = None if visible is None else _i32(visible)
    zk = None if zkey is None else _f32(zkey)
    lib.orc_render(N, _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(rgb), _ptr(feats), C.byref(make_cam(cam)),
                   C.byref(params), _ptr(rng), _ptr(sid), _ptr(vis), _ptr(zk),
                   _ptr(out["F"]), _ptr(out["rgb"]), _ptr(out["T"]),
                   _ptr(out["ids"]) if K else None, _ptr(out["w"]) if K else None, _ptr(out["pos"]) if K else None,
                   _ptr(out["nstop"]), _ptr(out["ncontrib"]), _ptr(out["flags"]), _ptr(out["counters"]), int(threads),
                   _ptr(out["depth"]), _ptr(out["depth_med"]), _ptr(out["normal"]),
                   _ptr(flip), _ptr(only), _ptr(out["nborder"]))
    if not K:
        for k in ("ids", "w", "pos"):
            out.pop(k)
    out["binned"] = binned
    return out


def render_backward(scene, cam, params, gF, grgb, gT=None, feats=None, binned=None, brute=False,
                    visible=None, zkey=None, sh=None, flip=None):
    """Analytic FP64 gradients of sum(gF*F) + sum(grgb*rgb) + sum(gT*T), and
    under "abs" [N, 10] the same chain over magnitudes (means, scales, quats,
    opacity): a bound on the sum of |terms| that each geometric gradient
    entry adds up.  With ``sh`` [N, B, 3] the colours are view dependent: "sh"
    holds dL/dcoefficients, "rgb" the gradient of this view's colours, and
    the direction term joins "means" (and its magnitude "abs").  ``flip``
    [H, W]: the per-pixel borderline outcomes, as in :func:`render`."""
    lib = _load()
    m, s, q, o = _scene_arrays64(scene)
    rgb = _f64(scene.rgb) if sh is None else sh_colors(sh, scene.means, cam)
    feats = _f64(scene.feats if feats is None else feats)
    N, Cc = m.shape[0], feats.shape[1]
    params.C = Cc
    if not brute and binned is None:
        binned = binning(scene, cam, params)
    g = dict(means=np.zeros((N, 3)), scales=np.zeros((N, 2)), quats=np.zeros((N, 4)), opac=np.zeros(N),
             rgb=np.zeros((N, 3)), feat=np.zeros((N, Cc)), Tmat=np.zeros((N, 9)), abs=np.zeros((N, 10)))
    rng = None if brute else _i32(binned["ranges"])
    sid = None if brute else _i32(binned["ids"])
    vis = None if visible is None else _i32(visible)
    zk = None if zkey is None else _f32(zkey)
    gF = None if gF is None else _f64(gF)
    grgb = _f64(grgb)
    gT = None if gT is None else _f64(gT)
    lib.orc_render_backward(N, _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(rgb), _ptr(feats), C.byref(make_cam(cam)),
                            C.byref(params), _ptr(rng), _ptr(sid), _ptr(vis), _ptr(zk),
                            _ptr(gF), _ptr(grgb), _ptr(gT),
                            _ptr(g["means"]), _ptr(g["scales"]), _ptr(g["quats"]), _ptr(g["opac"]),
                            _ptr(g["rgb"]), _ptr(g["feat"]), _ptr(g["Tmat"]), _ptr(g["abs"]),
                            _ptr(_u32(flip)))
    if sh is not None:
        shc = _f64(sh)
        g["sh"] = np.zeros_like(shc)
        lib.orc_sh_backward(N, _sh_degree(shc), _ptr(shc), _ptr(m), C.byref(make_cam(cam)), _ptr(g["rgb"]),
                            _ptr(g["sh"]), _ptr(g["means"]), _ptr(g["abs"]))
    return g


def _sh_degree(sh):
    nb = sh.shape[1]
    deg = int(round(nb ** 0.5)) - 1
    assert (deg + 1) ** 2 == nb and 0 <= deg <= 3 and sh.shape[2] == 3, sh.shape
    return deg


def sh_basis(deg, dirs):
    """Real spherical harmonics of degree <= deg at unit directions [M, 3]:
    (Y [M, B], dY/d(x, y, z) [M, B, 3]) of the Cartesian polynomials."""
    lib = _load()
    dirs = _f64(dirs).reshape(-1, 3)
    nb = (deg + 1) ** 2
    Y, G = np.zeros((len(dirs), 16)), np.zeros((len(dirs), 16, 3))
    for i, d in enumerate(dirs):
        lib.orc_sh_basis(deg, _ptr(np.ascontiguousarray(d)), _ptr(Y[i]), _ptr(G[i]))
    return Y[:, :nb], G[:, :nb]


def sh_colors(sh, means, cam):
    """Per-surfel colours [N, 3] seen from ``cam``: max(0, sum_b sh[:, b] Y_b(d) + 1/2)."""
    lib = _load()
    shc, m = _f64(sh), _f64(means)
    out = np.zeros((m.shape[0], 3))
    lib.orc_sh_colors(m.shape[0], _sh_degree(shc), _ptr(shc), _ptr(m), C.byref(make_cam(cam)), _ptr(out))
    return out


def query_labels(f_ins, means, f_q, p_q, prec):
    """Instance label distributions l_ins [N, nq] of Sec. 3.3 in FP64:
    softmax over queries of sigmoid(f_q . f_ins) exp(-1/2 d^T prec d),
    d = p_g - p_q, prec [nq, 6] = (xx, yy, zz, xy, xz, yz) of Sigma_q^-1."""
    lib = _load()
    f_ins, means, f_q, p_q, prec = (_f64(a) for a in (f_ins, means, f_q, p_q, prec))
    N, dim = f_ins.shape
    nq = f_q.shape[0]
    assert f_q.shape[1] == dim and means.shape == (N, 3) and p_q.shape == (nq, 3) and prec.shape == (nq, 6)
    out = np.zeros((N, nq))
    lib.orc_query_labels(N, nq, dim, _ptr(f_ins), _ptr(means), _ptr(f_q), _ptr(p_q), _ptr(prec), _ptr(out))
    return out


def check_conservative(scene, cam, params, mode=None):
    """(violations, checked) of the mirror binning against FP64 brute force."""
    lib = _load()
    mode = params.bin_mode if mode is None else mode
    m, s, q, o = _scene_arrays(scene)
    checked = np.zeros(1, np.int64)
    bad = lib.orc_check_conservative(m.shape[0], _ptr(m), _ptr(s), _ptr(q), _ptr(o), C.byref(make_cam(cam)),
                                     C.byref(params), int(mode), _ptr(checked))
    return int(bad), int(checked[0])

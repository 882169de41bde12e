"""GPU parity of projection, Precise Tile Intersection and the depth sort.

Every integer result (culling, pixel and tile ranges, per-surfel tile
counts, the tile lists and their order) is bit-exact against the oracle's
binary32 binning mirror, and so are the binary32 values the decisions are
taken from (adjugate rows, centre, conic, ellipse extents, depth, cutoff).
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene

pytestmark = pytest.mark.gpu

MODES = {"aabb": O.AABB, "snug": O.SNUG, "accu": O.ACCU}


def _check_view(run, scene, cam, ts, mode, view=0, lowpass=0):
    p = O.make_params(tile_size=ts, K=run.params.K, lowpass=lowpass)
    recf, reci, cnt = O.mirror_project(scene, cam, p, MODES[mode])
    N = scene.n
    sl = slice(view * N, (view + 1) * N)
    rec = run.rec()[sl]            # r0=(m0,xc) r1=(m1,yc) r2=(m2,det) r3=(o,z,k2,s)
    bf, bi, flags = run.binrec()
    bf, bi, flags = bf[sl], bi[sl], flags[sl]
    vis = reci[:, 0] == 1
    np.testing.assert_array_equal((flags & 1) == 1, vis)
    m = vis
    # binary32 values behind every decision, bit for bit
    np.testing.assert_array_equal(rec[m, 13], recf[m, 0])   # centre depth z
    np.testing.assert_array_equal(rec[m, 14], recf[m, 1])   # cutoff k^2
    np.testing.assert_array_equal(rec[m, 3], recf[m, 2])    # xc
    np.testing.assert_array_equal(rec[m, 7], recf[m, 3])    # yc
    np.testing.assert_array_equal(rec[m, 12], scene.opacities[m])
    _check_render_record(rec, recf, m, scene, cam)
    np.testing.assert_array_equal(bf[m][:, 0:6], recf[m, 14:20])      # conic A..F
    bounded = m & (reci[:, 2] == 0)
    ell = bounded & ((flags & 4) != 0)  # the ellipse has pixels (always, without the low-pass filter)
    if not lowpass:
        np.testing.assert_array_equal(ell, bounded)
    np.testing.assert_array_equal(bf[ell][:, 6:10], recf[ell, 20:24])  # X0, Y0, hx, hy
    np.testing.assert_array_equal((flags[m] & 2) != 0, reci[m, 2] == 1)       # unbounded
    np.testing.assert_array_equal(bi[m][:, 0:4], reci[m][:, [3, 4, 5, 6]])   # pixel range
    np.testing.assert_array_equal(bi[m][:, 4:8], reci[m][:, [7, 8, 9, 10]])  # tile rectangle
    # tile counts per surfel (bounded ones; unbounded ones use the per-view list)
    gc = run.count()[sl]
    np.testing.assert_array_equal(gc[bounded], cnt[bounded])
    return recf, reci


def _check_render_record(rec, recf, m, scene, cam):
    """The render record's adjugate rows are the FP64 adjugate of the shifted
    homography, rounded once: M = s * adj(S^-1 T) with the stored total scale
    s, to a few binary32 ulps of the largest entry (the record is computed in
    double-float so that nearly edge-on surfels keep their accuracy)."""
    T64, _, _, _ = O.geometry(scene, cam, O.make_params())
    for i in np.nonzero(m)[0]:
        xc, yc = float(recf[i, 2]), float(recf[i, 3])
        Tp = np.array([[1, 0, -xc], [0, 1, -yc], [0, 0, 1.0]]) @ T64[i]
        c0, c1, c2 = Tp[:, 0], Tp[:, 1], Tp[:, 2]
        A = np.stack([np.cross(c1, c2), np.cross(c2, c0), np.cross(c0, c1)])
        M = rec[i][[0, 1, 2, 4, 5, 6, 8, 9, 10]].reshape(3, 3).astype(np.float64)
        scale = float(rec[i, 15])
        err = np.abs(M - scale * A).max() / np.abs(M).max()
        assert err <= 2.0 ** -22, (i, err)
        det = np.linalg.det(Tp) * scale
        assert abs(rec[i, 11] - det) <= 1e-5 * abs(det), i


def _check_lists(run, scene, cams, ts, mode, lowpass=0):
    """Sorted per-tile lists of all views equal the oracle's, bit for bit."""
    tile_off = 0
    all_ranges = run.ranges()
    lists = run.lists()
    N = scene.n
    for v, cam in enumerate(cams):
        p = O.make_params(tile_size=ts, lowpass=lowpass)
        b = O.binning(scene, cam, p, MODES[mode])
        nt = O.n_tiles(cam, ts)
        rng = all_ranges[tile_off:tile_off + nt]
        for t in range(nt):
            mine = lists[rng[t, 0]:rng[t, 1]] - v * N
            ref = b["ids"][b["ranges"][t, 0]:b["ranges"][t, 1]]
            np.testing.assert_array_equal(mine, ref, err_msg=f"view {v} tile {t}")
        tile_off += nt


@pytest.mark.parametrize("mode", ["aabb", "snug", "accu"])
@pytest.mark.parametrize("ts", [8, 16, 32])
def test_tiny_scene_binning_bit_exact(mode, ts):
    from tests.gpu_util import GpuRun
    sc, cam = scenes.tiny_scene(seed=0)
    run = GpuRun(sc, [cam], K=4, tile_size=ts, bin_mode=mode, render=False)
    _check_view(run, sc, cam, ts, mode)
    _check_lists(run, sc, [cam], ts, mode)
    b = O.binning(sc, cam, O.make_params(tile_size=ts), MODES[mode])
    assert run.P == b["P"]


def test_room_view_binning_bit_exact():
    from tests.gpu_util import GpuRun
    sc = scenes.room_scene(n=200_000, C=8, seed=1)
    cams = scenes.circle_poses(16)[:2]
    run = GpuRun(sc, cams, K=8, tile_size=16, render=False, cap=1 << 20)
    for v, cam in enumerate(cams):
        _check_view(run, sc, cam, 16, "accu", view=v)
    _check_lists(run, sc, cams, 16, "accu")


def _check_masks(run, scene, cam, ts, lowpass=0):
    """Every pixel centre of a tile inside a listed surfel's binning ellipse
    (FP64 test on the bit-exact binary32 conic), or inside the pixel box of
    an unbounded footprint, or (low-pass filter) inside the screen disc
    2 |x - c|^2 <= k^2 (1 + 2^-10), lies in a warp block that the pair's mask
    keeps (warps own 8 x 4 pixel blocks, row-major over the tile)."""
    p = O.make_params(tile_size=ts, lowpass=lowpass)
    recf, reci, _ = O.mirror_project(scene, cam, p, O.ACCU)
    rng, lists, masks = run.ranges(), run.lists(), run.masks()
    txn = (cam.width + ts - 1) // ts
    tile = np.repeat(np.arange(len(rng)), rng[:, 1] - rng[:, 0])
    ids = lists[rng[0, 0]:rng[-1, 1]]
    masks = masks[rng[0, 0]:rng[-1, 1]]
    X0t, Y0t = (tile % txn) * ts, (tile // txn) * ts
    A, B, C, D, E, F = (recf[ids, 14 + k] for k in range(6))
    xc, yc = recf[ids, 2], recf[ids, 3]
    px0, px1, py0, py1 = (reci[ids, 3 + k] for k in range(4))
    unb = reci[ids, 2] == 1
    covered = 0
    for ly in range(ts):
        for lx in range(ts):
            x, y = X0t + lx, Y0t + ly
            X, Y = x + 0.5 - xc, y + 0.5 - yc
            q = A * X * X + 2 * B * X * Y + C * Y * Y + 2 * D * X + 2 * E * Y + F
            inbox = (x >= px0) & (x <= px1) & (y >= py0) & (y <= py1) & (x < cam.width) & (y < cam.height)
            ell = (A * C - B * B > 0) & (A > 0)
            hit = inbox & (unb | ((q <= 0) & ell))
            if lowpass:
                kb = recf[ids, 1].astype(np.float64) * 1.0009765625
                hit |= inbox & (2 * (X * X + Y * Y) <= kb)
            bit = (masks >> np.uint32((ly // 4) * (ts // 8) + lx // 8)) & 1
            assert not np.any(hit & (bit == 0)), (ts, lx, ly)
            covered += int(hit.sum())
    warps = np.array([bin(int(m)).count("1") for m in masks])
    assert covered > 0 and warps.sum() < len(ids) * (ts * ts // 32)  # the masks do cull


@pytest.mark.parametrize("ts", [8, 16, 32])
def test_warp_masks_cover_every_pixel_inside_the_cutoff(ts):
    from tests.gpu_util import GpuRun
    sc, cam = scenes.tiny_scene(seed=0)
    run = GpuRun(sc, [cam], K=4, tile_size=ts, render=False)
    _check_masks(run, sc, cam, ts)


def test_warp_masks_room_view():
    from tests.gpu_util import GpuRun
    sc = scenes.room_scene(n=200_000, C=8, seed=1)
    cam = scenes.circle_poses(16)[5]
    run = GpuRun(sc, [cam], K=8, tile_size=16, render=False, cap=1 << 20)
    _check_masks(run, sc, cam, 16)


def test_ragged_image_and_small_scene():
    from tests.gpu_util import GpuRun
    sc, _ = scenes.tiny_scene(seed=3, n=300)
    cam = ident_cam(W=100, H=75, f=90.0)
    cam.viewmat[2, 3] = 3.0
    run = GpuRun(sc, [cam], K=4, tile_size=16, render=False)
    _check_view(run, sc, cam, 16, "accu")
    _check_lists(run, sc, [cam], 16, "accu")


def test_capacity_overflow_reports_needed_pairs_and_recovers():
    from paper_2604_10951_gb300 import _lib as L
    from tests.gpu_util import GpuRun, dev
    sc, cam = scenes.tiny_scene(seed=0)
    run = GpuRun(sc, [cam], K=4, render=False, cap=1 << 16)
    need = run.P
    fr = run.frame
    fr._alloc(100)
    fr.project_bin(run.means, run.scales, run.quats, run.opac)
    status, got = fr.read_status()
    assert status == L.FSS_ERR_CAPACITY and got == need
    status, _ = fr.read_status()  # flags are cleared by the read
    assert status == L.FSS_OK
    assert fr.bin_and_sort(run.means, run.scales, run.quats, run.opac) == need


def test_invalid_arguments_are_rejected_without_launch():
    from paper_2604_10951_gb300 import _lib as L
    from paper_2604_10951_gb300.raster import make_cams, make_params
    sc, cam = scenes.tiny_scene(seed=0)
    cams = make_cams([cam])
    bad = [dict(tile_size=12), dict(K=33), dict(C=6, feat_dtype=None), dict(alpha_min=0.0)]
    for kw in bad:
        kw2 = {k: v for k, v in kw.items() if v is not None}
        p = make_params(C=kw2.pop("C", 16), **kw2)
        with pytest.raises(L.FssError) as ei:
            L.fss_workspace_size(p, cams, 1, sc.n, 1000)
        assert ei.value.status in (L.FSS_ERR_INVALID_ARG, L.FSS_ERR_UNSUPPORTED)
    p = make_params(C=16)
    with pytest.raises(L.FssError):
        L.fss_project_bin(p, cams, 1, sc.n, None, None, None, None, None, 1000, None)


def test_tile_order_is_heavy_first_permutation():
    """The tile order the tile kernels follow: a permutation of the tiles of
    all views, with the pair-count bucket (16 pairs) never increasing."""
    import torch
    from paper_2604_10951_gb300 import _lib as L
    from tests.gpu_util import GpuRun
    sc = scenes.room_scene(n=100_000, C=8, seed=2)
    cams = scenes.circle_poses(16)[3:5]
    run = GpuRun(sc, cams, K=8, tile_size=16, render=False, cap=1 << 20)
    torch.cuda.synchronize()
    order = run.frame.region(L.REG_ORDER).view(torch.int32).cpu().numpy()
    ranges = run.frame.region(L.REG_RANGES).view(torch.int32).cpu().numpy().reshape(-1, 2)
    n_tiles = ranges.shape[0]
    assert order.shape[0] == n_tiles
    np.testing.assert_array_equal(np.sort(order), np.arange(n_tiles))
    bucket = np.minimum(255, (ranges[:, 1] - ranges[:, 0]) >> 4)[order]
    assert (np.diff(bucket) <= 0).all()
    assert bucket[0] > bucket[-1]  # the frames have heavy and light tiles


def _dense_tile_scene(n_small=5200, seed=0, C=16):
    """32x32 camera at the origin looking +z (f = 32): n_small camera-facing
    surfels of about 0.4 pixel at depths 2..3 with centres inside tile (0, 0)
    (pixels 2..14): with 5,200 of them that tile's list is longer than the
    1,024 keys the shared-memory sort takes and the per-tile radix sort runs;
    with about 1,000 it fills nearly all 32 chunks of the shared-memory sort."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(2.0, 3.0, n_small)
    px = rng.uniform(2.0, 14.0, n_small)
    py = rng.uniform(2.0, 14.0, n_small)
    f, c = 32.0, 16.0
    means = np.stack([(px - c) / f * z, (py - c) / f * z, z], axis=1)
    log_scales = np.log(np.stack([0.4 * z / f, 0.4 * z / f], axis=1) * rng.uniform(0.8, 1.25, (n_small, 2)))
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (n_small, 1))
    logits = rng.normal(-1.0, 0.5, n_small)
    sc = scenes.Scene(means, log_scales, quats, logits, rng.uniform(0.0, 1.0, (n_small, 3)),
                      rng.normal(0.0, 1.0, (n_small, C)))
    vm = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], dtype=np.float32)
    return sc, scenes.Camera(f, f, c, c, 32, 32, vm)


def test_chunked_sort_for_a_tile_of_nearly_1024_pairs():
    """A tile list of close to the 1,024 keys of the shared-memory sort (32
    warp-sorted chunks of 32 merged by rank, a ragged last chunk): order and
    warp masks bit-exact against the oracle, and the frame's features, ids
    and stop counts against the oracle."""
    from tests.gpu_util import GpuRun
    from tests.test_gpu_render import _compare, _oracle
    sc, cam = _dense_tile_scene(n_small=1000, seed=1)
    run = GpuRun(sc, [cam], K=8)
    r = run.ranges()
    assert 960 < r[0, 1] - r[0, 0] <= 1024 and (r[0, 1] - r[0, 0]) % 32 != 0
    _check_lists(run, sc, [cam], 16, "accu")
    _check_masks(run, sc, cam, 16)
    ref, S = _oracle(sc, cam, 8)
    _compare(run.view(0), ref, S, 1e-4, 8)


def test_radix_sort_branch_for_a_tile_over_4096_pairs():
    """A tile list of more than 4096 pairs (the per-tile LSD radix sort in
    global scratch, with passes skipped where every key has the same digit):
    order and warp masks bit-exact against the oracle, in a two-view call
    (the second view's items have indices above N, so more digits vary), and
    the features, colour, ids and gradients of the frame against the oracle."""
    from tests.gpu_util import GpuRun
    from tests.test_gpu_backward import _assert_close, _gpu_backward, _resolved, _upstream
    from tests.test_gpu_render import _compare, _oracle
    sc, cam = _dense_tile_scene()
    run2 = GpuRun(sc, [cam, cam], K=8, render=False)
    _check_lists(run2, sc, [cam, cam], 16, "accu")
    r = run2.ranges()
    assert r[0, 1] - r[0, 0] > 4096 and r[4, 1] - r[4, 0] > 4096  # tile (0, 0) of each view
    run = GpuRun(sc, [cam], K=8)
    _check_lists(run, sc, [cam], 16, "accu")
    _check_masks(run, sc, cam, 16)
    ref, S = _oracle(sc, cam, 8)
    _compare(run.view(0), ref, S, 1e-4, 8)
    p = O.make_params(K=8)
    ref = _resolved(run, sc, cam, p)
    gF, grgb, gT = _upstream(ref, sc.C, seed=9)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, binned=ref["binned"], flip=ref["flip"])
    _assert_close(_gpu_backward(run, gF, grgb, gT), g_ref)

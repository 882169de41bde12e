"""Pins for Precise Tile Intersection (Sec. 3.2): SnugBox and AccuTile.

The binning mirror decides integers in binary32; these checks tie it to
FP64 geometry: conservativeness against brute-force alpha, nesting of the
three box modes, the fronto-parallel circle, and a sandwich of each AccuTile
tile set between FP64 exact sets at slightly smaller and larger cutoffs.
Sorting and ranges are checked against numpy's lexsort and bincount.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene


@pytest.mark.parametrize("ts", [8, 16, 32])
@pytest.mark.parametrize("mode", [O.AABB, O.SNUG, O.ACCU])
def test_binning_is_conservative_tiny(ts, mode):
    sc, cam = scenes.tiny_scene(seed=20 + ts, n=1500)
    bad, checked = O.check_conservative(sc, cam, O.make_params(tile_size=ts), mode)
    assert checked > 10_000
    assert bad == 0


def test_binning_is_conservative_room_views():
    sc = scenes.room_scene(n=30_000, C=4, seed=21)
    for cam in scenes.circle_poses(16, 320, 240, 262.5)[::5]:
        bad, checked = O.check_conservative(sc, cam, O.make_params(tile_size=16), O.ACCU)
        assert checked > 1000
        assert bad == 0


def test_mode_nesting_and_pair_counts():
    sc, cam = scenes.tiny_scene(seed=22, n=2000)
    p = O.make_params()
    sets = {}
    for mode in (O.AABB, O.SNUG, O.ACCU):
        tiles, ids = O.bin_pairs(sc, cam, p, mode)
        sets[mode] = set(zip(ids.tolist(), tiles.tolist()))
        _, _, cnt = O.mirror_project(sc, cam, p, mode)
        assert cnt.sum() == len(tiles)
    assert sets[O.ACCU] <= sets[O.SNUG] <= sets[O.AABB]
    assert len(sets[O.ACCU]) < len(sets[O.SNUG]) < len(sets[O.AABB])


def test_fronto_parallel_conic_is_circle_of_radius_k_r_f_over_z():
    cam = ident_cam(W=200, H=200, f=150.0)
    z, r, o = 2.5, 0.08, 0.6
    sc = make_scene([[0.1, 0.05, z]], [[r, r]], [[1, 0, 0, 0]], [o])
    recf, reci, cnt = O.mirror_project(sc, cam, O.make_params())
    rec = dict(zip(O.REC_FIELDS, recf[0]))
    kb = np.float32(rec["k2"]) * np.float32(1.0009765625)
    k2 = 2 * np.log(np.float32(o) / np.float32(1 / 255))
    assert rec["k2"] == pytest.approx(k2, rel=1e-7)
    rad = np.sqrt(float(kb)) * float(np.float32(r)) * 150.0 / z
    assert rec["hx"] == pytest.approx(rad, rel=2e-6)
    assert rec["hy"] == pytest.approx(rad, rel=2e-6)
    assert abs(rec["X0"]) < 1e-4 and abs(rec["Y0"]) < 1e-4
    assert rec["xc"] == pytest.approx(100.0 + 150.0 * 0.1 / z, rel=1e-6)
    assert abs(rec["B"]) <= 1e-6 * abs(rec["A"])
    assert rec["A"] == pytest.approx(rec["C"], rel=1e-5)


def _fp64_conic(T, kk):
    c = [T[:, 0], T[:, 1], T[:, 2]]
    m = [np.cross(c[1], c[2]), np.cross(c[2], c[0]), np.cross(c[0], c[1])]
    Q = np.outer(m[0], m[0]) + np.outer(m[1], m[1]) - kk * np.outer(m[2], m[2])
    return Q


def _chord(Q, t, axis):
    """Interval of the other coordinate where the conic is <= 0 along the
    line (axis 0: x = t, returns y-interval; axis 1: y = t, x-interval)."""
    if axis == 0:
        a = Q[1, 1]; b = Q[0, 1] * t + Q[1, 2]; c = Q[0, 0] * t * t + 2 * Q[0, 2] * t + Q[2, 2]
    else:
        a = Q[0, 0]; b = Q[0, 1] * t + Q[0, 2]; c = Q[1, 1] * t * t + 2 * Q[1, 2] * t + Q[2, 2]
    disc = b * b - a * c
    if disc < 0 or a <= 0:
        return None
    s = np.sqrt(disc)
    return (-b - s) / a, (-b + s) / a


def _fp64_accu_set(T, kk, reci, ts, tiles_x):
    """Tiles the AccuTile traversal must list in exact arithmetic."""
    vis, _, unb, px0, px1, py0, py1, tx0, tx1, ty0, ty1 = reci
    Q = _fp64_conic(T, kk)
    out = set()
    rows_outer = (ty1 - ty0 + 1) <= (tx1 - tx0 + 1)
    for ty in range(ty0, ty1 + 1):
        for tx in range(tx0, tx1 + 1):
            ra, rb = max(py0, ty * ts), min(py1, ty * ts + ts - 1)
            ca, cb = max(px0, tx * ts), min(px1, tx * ts + ts - 1)
            if ra > rb or ca > cb:
                continue
            hit = False
            if rows_outer:  # discrete columns, continuous rows of the strip
                for col in range(ca, cb + 1):
                    ch = _chord(Q, col + 0.5, 0)
                    if ch and ch[1] >= ra + 0.5 and ch[0] <= rb + 0.5:
                        hit = True
                        break
            else:
                for row in range(ra, rb + 1):
                    ch = _chord(Q, row + 0.5, 1)
                    if ch and ch[1] >= ca + 0.5 and ch[0] <= cb + 0.5:
                        hit = True
                        break
            if hit:
                out.add(ty * tiles_x + tx)
    return out


@pytest.mark.parametrize("ts", [8, 16])
def test_accutile_sets_sandwiched_by_fp64(ts):
    sc, cam = scenes.tiny_scene(seed=23, n=400)
    p = O.make_params(tile_size=ts)
    recf, reci, cnt = O.mirror_project(sc, cam, p, O.ACCU)
    tiles, ids = O.bin_pairs(sc, cam, p, O.ACCU)
    T, *_ = O.geometry(sc, cam, p)
    tiles_x = (cam.width + ts - 1) // ts
    n_checked = 0
    for i in range(sc.n):
        if not reci[i, 0] or reci[i, 2]:
            continue
        kb = float(np.float32(recf[i, 1]) * np.float32(1.0009765625))
        mine = set(tiles[ids == i].tolist())
        inner = _fp64_accu_set(T[i], kb * (1 - 1e-4), reci[i], ts, tiles_x)
        outer = _fp64_accu_set(T[i], kb * (1 + 1e-4), reci[i], ts, tiles_x)
        assert inner <= mine <= outer, i
        n_checked += 1
    assert n_checked > 300


def test_snugbox_pixel_range_matches_fp64_tight_box():
    sc, cam = scenes.tiny_scene(seed=24, n=500)
    p = O.make_params()
    recf, reci, _ = O.mirror_project(sc, cam, p, O.SNUG)
    T, *_ = O.geometry(sc, cam, p)
    for i in range(sc.n):
        if not reci[i, 0] or reci[i, 2]:
            continue
        kb = float(np.float32(recf[i, 1]) * np.float32(1.0009765625))
        for f, exact in ((1 - 1e-5, False), (1 + 1e-5, True)):
            Q = _fp64_conic(T[i], kb * f)
            A, B, Cc, D, E, F = Q[0, 0], Q[0, 1], Q[1, 1], Q[0, 2], Q[1, 2], Q[2, 2]
            g = A * Cc - B * B
            X0 = (B * E - Cc * D) / g; Y0 = (B * D - A * E) / g
            Fp = F + D * X0 + E * Y0
            hx = np.sqrt(-Fp * Cc / g); hy = np.sqrt(-Fp * A / g)
            lo_x, hi_x = int(np.ceil(X0 - hx - 0.5)), int(np.floor(X0 + hx - 0.5))
            lo_y, hi_y = int(np.ceil(Y0 - hy - 0.5)), int(np.floor(Y0 + hy - 0.5))
            lo_x, lo_y = max(lo_x, 0), max(lo_y, 0)
            hi_x, hi_y = min(hi_x, cam.width - 1), min(hi_y, cam.height - 1)
            if exact:   # slightly larger box contains the mirror's
                assert lo_x <= reci[i, 3] and reci[i, 4] <= hi_x
                assert lo_y <= reci[i, 5] and reci[i, 6] <= hi_y
            else:       # slightly smaller box is contained in it
                assert reci[i, 3] <= lo_x or lo_x > hi_x
                assert hi_x <= reci[i, 4] or lo_x > hi_x
                assert reci[i, 5] <= lo_y or lo_y > hi_y
                assert hi_y <= reci[i, 6] or lo_y > hi_y


def test_sort_order_and_ranges_match_numpy():
    sc, cam = scenes.tiny_scene(seed=25, n=2000)
    p = O.make_params()
    b = O.binning(sc, cam, p)
    tiles, ids = O.bin_pairs(sc, cam, p)
    z = b["recf"][:, 0]
    order = np.lexsort((ids, z[ids].view(np.uint32), tiles))
    np.testing.assert_array_equal(b["tiles"], tiles[order])
    np.testing.assert_array_equal(b["ids"], ids[order])
    nt = O.n_tiles(cam, 16)
    counts = np.bincount(tiles, minlength=nt)
    ends = np.cumsum(counts)
    nz = counts > 0
    np.testing.assert_array_equal(b["ranges"][nz, 1], ends[nz])
    np.testing.assert_array_equal(b["ranges"][nz, 0], (ends - counts)[nz])
    assert np.all(b["ranges"][~nz] == 0)


def test_opacity_aware_cutoff_shrinks_low_opacity_boxes():
    # same surfel at two opacities: k^2 = 2 ln(o / alpha_min) sets the box
    cam = ident_cam(W=128, H=128, f=128.0)
    sc = make_scene([[0, 0, 2.0]] * 2, [[0.1, 0.1]] * 2, [[1, 0, 0, 0]] * 2, [0.95, 0.02])
    recf, reci, cnt = O.mirror_project(sc, cam, O.make_params())
    assert recf[1, 22] < recf[0, 22]
    ratio = recf[1, 22] / recf[0, 22]
    assert ratio == pytest.approx(np.sqrt(np.log(0.02 * 255) / np.log(0.95 * 255)), rel=1e-5)

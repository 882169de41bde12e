"""Pins for the oracle's alternative outcomes at borderline decisions.

A decision of Eq. 2 or Eq. 7 taken within rounding distance of its threshold
can go either way in a binary32 evaluation.  The oracle's per-pixel flip
mask takes such a decision the other way.  Each flipped outcome is pinned
against an independent computation of the other result:

- alpha_min (both directions), the near plane and the T_min stop: the plain
  render with the threshold moved past the borderline value (so that the
  decision is no longer borderline and goes the other way);
- the K-th place of the Top-K set: the other surfel's weight, written out
  from Eq. 2 for two fronto-parallel surfels;
- the exact Top-K stop: the T_min rule, which never stops early;
- the median-depth switch: the closed form of one surfel.

And on random scenes: flipped outcomes keep the invariants of Eq. 2, masks
change nothing at ordinary pixels, the borderline count marks exactly the
flagged pixels, and the test helper that matches GPU results against the
outcomes recovers a result drawn from randomly flipped outcomes.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene
from tests.outcomes import resolve

AMIN = float(np.float32(1.0 / 255.0))
X, Y = 4, 4  # the pixel the constructions aim at (centre 4.5, 4.5)


def _cam():
    return ident_cam(W=8, H=8, f=8.0)


def _surfel_at(cam, z, r, rho_dir=0.0):
    """Mean of a fronto-parallel surfel of scale r at depth z whose
    object-space radius^2 at pixel (X, Y)'s centre is rho_dir."""
    u = np.sqrt(rho_dir)
    x = (X + 0.5 - cam.cx) * z / cam.fx - u * r
    y = (Y + 0.5 - cam.cy) * z / cam.fy
    return [x, y, z]


def _render(sc, cam, flip=0, **kw):
    K = kw.pop("K", 0)
    p = O.make_params(K=K, **kw)
    fl = np.zeros((cam.height, cam.width), np.uint32)
    fl[Y, X] = flip
    return O.render(sc, cam, p, brute=True, flip=fl)


def _same_pixel(a, b, keys=("F", "rgb", "T", "nstop", "ncontrib")):
    for k in keys:
        np.testing.assert_array_equal(a[k][Y, X], b[k][Y, X], err_msg=k)


def test_alpha_min_above_flip_equals_raised_threshold():
    cam = _cam()
    o = np.float32(AMIN + 4e-7)
    sc = make_scene([_surfel_at(cam, 2.0, 0.05)], [[0.05, 0.05]], [[1, 0, 0, 0]], [o], C=3)
    plain = _render(sc, cam)
    assert plain["nborder"][Y, X] == 1 and plain["flags"][Y, X] & O.FLAG_ALPHA
    assert plain["ncontrib"][Y, X] == 1
    flipped = _render(sc, cam, flip=1)
    assert flipped["ncontrib"][Y, X] == 0 and flipped["T"][Y, X] == 1.0
    moved = _render(sc, cam, alpha_min=AMIN + 2e-6)
    assert moved["nborder"][Y, X] == 0
    _same_pixel(flipped, moved)


def test_alpha_min_below_flip_equals_lowered_threshold():
    cam = _cam()
    o = 2 * AMIN
    rho = -2.0 * np.log((AMIN - 4e-7) / o)
    sc = make_scene([_surfel_at(cam, 2.0, 0.05, rho)], [[0.05, 0.05]], [[1, 0, 0, 0]], [o], C=3)
    plain = _render(sc, cam)
    assert plain["nborder"][Y, X] == 1 and plain["ncontrib"][Y, X] == 0
    flipped = _render(sc, cam, flip=1)
    assert flipped["ncontrib"][Y, X] == 1
    moved = _render(sc, cam, alpha_min=AMIN - 2e-6)
    assert moved["nborder"][Y, X] == 0
    _same_pixel(flipped, moved)
    # the blended alpha is o G itself, as Eq. 2 gives it
    assert 1.0 - flipped["T"][Y, X] == pytest.approx(AMIN - 4e-7, abs=2e-9)


def test_near_plane_flip_equals_moved_plane():
    cam = _cam()
    sc = make_scene([_surfel_at(cam, 0.200005, 0.05)], [[0.05, 0.05]], [[1, 0, 0, 0]], [0.5], C=3)
    plain = _render(sc, cam)
    assert plain["nborder"][Y, X] == 1 and plain["flags"][Y, X] & O.FLAG_NEAR and plain["ncontrib"][Y, X] == 1
    flipped = _render(sc, cam, flip=1)
    assert flipped["ncontrib"][Y, X] == 0
    far = _cam()
    far.near = 0.20002
    moved = O.render(sc, far, O.make_params(), brute=True)
    _same_pixel(flipped, moved)


def test_tmin_stop_flip_equals_moved_threshold():
    cam = _cam()
    # two clamped surfels (alpha = alpha_max = 0.99) on the pixel's ray: T after both is (1 - 0.99)^2 = 1e-4
    means = [_surfel_at(cam, 2.0, 0.05), _surfel_at(cam, 3.0, 0.05)]
    sc = make_scene(means, [[0.05, 0.05]] * 2, [[1, 0, 0, 0]] * 2, [0.995, 0.995], C=3)
    plain = _render(sc, cam)
    assert plain["nborder"][Y, X] == 1 and plain["flags"][Y, X] & O.FLAG_TMIN
    flipped = _render(sc, cam, flip=1)
    assert {int(plain["ncontrib"][Y, X]), int(flipped["ncontrib"][Y, X])} == {1, 2}
    tmin = float(np.float32(1e-4))
    # the side the plain decision took decides which way the threshold moves
    shift = 2e-8 if plain["ncontrib"][Y, X] == 2 else -2e-8
    moved = _render(sc, cam, T_min=tmin + shift)
    assert moved["nborder"][Y, X] == 0
    _same_pixel(flipped, moved)


def test_topk_tie_flip_selects_the_other_surfel():
    cam = _cam()
    # K = 1; the near surfel's weight a1 and the far one's a2 (1 - a1) differ by 5e-7
    a1 = 0.4
    a2 = (a1 - 5e-7) / (1 - a1)
    means = [_surfel_at(cam, 2.0, 0.05), _surfel_at(cam, 3.0, 0.05)]
    sc = make_scene(means, [[0.05, 0.05]] * 2, [[1, 0, 0, 0]] * 2, [a1, a2], feats=np.eye(2, dtype=np.float32))
    a1, a2 = float(sc.opacities[0]), float(sc.opacities[1])  # binary32 inputs
    plain = _render(sc, cam, K=1)
    assert plain["nborder"][Y, X] == 1 and plain["flags"][Y, X] & O.FLAG_TIE
    flipped = _render(sc, cam, K=1, flip=1)
    assert plain["ids"][Y, X, 0] == 0 and flipped["ids"][Y, X, 0] == 1
    np.testing.assert_allclose(flipped["F"][Y, X], [0.0, a2 * (1 - a1)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(plain["F"][Y, X], [a1, 0.0], rtol=0, atol=1e-15)
    # the traversal is the same: colour and transmittance do not depend on the selection
    for k in ("rgb", "T", "nstop"):
        np.testing.assert_array_equal(flipped[k][Y, X], plain[k][Y, X])


def test_exact_stop_flip_equals_the_tmin_rule():
    cam = _cam()
    # K = 1: after the first surfel the set is full and alpha_max (1 - a1) <= a1 decides the stop
    a1 = 0.99 / 1.99 + 3e-7
    means = [_surfel_at(cam, 2.0, 0.05), _surfel_at(cam, 3.0, 0.05)]
    sc = make_scene(means, [[0.05, 0.05]] * 2, [[1, 0, 0, 0]] * 2, [a1, 0.5], C=3)
    plain = _render(sc, cam, K=1, stop_rule=O.EXACT_TOPK)
    assert plain["nborder"][Y, X] == 1 and plain["flags"][Y, X] & O.FLAG_EXACT
    assert plain["nstop"][Y, X] == 1
    flipped = _render(sc, cam, K=1, stop_rule=O.EXACT_TOPK, flip=1)
    tmin_rule = _render(sc, cam, K=1, stop_rule=O.TMIN)
    _same_pixel(flipped, tmin_rule, keys=("F", "rgb", "T", "nstop", "ncontrib", "ids"))
    # the features never depend on the stop rule
    np.testing.assert_array_equal(flipped["F"][Y, X], plain["F"][Y, X])


def test_median_depth_flip_closed_form():
    cam = _cam()
    z = 2.5
    sc = make_scene([_surfel_at(cam, z, 0.05)], [[0.05, 0.05]], [[1, 0, 0, 0]], [0.5 + 4e-7], C=3)
    plain = _render(sc, cam)
    assert plain["flags"][Y, X] & O.FLAG_MEDIAN
    assert plain["depth_med"][Y, X] == pytest.approx(z, abs=1e-6)
    flipped = _render(sc, cam, flip=O.FLIP_MEDIAN)
    assert flipped["depth_med"][Y, X] == 0.0
    _same_pixel(flipped, plain, keys=("F", "rgb", "T", "nstop", "ncontrib", "depth", "normal"))


def _flagged_scene():
    # dense enough that some pixels meet borderline decisions
    sc, cam = scenes.tiny_scene(seed=0, n=2000)
    p = O.make_params(K=4, stop_rule=O.EXACT_TOPK)
    b = O.binning(sc, cam, p)
    return sc, cam, p, b


def test_borderline_count_marks_exactly_the_flagged_pixels_and_masks_act_only_there():
    sc, cam, p, b = _flagged_scene()
    plain = O.render(sc, cam, p, binned=b)
    border = plain["nborder"] > 0
    np.testing.assert_array_equal(border, (plain["flags"] & O.FLAGS_BORDER) != 0)
    assert border.any()
    rng = np.random.default_rng(0)
    fl = rng.integers(0, 2 ** 31, size=border.shape, dtype=np.uint32)
    fl[border] = 0
    same = O.render(sc, cam, p, binned=b, flip=fl)
    for k in ("F", "rgb", "T", "ids", "pos", "nstop", "nborder"):
        np.testing.assert_array_equal(same[k], plain[k], err_msg=k)


def test_flipped_outcomes_keep_the_invariants_of_eq2():
    sc, cam, _, _ = _flagged_scene()
    p = O.make_params(K=32)
    b = O.binning(sc, cam, p)
    plain = O.render(sc, cam, p, binned=b)
    border = plain["nborder"] > 0
    assert border.any()
    ones = make_scene(sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, np.ones((sc.n, 1), np.float32))
    for m in (1, 2, 3):
        fl = np.where(border, np.uint32(m), np.uint32(0))
        out = O.render(sc, cam, p, binned=b, flip=fl, only=border)
        one = O.render(ones, cam, p, binned=b, flip=fl, only=border)
        small = border & (out["ncontrib"] <= 32)
        # weights plus final transmittance is one; constant features give 1 - T
        assert np.abs(out["w"].sum(-1) + out["T"] - 1.0)[small].max() < 1e-12
        assert np.abs(one["F"][..., 0] + one["T"] - 1.0)[small].max() < 1e-12


def test_resolver_recovers_randomly_flipped_outcomes():
    sc, cam, p, b = _flagged_scene()
    plain = O.render(sc, cam, p, binned=b)
    border = plain["nborder"] > 0
    rng = np.random.default_rng(1)
    want = np.where(border, rng.integers(0, 2, size=border.shape), 0).astype(np.uint32)
    truth = O.render(sc, cam, p, binned=b, flip=want)
    # a result as the GPU would store it: binary32 values, integer ids and positions
    g = dict(F=truth["F"].astype(np.float32).astype(np.float64), rgb=truth["rgb"].astype(np.float32),
             T=truth["T"].astype(np.float32), ids=truth["ids"], pos=truth["pos"], nstop=truth["nstop"])
    ref, S, flip, unmatched, stats = resolve(g, sc, cam, p, b, 1e-4, p.K)
    assert not unmatched.any() and stats["border"] == int(border.sum())
    assert stats["flipped"] >= 1
    for k in ("ids", "pos", "nstop"):
        np.testing.assert_array_equal(ref[k], truth[k], err_msg=k)
    np.testing.assert_allclose(ref["T"], truth["T"], rtol=0, atol=1e-6)
    # a result that equals no outcome at a borderline pixel stays unmatched
    bad = dict(g, ids=g["ids"].copy())
    y, x = np.argwhere(border)[0]
    bad["ids"][y, x, 0] = -7
    _, _, _, unmatched2, _ = resolve(bad, sc, cam, p, b, 1e-4, p.K)
    assert unmatched2[y, x] and unmatched2.sum() == 1

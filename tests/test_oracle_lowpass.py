"""Pins for the oracle's screen-space low-pass filter (the 2DGS renderer
variant: alpha = o exp(-rho/2) with rho = min(u^2 + v^2, 2 |x - c|^2), c the
projected centre, the screen term taking the centre's depth): the closed
form of a vanishing surfel, equality with the plain render where the object
term always wins, conservative binning of the screen disc (FP64 brute force
over every pixel) in every bin mode, brute force equal to tiled rendering,
and the gradients (including the chain through the projected centre) by
central differences."""
import types

import numpy as np
import pytest

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene


def test_vanishing_surfel_is_the_screen_gaussian():
    cam = ident_cam(W=24, H=20, f=30.0)
    p = np.array([0.07, -0.03, 2.5])
    sc = make_scene([p], [[1e-5, 2e-5]], [[0.9, 0.1, 0.3, 0.2]], [0.8], C=3)
    out = O.render(sc, cam, O.make_params(K=0, lowpass=1), brute=True)
    p = sc.means[0].astype(np.float64)  # the stored binary32 centre
    c = (30.0 * p[0] / p[2] + cam.cx, 30.0 * p[1] / p[2] + cam.cy)
    o = float(sc.opacities[0])
    for py in range(cam.height):
        for px in range(cam.width):
            a = o * np.exp(-((px + 0.5 - c[0]) ** 2 + (py + 0.5 - c[1]) ** 2))
            a = 0.0 if a < 1 / 255 else a
            assert out["T"][py, px] == pytest.approx(1.0 - a, abs=1e-12)
            if a > 0:
                assert out["depth"][py, px] == pytest.approx(a * p[2], abs=1e-12)  # the centre's depth
    assert (out["T"] < 1).sum() >= 9
    # without the filter the same surfel covers no pixel centre
    assert (O.render(sc, cam, O.make_params(K=0), brute=True)["T"] == 1).all()


def test_large_surfels_render_as_without_the_filter():
    cam = ident_cam(W=32, H=32, f=32.0)
    rng = np.random.default_rng(1)
    n = 12
    means = np.c_[rng.uniform(-0.4, 0.4, (n, 2)), rng.uniform(2.0, 3.0, n)]
    sc = make_scene(means, np.full((n, 2), 0.4), [[1, 0, 0, 0]] * n, rng.uniform(0.2, 0.9, n), C=4)
    a = O.render(sc, cam, O.make_params(K=0), brute=True)
    b = O.render(sc, cam, O.make_params(K=0, lowpass=1), brute=True)
    for k in ("F", "rgb", "T"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("mode", [O.AABB, O.SNUG, O.ACCU])
def test_binning_holds_every_screen_disc_pixel(mode):
    sc, cam = scenes.tiny_scene(seed=21, n=1500)
    sc = make_scene(sc.means, sc.scales * 0.05, sc.quats, sc.opacities, sc.rgb, sc.feats)  # most surfels < 1 px
    p = O.make_params(K=4, bin_mode=mode, lowpass=1)
    bad, checked = O.check_conservative(sc, cam, p)
    assert bad == 0 and checked > 5000
    # the plain binning misses pixels that the filter covers
    plain_tiles = O.binning(sc, cam, O.make_params(K=4, bin_mode=mode))["ids"].size
    assert O.binning(sc, cam, p)["ids"].size > plain_tiles


def test_binning_holds_the_room_view():
    sc = scenes.room_scene(n=60_000, C=4, seed=8)
    cam = scenes.circle_poses(16, 160, 120, 131.25)[2]
    for mode in (O.SNUG, O.ACCU):
        bad, checked = O.check_conservative(sc, cam, O.make_params(K=4, bin_mode=mode, lowpass=1))
        assert bad == 0 and checked > 10000


def test_brute_force_equals_tiled():
    sc, cam = scenes.tiny_scene(seed=22, n=800)
    sc = make_scene(sc.means, sc.scales * 0.2, sc.quats, sc.opacities, sc.rgb, sc.feats)
    for mode in (O.AABB, O.ACCU):
        p = O.make_params(K=4, bin_mode=mode, lowpass=1)
        t = O.render(sc, cam, p)
        b = O.render(sc, cam, p, brute=True)
        for k in ("F", "rgb", "T", "ids"):
            np.testing.assert_allclose(t[k], b[k], atol=1e-12)


def test_gradients_by_central_differences():
    sc, cam = scenes.fd_subscene(seed=6)
    s64 = types.SimpleNamespace(means=sc.means.astype(np.float64), scales=sc.scales.astype(np.float64) * 0.15,
                                quats=sc.quats.astype(np.float64), opacities=sc.opacities.astype(np.float64),
                                rgb=sc.rgb.astype(np.float64), feats=sc.feats.astype(np.float64))
    p = O.make_params(K=4, alpha_min=1e-8, T_min=0.0, lowpass=1)
    rng = np.random.default_rng(2)
    H, W = cam.height, cam.width
    gF, grgb, gT = rng.normal(size=(H, W, sc.C)), rng.normal(size=(H, W, 3)), rng.normal(size=(H, W))
    ref = O.render(s64, cam, p, brute=True)
    kink = (ref["flags"] & O.FLAG_LOWPASS) != 0
    gF[kink] = 0; grgb[kink] = 0; gT[kink] = 0
    g = O.render_backward(s64, cam, p, gF, grgb, gT, brute=True)

    def loss():
        out = O.render(s64, cam, p, brute=True)
        return (gF * out["F"]).sum() + (grgb * out["rgb"]).sum() + (gT * out["T"]).sum(), [out["ncontrib"], out["ids"]]

    L0, st0 = loss()
    pick = rng.choice(np.nonzero(np.abs(g["opac"]) > 0)[0], 20, replace=False)
    scale = max(np.abs(g[k][pick]).max() for k in ("means", "scales", "quats", "opac"))
    errs = []
    for i in pick:
        for arr, name, n in ((s64.means, "means", 3), (s64.scales, "scales", 2), (s64.quats, "quats", 4)):
            for k in range(n):
                th = arr[i, k]
                h = 1e-6 * max(1.0, abs(th))
                arr[i, k] = th + h
                Lp, stp = loss()
                arr[i, k] = th - h
                Lm, stm = loss()
                arr[i, k] = th
                if any(not np.array_equal(a, b) or not np.array_equal(a, c) for a, b, c in zip(st0, stp, stm)):
                    continue
                an = g[name][i, k]
                errs.append(abs((Lp - Lm) / (2 * h) - an) / (abs(an) + 1e-4 * scale))
    assert len(errs) > 150
    assert max(errs) < 1e-6, max(errs)

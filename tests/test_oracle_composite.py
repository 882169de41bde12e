"""Pins for the oracle's compositing (Eq. 2) and Top-K Hard Selection (Eq. 7).

Closed forms (one and two fronto-parallel surfels), invariants of the
front-to-back recurrence, reductions of Top-K to full accumulation, and a
numpy brute-force top-K on weights recovered through one-hot features.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene


def _fronto_alpha(cam, p, r, o, x, y):
    u = ((x - cam.cx) * p[2] / cam.fx - p[0]) / r[0]
    v = ((y - cam.cy) * p[2] / cam.fy - p[1]) / r[1]
    return min(0.99, o * np.exp(-0.5 * (u * u + v * v)))


def test_single_surfel_closed_form():
    cam = ident_cam(W=24, H=20, f=24.0)
    sc = make_scene([[0.05, -0.02, 2.0]], [[0.3, 0.2]], [[1, 0, 0, 0]], [0.7], C=5)
    bg = (0.1, 0.2, 0.3)
    out = O.render(sc, cam, O.make_params(K=0, bg=bg), brute=True)
    p = sc.means[0].astype(float); r = sc.scales[0].astype(float); o = float(sc.opacities[0])
    for py in range(cam.height):
        for px in range(cam.width):
            a = _fronto_alpha(cam, p, r, o, px + 0.5, py + 0.5)
            if a < 1 / 255 or (1 - a) < 1e-4:
                a = 0.0
            np.testing.assert_allclose(out["T"][py, px], 1 - a, rtol=0, atol=1e-14)
            np.testing.assert_allclose(out["F"][py, px], a * sc.feats[0].astype(float), atol=1e-13)
            np.testing.assert_allclose(out["rgb"][py, px], a * sc.rgb[0] + (1 - a) * np.array(bg), atol=1e-13)


def test_two_surfels_by_hand():
    # Eq. 2 written out for two surfels: w1 = a1, w2 = a2 (1 - a1), near one first
    cam = ident_cam(W=8, H=8, f=8.0)
    means = [[0.0, 0.0, 3.0], [0.02, 0.01, 2.0]]  # the second is nearer
    sc = make_scene(means, [[0.5, 0.4], [0.3, 0.6]], [[1, 0, 0, 0]] * 2, [0.6, 0.8], C=3)
    out = O.render(sc, cam, O.make_params(K=0), brute=True)
    outk = O.render(sc, cam, O.make_params(K=1), brute=True)
    x, y = 4.5, 3.5
    a_far = _fronto_alpha(cam, sc.means[0].astype(float), sc.scales[0].astype(float), float(sc.opacities[0]), x, y)
    a_near = _fronto_alpha(cam, sc.means[1].astype(float), sc.scales[1].astype(float), float(sc.opacities[1]), x, y)
    w_near, w_far = a_near, a_far * (1 - a_near)
    F = w_near * sc.feats[1].astype(float) + w_far * sc.feats[0].astype(float)
    np.testing.assert_allclose(out["F"][3, 4], F, atol=1e-14)
    assert out["T"][3, 4] == pytest.approx((1 - a_near) * (1 - a_far), abs=1e-15)
    # K = 1 keeps the larger weight only (Eq. 7)
    best = 1 if w_near >= w_far else 0
    np.testing.assert_allclose(outk["F"][3, 4], max(w_near, w_far) * sc.feats[best].astype(float), atol=1e-14)
    assert outk["ids"][3, 4, 0] == best


def test_weights_plus_final_transmittance_is_one():
    sc, cam = scenes.tiny_scene(seed=3, n=600)
    out = O.render(sc, cam, O.make_params(K=32, tile_size=16))
    ok = out["ncontrib"] <= 32
    s = out["w"].sum(-1) + out["T"]
    assert np.abs(s[ok] - 1.0).max() < 1e-12
    # ... and the Top-K weights are the leading factor of the blend: w = alpha T
    assert np.all(out["w"] >= 0) and np.all(out["w"] <= 0.99 + 1e-15)


def test_constant_features_give_one_minus_T():
    sc, cam = scenes.tiny_scene(seed=4, n=500, C=3)
    sc.feats[:] = 1.0
    out = O.render(sc, cam, O.make_params(K=0))
    np.testing.assert_allclose(out["F"][..., 0], 1.0 - out["T"], atol=1e-12)


def test_one_hot_features_recover_weights_and_topk_matches_numpy_brute_force():
    # features e_i turn F into the per-surfel weight vector; numpy then picks
    # the K largest weights (ties to the earlier surfel in depth order)
    sc, cam = scenes.tiny_scene(seed=5, n=120)
    n = sc.n
    sc = make_scene(sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, np.eye(n, dtype=np.float32))
    full = O.render(sc, cam, O.make_params(K=0))
    W = full["F"]  # [H, W, n] weights
    z = O.mirror_project(sc, cam, O.make_params())[0][:, 0]
    order = np.lexsort((np.arange(n), z.view(np.uint32)))
    rank = np.empty(n, int); rank[order] = np.arange(n)
    for K in (1, 3, 6):
        tk = O.render(sc, cam, O.make_params(K=K))
        for py in range(0, cam.height, 7):
            for px in range(0, cam.width, 5):
                w = W[py, px]
                nz = np.nonzero(w > 0)[0]
                if tk["flags"][py, px] & O.FLAG_TIE:
                    continue
                sel = sorted(nz, key=lambda i: (-w[i], rank[i]))[:K]
                expect = np.zeros(n); expect[sel] = w[sel]
                np.testing.assert_allclose(tk["F"][py, px], expect, atol=1e-13)
                ids = tk["ids"][py, px]
                got = [i for i in ids if i >= 0]
                assert got == sorted(sel, key=lambda i: rank[i])  # front-to-back


def test_topk_with_large_K_equals_full_accumulation():
    sc, cam = scenes.tiny_scene(seed=6, n=800)
    full = O.render(sc, cam, O.make_params(K=0))
    big = O.render(sc, cam, O.make_params(K=32))
    ok = full["ncontrib"] <= 32
    assert ok.mean() > 0.9
    np.testing.assert_allclose(big["F"][ok], full["F"][ok], atol=1e-12)
    np.testing.assert_array_equal(big["T"], full["T"])
    np.testing.assert_array_equal(big["rgb"], full["rgb"])


def test_zero_opacity_surfels_change_nothing():
    sc, cam = scenes.tiny_scene(seed=7, n=300)
    extra, _ = scenes.tiny_scene(seed=8, n=100)
    both = make_scene(np.concatenate([sc.means, extra.means]), np.concatenate([sc.scales, extra.scales]),
                      np.concatenate([sc.quats, extra.quats]),
                      np.concatenate([sc.opacities, np.zeros(100, np.float32)]),
                      np.concatenate([sc.rgb, extra.rgb]), np.concatenate([sc.feats, extra.feats]))
    a = O.render(sc, cam, O.make_params(K=4))
    b = O.render(both, cam, O.make_params(K=4))
    for k in ("F", "rgb", "T", "ids", "w"):
        np.testing.assert_array_equal(a[k], b[k])


def test_input_permutation_only_relabels():
    sc, cam = scenes.tiny_scene(seed=9, n=400)
    perm = np.random.default_rng(0).permutation(sc.n)
    a = O.render(sc, cam, O.make_params(K=4))
    b = O.render(sc.subset(perm), cam, O.make_params(K=4))
    np.testing.assert_array_equal(a["F"], b["F"])
    np.testing.assert_array_equal(a["T"], b["T"])
    ids_b = np.where(b["ids"] >= 0, perm[np.maximum(b["ids"], 0)], -1)
    np.testing.assert_array_equal(a["ids"], ids_b)


@pytest.mark.parametrize("ts", [8, 16, 32])
def test_brute_force_equals_tiled_for_every_binning(ts):
    sc, cam = scenes.tiny_scene(seed=10, n=700)
    p = O.make_params(K=4, tile_size=ts)
    ref = None
    for mode in (O.AABB, O.SNUG, O.ACCU):
        p.bin_mode = mode
        b = O.binning(sc, cam, p)
        out = O.render(sc, cam, p, binned=b)
        if ref is None:
            vis = b["reci"][:, 1] == 0
            ref = O.render(sc, cam, p, brute=True, visible=vis, zkey=b["recf"][:, 0])
        for k in ("F", "rgb", "T", "ids", "w", "ncontrib"):
            np.testing.assert_array_equal(out[k], ref[k])


def test_exact_topk_stop_keeps_features_and_shortens_traversal():
    sc, cam = scenes.tiny_scene(seed=11, n=1500)
    a = O.render(sc, cam, O.make_params(K=4, stop_rule=O.TMIN))
    b = O.render(sc, cam, O.make_params(K=4, stop_rule=O.EXACT_TOPK))
    np.testing.assert_allclose(a["F"], b["F"], atol=1e-13)
    np.testing.assert_array_equal(a["ids"], b["ids"])
    assert b["counters"][0] < a["counters"][0]
    assert np.all(b["nstop"] <= a["nstop"])
    # the prefix transmittance bounds the final one from above
    assert np.all(b["T"] >= a["T"] - 1e-15)


def test_front_k_selection_variant_takes_the_first_contributors():
    sc, cam = scenes.tiny_scene(seed=12, n=300)
    sc = make_scene(sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, np.eye(sc.n, dtype=np.float32))
    full = O.render(sc, cam, O.make_params(K=0))
    front = O.render(sc, cam, O.make_params(K=3, select=1))
    z = O.mirror_project(sc, cam, O.make_params())[0][:, 0]
    order = np.lexsort((np.arange(sc.n), z.view(np.uint32)))
    for py in range(0, 128, 9):
        for px in range(0, 128, 11):
            w = full["F"][py, px]
            first = [i for i in order if w[i] > 0][:3]
            assert [i for i in front["ids"][py, px] if i >= 0] == first


def test_front_k_exact_stop_keeps_features_and_stops_after_k_contributors():
    sc, cam = scenes.tiny_scene(seed=13, n=1500)
    a = O.render(sc, cam, O.make_params(K=3, select=1, stop_rule=O.TMIN))
    b = O.render(sc, cam, O.make_params(K=3, select=1, stop_rule=O.EXACT_TOPK))
    np.testing.assert_allclose(a["F"], b["F"], atol=1e-13)
    np.testing.assert_array_equal(a["ids"], b["ids"])
    # the traversal ends at the third contributor: exactly min(3, n) of them
    np.testing.assert_array_equal(b["ncontrib"], np.minimum(a["ncontrib"], 3))
    assert b["counters"][0] < a["counters"][0]


def test_renormalised_topk_constant_and_one_hot_features():
    # the renormalised variant divides the Top-K sum by the selected weights'
    # sum: constant features give exactly 1 wherever a surfel is selected, and
    # one-hot features give the selected weights over their sum
    sc, cam = scenes.tiny_scene(seed=14, n=120)
    n = sc.n
    one = make_scene(sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, np.ones((n, 3), np.float32))
    hot = make_scene(sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, np.eye(n, dtype=np.float32))
    for K, sel in ((1, 0), (4, 0), (4, 1)):
        c = O.render(one, cam, O.make_params(K=K, select=sel, renorm=1))
        has = c["ids"][..., 0] >= 0
        assert has.mean() > 0.3
        np.testing.assert_allclose(c["F"][has], 1.0, atol=1e-14)
        assert (c["F"][~has] == 0).all()
        h = O.render(hot, cam, O.make_params(K=K, select=sel, renorm=1))
        plain = O.render(hot, cam, O.make_params(K=K, select=sel))
        Wk = plain["w"].sum(-1)
        np.testing.assert_allclose(h["F"][has], plain["F"][has] / Wk[has, None], atol=1e-14)
        np.testing.assert_array_equal(h["ids"], plain["ids"])


def test_renormalised_topk_with_large_K_is_the_full_blend_over_its_coverage():
    # K >= every pixel's contributor count: W_K = 1 - T, so the renormalised
    # features are the full blend divided by the covered fraction
    sc, cam = scenes.tiny_scene(seed=6, n=800)
    full = O.render(sc, cam, O.make_params(K=0))
    rn = O.render(sc, cam, O.make_params(K=32, renorm=1))
    ok = (full["ncontrib"] <= 32) & (full["T"] < 1.0)
    assert ok.mean() > 0.5
    np.testing.assert_allclose(rn["F"][ok], full["F"][ok] / (1.0 - full["T"][ok, None]), rtol=1e-11, atol=1e-12)

"""Pins for the oracle's analytic gradients: central finite differences in FP64.

Exact mode (alpha_min = 1e-8, T_min = 0, opacities < alpha_max) keeps every
skip/stop/clamp decision away from the perturbation; a coordinate whose
+-h perturbation still changes the contributor structure or the Top-K set
is excluded and counted.  The loss is the linear functional
L = sum gF.F + grgb.RGB + gT.T, whose gradient is the vector-Jacobian
product the renderer's backward pass computes.
"""
import types

import numpy as np
import pytest

import oracle as O
from paper_2604_10951_gb300 import scenes


def _as64(sc):
    return types.SimpleNamespace(means=sc.means.astype(np.float64), scales=sc.scales.astype(np.float64),
                                 quats=sc.quats.astype(np.float64), opacities=sc.opacities.astype(np.float64),
                                 rgb=sc.rgb.astype(np.float64), feats=sc.feats.astype(np.float64))


def _loss(s64, cam, p, gF, grgb, gT):
    out = O.render(s64, cam, p, brute=True)
    L = (gF * out["F"]).sum() + (grgb * out["rgb"]).sum() + (gT * out["T"]).sum()
    struct = [out["ncontrib"]]
    if p.K:
        struct.append(out["ids"])
    return L, struct


@pytest.mark.parametrize("K,renorm", [(0, 0), (4, 0), (4, 1)])
def test_analytic_gradients_match_central_differences(K, renorm):
    sc, cam = scenes.fd_subscene(seed=5)
    p = O.make_params(K=K, alpha_min=1e-8, T_min=0.0, bg=(0.2, 0.3, 0.1), renorm=renorm)
    rng = np.random.default_rng(1)
    H, W, Cc = cam.height, cam.width, sc.C
    gF = rng.normal(size=(H, W, Cc)); grgb = rng.normal(size=(H, W, 3)); gT = rng.normal(size=(H, W))
    s64 = _as64(sc)
    g = O.render_backward(s64, cam, p, gF, grgb, gT, brute=True)
    L0, st0 = _loss(s64, cam, p, gF, grgb, gT)
    assert np.isfinite(L0)

    active = np.nonzero(np.abs(g["opac"]) > 0)[0]
    assert len(active) > 100
    pick = rng.choice(active, 24, replace=False)
    fields = [("means", 3), ("scales", 2), ("quats", 4), ("opacities", 1), ("rgb", 3), ("feats", Cc)]
    gname = {"means": "means", "scales": "scales", "quats": "quats", "opacities": "opac", "rgb": "rgb", "feats": "feat"}
    errs, excluded, scale = [], 0, 0.0
    for f, _ in fields:
        scale = max(scale, np.abs(g[gname[f]][pick]).max())
    for i in pick:
        for f, n in fields:
            arr = getattr(s64, f)
            for k in range(n):
                idx = (i, k) if arr.ndim == 2 else (i,)
                th = arr[idx]
                h = 1e-6 * max(1.0, abs(th))
                arr[idx] = th + h
                Lp, stp = _loss(s64, cam, p, gF, grgb, gT)
                arr[idx] = th - h
                Lm, stm = _loss(s64, cam, p, gF, grgb, gT)
                arr[idx] = th
                if any(not np.array_equal(a, b) or not np.array_equal(a, c) for a, b, c in zip(st0, stp, stm)):
                    excluded += 1
                    continue
                fd = (Lp - Lm) / (2 * h)
                an = g[gname[f]][idx]
                errs.append(abs(fd - an) / (abs(an) + 1e-4 * scale))
    errs = np.array(errs)
    assert excluded <= 0.02 * (len(errs) + excluded)
    assert len(errs) > 400
    assert errs.max() < 1e-6, (errs.max(), np.argmax(errs))


def test_feature_and_rgb_gradients_are_weight_sums():
    # L is linear in features and colours: dL/dc_i = sum_x w_i(x) gF(x) over
    # the pixels where i is selected (Eq. 7), dL/drgb_i = sum_x w_i(x) grgb(x)
    sc, cam = scenes.tiny_scene(seed=30, n=300, C=6)
    p = O.make_params(K=3)
    out = O.render(sc, cam, p)
    rng = np.random.default_rng(2)
    gF = rng.normal(size=out["F"].shape); grgb = rng.normal(size=out["rgb"].shape)
    g = O.render_backward(sc, cam, p, gF, grgb, None)
    expect = np.zeros((sc.n, sc.C))
    ids, w = out["ids"].reshape(-1, 3), out["w"].reshape(-1, 3)
    gFf = gF.reshape(-1, sc.C)
    for k in range(3):
        m = ids[:, k] >= 0
        np.add.at(expect, ids[m, k], w[m, k, None] * gFf[m])
    np.testing.assert_allclose(g["feat"], expect, atol=1e-11)
    # colour gradient: all contributors, via one-hot colours on a single channel
    assert np.abs(g["rgb"]).max() > 0

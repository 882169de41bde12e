"""GPU parity of the backward render against the oracle's FP64 analytic
gradients (themselves pinned by central finite differences).

Upstream gradients are random; they are zeroed at pixels the oracle flags
(a decision within rounding distance of a threshold), so both sides
differentiate the same piecewise-smooth function.  FP32 tolerance: per
element |g - g_ref| <= 1e-4 |g_ref| + 1e-5 max|g_ref| of that parameter,
and for the geometric parameters (means, scales, quats, opacity) also
1e-5 G_abs, with G_abs the oracle's magnitude chain (the same chain over
absolute values): the forward error bound of an FP32 evaluation, about
170 units in the last place of the magnitudes it sums.  It matters where an
entry is a small sum of large terms of both signs, as for a surfel seen
nearly edge-on.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import render
from tests.gpu_util import GpuRun, dev

pytestmark = pytest.mark.gpu

FLAGS = O.FLAG_ALPHA | O.FLAG_TMIN | O.FLAG_TIE | O.FLAG_EXACT | O.FLAG_NEAR | O.FLAG_CLAMP


def _upstream(ref, C, seed=0, with_T=True):
    rng = np.random.default_rng(seed)
    H, W = ref["T"].shape
    gF = rng.normal(size=(H, W, C))
    grgb = rng.normal(size=(H, W, 3))
    gT = rng.normal(size=(H, W)) if with_T else np.zeros((H, W))
    bad = (ref["flags"] & FLAGS) != 0
    gF[bad] = 0; grgb[bad] = 0; gT[bad] = 0
    return gF, grgb, gT


def _gpu_backward(run, gF, grgb, gT, feat_dtype=torch.float32):
    fr = run.frame
    N = run.scene.n
    out = dict(means=torch.empty(N, 3, device="cuda"), scales=torch.empty(N, 2, device="cuda"),
               quats=torch.empty(N, 4, device="cuda"), opac=torch.empty(N, device="cuda"),
               rgb=torch.empty(N, 3, device="cuda"), feat=torch.empty(N, run.scene.C, device="cuda", dtype=feat_dtype))
    fr.render_backward(run.means, run.scales, run.quats, run.opac, run.rgb, run.feats, run.T,
                       dev(gF.reshape(-1, gF.shape[-1]), feat_dtype), dev(grgb.reshape(-1, 3)),
                       None if gT is None else dev(gT.reshape(-1)),
                       out["means"], out["scales"], out["quats"], out["opac"], out["rgb"], out["feat"])
    torch.cuda.synchronize()
    return {k: v.float().cpu().numpy() for k, v in out.items()}


MAG_COLS = {"means": slice(0, 3), "scales": slice(3, 5), "quats": slice(5, 9), "opac": slice(9, 10)}


def _assert_close(g, ref, rel=1e-4, floor=1e-5, names=("means", "scales", "quats", "opac", "rgb", "feat"), mag=1e-5):
    for k in names:
        a, b = g[k], ref[k]
        scale = np.abs(b).max()
        assert scale > 0, k
        tol = rel * np.abs(b) + floor * scale
        if k in MAG_COLS and "abs" in ref:
            tol = tol + mag * ref["abs"][:, MAG_COLS[k]].reshape(b.shape)
        err = np.abs(a - b) - tol
        assert err.max() <= 0, (k, float((np.abs(a - b) / scale).max()))


@pytest.mark.parametrize("K", [4, 0])
def test_backward_fp32_matches_oracle(K):
    sc, cam = scenes.tiny_scene(seed=0, n=1500)
    run = GpuRun(sc, [cam], K=K, bg=(0.1, 0.2, 0.3))
    p = O.make_params(K=K, bg=(0.1, 0.2, 0.3))
    b = O.binning(sc, cam, p)
    ref = O.render(sc, cam, p, binned=b)
    gF, grgb, gT = _upstream(ref, sc.C)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, binned=b)
    g = _gpu_backward(run, gF, grgb, gT)
    _assert_close(g, g_ref)


def test_backward_without_dT_and_exact_stop():
    sc, cam = scenes.tiny_scene(seed=1, n=1500)
    run = GpuRun(sc, [cam], K=4, stop_rule="exact_topk")
    p = O.make_params(K=4, stop_rule=O.EXACT_TOPK)
    b = O.binning(sc, cam, p)
    ref = O.render(sc, cam, p, binned=b)
    gF, grgb, _ = _upstream(ref, sc.C, seed=1, with_T=False)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, None, binned=b)
    g = _gpu_backward(run, gF, grgb, None)
    _assert_close(g, g_ref)


def test_backward_bf16_features():
    sc, cam = scenes.tiny_scene(seed=2, n=1500, C=32)
    run = GpuRun(sc, [cam], K=8, feat_dtype=torch.bfloat16)
    p = O.make_params(K=8)
    b = O.binning(sc, cam, p)
    f16 = torch.as_tensor(sc.feats).bfloat16().double().numpy()
    ref = O.render(sc, cam, p, feats=f16, binned=b)
    gF, grgb, gT = _upstream(ref, sc.C, seed=2)
    gF = torch.as_tensor(gF).bfloat16().double().numpy()  # the upstream gradient is stored in BF16
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, feats=f16, binned=b)
    g = _gpu_backward(run, gF, grgb, gT, feat_dtype=torch.bfloat16)
    _assert_close(g, g_ref, names=("means", "scales", "quats", "opac", "rgb"))
    # feature gradients are stored in BF16: 2^-8 relative rounding
    _assert_close(g, g_ref, rel=8e-3, floor=1e-4, names=("feat",))


def test_multi_view_gradients_are_sums_of_single_views():
    sc = scenes.room_scene(n=20_000, C=8, seed=3)
    cams = scenes.circle_poses(16, 160, 120, 131.25)[:3]
    multi = GpuRun(sc, cams, K=4)
    rng = np.random.default_rng(3)
    P = multi.frame.total_pix
    gF = rng.normal(size=(P, 8)).astype(np.float32)
    grgb = rng.normal(size=(P, 3)).astype(np.float32)
    gm = _gpu_backward(multi, gF, grgb, None)
    acc = None
    for v, cam in enumerate(cams):
        a, bnd = multi.frame.pix_off[v], multi.frame.pix_off[v + 1]
        single = GpuRun(sc, [cam], K=4)
        gs = _gpu_backward(single, gF[a:bnd], grgb[a:bnd], None)
        acc = gs if acc is None else {k: acc[k] + gs[k] for k in acc}
    for k in acc:
        scale = np.abs(acc[k]).max()
        assert np.abs(gm[k] - acc[k]).max() <= 1e-5 * scale, k


def test_autograd_loss_matches_oracle():
    # L = mean ||F - F_tgt||^2 + mean |rgb - rgb_tgt|  (feature L2 + RGB L1)
    sc, cam = scenes.fd_subscene(seed=5, C=8)
    from paper_2604_10951_gb300.raster import Frame, make_params
    frame = Frame([cam], sc.n, make_params(C=sc.C, K=4), pair_capacity=1 << 16)
    params = [dev(x).requires_grad_() for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, sc.feats)]
    F, rgb, T, ids = render(*params, frame)
    F_t, rgb_t = scenes.targets(4, frame.total_pix, sc.C)
    loss = ((F - dev(F_t)) ** 2).mean() + (rgb - dev(rgb_t)).abs().mean()
    loss.backward()
    p = O.make_params(K=4)
    b = O.binning(sc, cam, p)
    ref = O.render(sc, cam, p, binned=b)
    Fr = ref["F"].reshape(-1, sc.C)
    rr = ref["rgb"].reshape(-1, 3)
    gF = 2 * (Fr - F_t) / Fr.size
    grgb = np.sign(rr - rgb_t) / rr.size
    bad = (ref["flags"] & FLAGS).reshape(-1) != 0
    assert bad.sum() == 0
    g_ref = O.render_backward(sc, cam, p, gF.reshape(ref["F"].shape), grgb.reshape(ref["rgb"].shape), None, binned=b)
    got = dict(zip(("means", "scales", "quats", "opac", "rgb", "feat"), (x.grad.cpu().numpy() for x in params)))
    _assert_close(got, g_ref, rel=1e-3, floor=1e-4)


def test_backward_front_k_selection():
    sc, cam = scenes.tiny_scene(seed=5, n=1500)
    run = GpuRun(sc, [cam], K=4, select="front", stop_rule="exact_topk")
    p = O.make_params(K=4, select=1, stop_rule=O.EXACT_TOPK)
    b = O.binning(sc, cam, p)
    ref = O.render(sc, cam, p, binned=b)
    gF, grgb, gT = _upstream(ref, sc.C, seed=5)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, binned=b)
    g = _gpu_backward(run, gF, grgb, gT)
    _assert_close(g, g_ref)


@pytest.mark.parametrize("select", ["topw", "front"])
def test_backward_renormalised_topk(select):
    sc, cam = scenes.tiny_scene(seed=6, n=1500)
    run = GpuRun(sc, [cam], K=4, select=select, renorm=True)
    p = O.make_params(K=4, select=1 if select == "front" else 0, renorm=1)
    b = O.binning(sc, cam, p)
    ref = O.render(sc, cam, p, binned=b)
    gF, grgb, gT = _upstream(ref, sc.C, seed=6)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, binned=b)
    g = _gpu_backward(run, gF, grgb, gT)
    _assert_close(g, g_ref)

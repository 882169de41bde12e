"""GPU parity of the backward render against the oracle's FP64 analytic
gradients (themselves pinned by central finite differences).

Upstream gradients are random.  The forward's borderline pixels are first
resolved (tests/outcomes.py): the oracle differentiates the outcome the GPU
took there (its flip masks), so both sides differentiate the same
piecewise-smooth function.  Upstream gradients are zeroed only where the
forward cannot tell which side the GPU took: the unmatched borderline pixels
(at most 0.1 %) and alpha within rounding distance of the alpha_max clamp,
where the values are continuous but the derivative switches.  FP32
tolerance: per element |g - g_ref| <= 1e-4 |g_ref| + 1e-5 max|g_ref| of that
parameter, and for the geometric parameters (means, scales, quats, opacity)
also 1e-5 G_abs, with G_abs the oracle's magnitude chain (the same chain
over absolute values): the forward error bound of an FP32 evaluation, about
170 units in the last place of the magnitudes it sums.  It matters where an
entry is a small sum of large terms of both signs, as for a surfel seen
nearly edge-on; ``chain_only`` counts the entries that need it.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import render
from tests.gpu_util import GpuRun, dev
from tests.outcomes import oracle_ref, settle, upstream_mask

pytestmark = pytest.mark.gpu


def _resolved(run, sc, cam, p, tol=1e-4, feats=None, sh=None, g=None):
    """The oracle's forward with the GPU's outcomes at borderline pixels."""
    ref, S = oracle_ref(sc, cam, p, feats=feats, sh=sh)
    settle(run.view(0) if g is None else g, ref, S, tol, p.K)
    return ref


def _upstream(ref, C, seed=0, with_T=True, extra_flags=0):
    rng = np.random.default_rng(seed)
    H, W = ref["T"].shape
    gF = rng.normal(size=(H, W, C))
    grgb = rng.normal(size=(H, W, 3))
    gT = rng.normal(size=(H, W)) if with_T else np.zeros((H, W))
    bad = upstream_mask(ref, extra_flags)
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
    """Returns, per parameter, the number of entries and how many of them
    pass only through the magnitude-chain term."""
    counts = {}
    for k in names:
        a, b = g[k], ref[k]
        scale = np.abs(b).max()
        assert scale > 0, k
        base = rel * np.abs(b) + floor * scale
        tol = base
        if k in MAG_COLS and "abs" in ref:
            tol = base + mag * ref["abs"][:, MAG_COLS[k]].reshape(b.shape)
        d = np.abs(a - b)
        err = d - tol
        assert err.max() <= 0, (k, float((d / scale).max()))
        counts[k] = (int(d.size), int((d > base).sum()))
    if any(c[1] for c in counts.values()):
        print("entries passing only through the magnitude chain:", counts)
    return counts


@pytest.mark.parametrize("K", [4, 0])
def test_backward_fp32_matches_oracle(K):
    sc, cam = scenes.tiny_scene(seed=0, n=1500)
    run = GpuRun(sc, [cam], K=K, bg=(0.1, 0.2, 0.3))
    p = O.make_params(K=K, bg=(0.1, 0.2, 0.3))
    ref = _resolved(run, sc, cam, p)
    gF, grgb, gT = _upstream(ref, sc.C)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, binned=ref["binned"], flip=ref["flip"])
    g = _gpu_backward(run, gF, grgb, gT)
    print(f"K={K} entries (total, passing only through the magnitude chain):", _assert_close(g, g_ref))


def test_backward_without_dT_and_exact_stop():
    sc, cam = scenes.tiny_scene(seed=1, n=1500)
    run = GpuRun(sc, [cam], K=4, stop_rule="exact_topk")
    p = O.make_params(K=4, stop_rule=O.EXACT_TOPK)
    ref = _resolved(run, sc, cam, p)
    gF, grgb, _ = _upstream(ref, sc.C, seed=1, with_T=False)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, None, binned=ref["binned"], flip=ref["flip"])
    g = _gpu_backward(run, gF, grgb, None)
    _assert_close(g, g_ref)


def test_backward_bf16_features():
    sc, cam = scenes.tiny_scene(seed=2, n=1500, C=32)
    run = GpuRun(sc, [cam], K=8, feat_dtype=torch.bfloat16)
    p = O.make_params(K=8)
    f16 = torch.as_tensor(sc.feats).bfloat16().double().numpy()
    ref = _resolved(run, sc, cam, p, tol=2e-2, feats=f16)
    gF, grgb, gT = _upstream(ref, sc.C, seed=2)
    gF = torch.as_tensor(gF).bfloat16().double().numpy()  # the upstream gradient is stored in BF16
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, feats=f16, binned=ref["binned"], flip=ref["flip"])
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


def _loss_grads(frame, F, rgb, sc):
    """The workload's loss L = mean ||F - F_tgt||^2 + mean |rgb - rgb_tgt| and
    its upstream gradients from the GPU's own outputs (so both sides
    differentiate the renderer under the same upstream gradients)."""
    F_t, rgb_t = scenes.targets(4, frame.total_pix, sc.C)
    loss = ((F - dev(F_t)) ** 2).mean() + (rgb - dev(rgb_t)).abs().mean()
    Fg = F.detach().double().cpu().numpy()
    rg = rgb.detach().double().cpu().numpy()
    gF = 2 * (Fg - F_t) / Fg.size
    grgb = np.sign(rg - rgb_t) / rg.size
    return loss, gF, grgb


def _oracle_autograd(sc, cam, p, F, rgb, T, ids, gF, grgb):
    h, w = cam.height, cam.width
    g = dict(F=F.detach().float().cpu().numpy().reshape(h, w, -1), rgb=rgb.detach().cpu().numpy().reshape(h, w, 3),
             T=T.detach().cpu().numpy().reshape(h, w), ids=ids.cpu().numpy().reshape(h, w, -1))
    ref, S = oracle_ref(sc, cam, p)
    settle(g, ref, S, 1e-4, p.K)
    bad = upstream_mask(ref)
    gF = gF.reshape(h, w, -1).copy(); grgb = grgb.reshape(h, w, 3).copy()
    gF[bad] = 0; grgb[bad] = 0
    assert not bad.any()  # the sub-scene has no borderline pixel the forward could not resolve
    return O.render_backward(sc, cam, p, gF, grgb, None, binned=ref["binned"], flip=ref["flip"])


def test_autograd_loss_matches_oracle():
    """render() under torch.autograd on the forward+backward workload's loss
    (feature L2 + RGB L1), on the finite-difference sub-scene, at 1e-4."""
    sc, cam = scenes.fd_subscene(seed=5, C=8)
    from paper_2604_10951_gb300.raster import Frame, make_params
    frame = Frame([cam], sc.n, make_params(C=sc.C, K=4), pair_capacity=1 << 16)
    params = [dev(x).requires_grad_() for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, sc.feats)]
    F, rgb, T, ids = render(*params, frame)
    loss, gF, grgb = _loss_grads(frame, F, rgb, sc)
    loss.backward()
    g_ref = _oracle_autograd(sc, cam, O.make_params(K=4), F, rgb, T, ids, gF, grgb)
    got = dict(zip(("means", "scales", "quats", "opac", "rgb", "feat"), (x.grad.cpu().numpy() for x in params)))
    _assert_close(got, g_ref)


def test_render_raw_log_scales_and_logits_match_oracle():
    """render_raw(): gradients w.r.t. the raw training parameters of the
    forward+backward workload (log-scales, opacity logits, with means,
    quaternions, colours and features), against the oracle's analytic
    gradients chained through scales = exp(log_scales) and opacity =
    sigmoid(logit), at 1e-4."""
    from paper_2604_10951_gb300.raster import Frame, make_params, render_raw
    sc0, cam = scenes.fd_subscene(seed=5, C=8)
    raw = [dev(x).requires_grad_() for x in (sc0.means, sc0.log_scales, sc0.quats, sc0.opacity_logits, sc0.rgb,
                                             sc0.feats)]
    means, ls, quats, logit, rgb_in, feats = raw
    frame = Frame([cam], sc0.n, make_params(C=sc0.C, K=4), pair_capacity=1 << 16)
    F, rgb, T, ids = render_raw(*raw, frame)
    # the activated parameters exactly as the GPU path received them
    scales = torch.exp(ls).detach().cpu().numpy()
    opac = torch.sigmoid(logit).detach().cpu().numpy()
    sc = scenes.Scene(sc0.means, sc0.log_scales, sc0.quats, sc0.opacity_logits, sc0.rgb, sc0.feats, scales=scales,
                      opacities=opac)
    loss, gF, grgb = _loss_grads(frame, F, rgb, sc)
    loss.backward()
    g_ref = _oracle_autograd(sc, cam, O.make_params(K=4), F, rgb, T, ids, gF, grgb)
    s64, o64 = scales.astype(np.float64), opac.astype(np.float64)
    g_ref["scales"] = g_ref["scales"] * s64                   # d/d log_scale = d/d scale * scale
    g_ref["opac"] = g_ref["opac"] * o64 * (1.0 - o64)         # d/d logit = d/d opacity * o (1 - o)
    g_ref["abs"] = g_ref["abs"].copy()
    g_ref["abs"][:, 3:5] *= s64
    g_ref["abs"][:, 9] *= o64 * (1.0 - o64)
    got = dict(zip(("means", "scales", "quats", "opac", "rgb", "feat"), (x.grad.cpu().numpy() for x in raw)))
    _assert_close(got, g_ref)
    assert np.abs(got["scales"]).max() > 0 and np.abs(got["opac"]).max() > 0


def test_backward_front_k_selection():
    sc, cam = scenes.tiny_scene(seed=5, n=1500)
    run = GpuRun(sc, [cam], K=4, select="front", stop_rule="exact_topk")
    p = O.make_params(K=4, select=1, stop_rule=O.EXACT_TOPK)
    ref = _resolved(run, sc, cam, p)
    gF, grgb, gT = _upstream(ref, sc.C, seed=5)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, binned=ref["binned"], flip=ref["flip"])
    g = _gpu_backward(run, gF, grgb, gT)
    _assert_close(g, g_ref)


@pytest.mark.parametrize("select", ["topw", "front"])
def test_backward_renormalised_topk(select):
    sc, cam = scenes.tiny_scene(seed=6, n=1500)
    run = GpuRun(sc, [cam], K=4, select=select, renorm=True)
    p = O.make_params(K=4, select=1 if select == "front" else 0, renorm=1)
    ref = _resolved(run, sc, cam, p)
    gF, grgb, gT = _upstream(ref, sc.C, seed=6)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, binned=ref["binned"], flip=ref["flip"])
    g = _gpu_backward(run, gF, grgb, gT)
    _assert_close(g, g_ref)


@pytest.mark.parametrize("K,schedule", [(8, "grid"), (8, "persistent"), (0, "grid")])
def test_repeated_backward_calls_start_from_zero(K, schedule):
    """The backward's per-slot accumulators are cleared at the sort and again
    by the backward's last kernels after they are read (and the persistent
    work queues are reset there): backward calls repeated on one forward,
    with and without the feature-gradient output, give the same gradients
    each time (equal up to the order of the atomic sums)."""
    from tests.gpu_util import GpuRun
    sc, cam = scenes.tiny_scene(seed=12, n=2500, C=16)
    run = GpuRun(sc, [cam], K=K, stop_rule="tmin", schedule=schedule)
    rng = np.random.default_rng(3)
    gF = rng.normal(0.0, 1.0, run.F.shape).astype(np.float32)
    grgb = rng.normal(0.0, 1.0, run.rgb_out.shape).astype(np.float32)
    first = _gpu_backward(run, gF, grgb, None)
    fr, N = run.frame, run.scene.n
    # a call without the feature-gradient output in between
    outs = [torch.empty(N, 3, device="cuda"), torch.empty(N, 2, device="cuda"), torch.empty(N, 4, device="cuda"),
            torch.empty(N, device="cuda"), torch.empty(N, 3, device="cuda")]
    fr.render_backward(run.means, run.scales, run.quats, run.opac, run.rgb, run.feats, run.T,
                       dev(gF.reshape(-1, gF.shape[-1])), dev(grgb.reshape(-1, 3)), None, *outs, None)
    torch.cuda.synchronize()
    for t, k in zip(outs, ("means", "scales", "quats", "opac", "rgb")):
        scale = np.abs(first[k]).max()
        assert np.abs(t.cpu().numpy() - first[k]).max() <= 1e-5 * scale, k
    for _ in range(2):
        again = _gpu_backward(run, gF, grgb, None)
        for k, v in first.items():
            scale = np.abs(v).max()
            assert scale > 0 and np.abs(again[k] - v).max() <= 1e-5 * scale, k

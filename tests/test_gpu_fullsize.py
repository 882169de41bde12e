"""Parity at the workloads' full sizes, in the launch configuration the bench
uses (BF16 features, Top-K K=8, AccuTile, 16x16 tiles):

- large forward: 1.5M surfels in the room generator, C=128, one 1280x720 view
  (f=900), features and Top-K ids against the FP64 oracle on every pixel;
- forward + backward: 500k surfels, C=64, 640x480, all gradients against the
  oracle's FP64 analytic gradients on the whole frame;
- batched: 1M surfels, C=128, 12 views (4x 320x240, 4x 640x480, 4x 1280x720)
  in one persistent launch replayed from a CUDA graph: every view equal to its
  single-view call bit for bit, the smallest view against the oracle, the
  gradients equal to the sums of the single-view gradients, and the
  autotuner's choice valid.

Inputs of the oracle are the BF16-rounded features (and BF16 upstream feature
gradients), so both sides differentiate the same function; the remaining
difference is FP32 against FP64 arithmetic.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import Frame, make_params
from tests.gpu_util import GpuRun, dev
from tests.outcomes import upstream_mask
from tests.test_gpu_backward import _assert_close, _gpu_backward, _resolved
from tests.test_gpu_render import _compare, _oracle

pytestmark = pytest.mark.gpu


def _bf16(a):
    return torch.as_tensor(np.ascontiguousarray(a)).bfloat16().double().numpy()


def test_large_view_c128_bf16_against_oracle():
    sc = scenes.room_scene(n=1_500_000, C=128, seed=2)
    cam = scenes.circle_poses(32, 1280, 720, 900.0)[7]
    run = GpuRun(sc, [cam], K=8, feat_dtype=torch.bfloat16, out_dtype=torch.bfloat16, cap=1 << 22)
    ref, S = _oracle(sc, cam, 8, feats=_bf16(sc.feats))
    g = run.view(0)
    ok = _compare(g, ref, S, 2e-2, 8)
    err = (np.abs(g["F"] - ref["F"]) / S)[ok]
    print(f"1.5M surfels 1280x720 C=128: feature error / S max {err.max():.2e} mean {err.mean():.2e}, "
          f"outcomes {ref['outcomes']}")


def test_full_frame_backward_bf16_against_oracle():
    sc = scenes.room_scene(n=500_000, C=64, seed=3)
    cam = scenes.circle_poses(16)[0]
    run = GpuRun(sc, [cam], K=8, feat_dtype=torch.bfloat16, stop_rule="exact_topk", cap=1 << 20)
    p = O.make_params(K=8, stop_rule=O.EXACT_TOPK)
    f16 = _bf16(sc.feats)
    ref = _resolved(run, sc, cam, p, tol=2e-2, feats=f16)
    rng = np.random.default_rng(7)
    H, W = ref["T"].shape
    gF = _bf16(rng.normal(size=(H, W, sc.C)))
    grgb = rng.normal(size=(H, W, 3))
    bad = upstream_mask(ref)
    gF[bad] = 0
    grgb[bad] = 0
    g_ref = O.render_backward(sc, cam, p, gF, grgb, None, feats=f16, binned=ref["binned"], flip=ref["flip"])
    g = _gpu_backward(run, gF, grgb, None, feat_dtype=torch.bfloat16)
    # the scope table's 1e-4 relative, plus 1e-5 of the largest entry
    chain = _assert_close(g, g_ref, rel=1e-4, floor=1e-5, names=("means", "scales", "quats", "opac", "rgb"))
    # feature gradients are stored in BF16: 2^-8 relative rounding
    _assert_close(g, g_ref, rel=8e-3, floor=1e-4, names=("feat",))
    print("outcomes", ref["outcomes"], "upstream zeroed at", int(bad.sum()), "pixels")
    print("entries (total, passing only through the magnitude chain):", chain)
    for k in ("means", "scales", "quats", "opac", "rgb", "feat"):
        scale = np.abs(g_ref[k]).max()
        print(f"{k}: max |g - g_ref| / max|g_ref| = {np.abs(g[k] - g_ref[k]).max() / scale:.2e}")


def _grads(frame, ins, T, dF, drgb):
    means, scales, quats, opac, rgb, feats = ins
    out = [torch.empty_like(x) for x in ins]
    frame.render_backward(means, scales, quats, opac, rgb, feats, T, dF, drgb, None, *out)
    return out


def test_batched_twelve_views_one_million_surfels():
    sc = scenes.room_scene(n=1_000_000, C=128, seed=9)
    cams = scenes.batched_cameras()
    ins = [dev(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb)] + [dev(sc.feats, torch.bfloat16)]
    means, scales, quats, opac, rgb, feats = ins
    params = make_params(C=128, K=8, feat_dtype=torch.bfloat16, stop_rule="exact_topk", schedule="persistent")
    fr = Frame(cams, sc.n, params, pair_capacity=1 << 22)
    fr.bin_and_sort(means, scales, quats, opac)
    F, rgb_o, T, ids = fr.new_outputs()
    g = torch.Generator(device="cuda").manual_seed(1)
    dF = torch.randn(F.shape, generator=g, device="cuda").bfloat16()
    drgb = torch.randn(rgb_o.shape, generator=g, device="cuda")
    grads = [torch.empty_like(x) for x in ins]

    def step():
        fr.project_bin(means, scales, quats, opac)
        fr.sort()
        fr.render_forward(rgb, feats, F, rgb_o, T, ids)
        fr.render_backward(means, scales, quats, opac, rgb, feats, T, dF, drgb, None, *grads)

    step()  # sets kernel attributes outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for x in (F, T, *grads):
        x.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert fr.read_status()[0] == 0

    acc = None
    for v, cam in enumerate(cams):
        a, b = fr.pix_off[v], fr.pix_off[v + 1]
        one = Frame([cam], sc.n, make_params(C=128, K=8, feat_dtype=torch.bfloat16, stop_rule="exact_topk"),
                    pair_capacity=1 << 21)
        one.bin_and_sort(means, scales, quats, opac)
        F1, rgb1, T1, ids1 = one.new_outputs()
        one.render_forward(rgb, feats, F1, rgb1, T1, ids1)
        assert torch.equal(F[a:b], F1) and torch.equal(ids[a:b], ids1)
        assert torch.equal(T[a:b], T1) and torch.equal(rgb_o[a:b], rgb1)
        g1 = _grads(one, ins, T1, dF[a:b].contiguous(), drgb[a:b].contiguous())
        acc = [x.float() for x in g1] if acc is None else [p + x.float() for p, x in zip(acc, g1)]
        mag = [x.float().abs() for x in g1] if v == 0 else [m + x.float().abs() for m, x in zip(mag, g1)]
        if v == 0:  # the smallest view against the oracle
            ref, S = _oracle(sc, cam, 8, feats=_bf16(sc.feats), stop=O.EXACT_TOPK)
            h, w = fr.sizes[0]
            gv = dict(F=F1.float().cpu().numpy().reshape(h, w, -1), rgb=rgb1.cpu().numpy().reshape(h, w, 3),
                      T=T1.cpu().numpy().reshape(h, w), ids=ids1.cpu().numpy().reshape(h, w, -1))
            _compare(gv, ref, S, 2e-2, 8)
        del one
    for x, y, m in zip(grads, acc, mag):
        # the same terms summed in another order (the FP32 summation-order bound, a few
        # 1e-4 of the largest entry); BF16 outputs add one rounding (2^-9 relative) per
        # single-view result and one for the batched result
        scale = y.abs().max().item()
        rel = 2.0 ** -8 if x.dtype == torch.bfloat16 else 0.0
        assert bool(((x.float() - y).abs() <= rel * (m + x.float().abs()) + 2e-3 * scale).all())

    from paper_2604_10951_gb300.tune import Autotuner
    best = Autotuner().tune(cams, means, scales, quats, opac, rgb, feats, K=8, reps=2)
    assert best["tile_size"] in (8, 16, 32) and best["schedule"] in ("grid", "persistent")
    print("autotuner on 12 views, 1M surfels:", {k: v for k, v in best.items() if k != "all"})

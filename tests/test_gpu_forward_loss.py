"""fss_render_forward_loss, the forward render with the training loss in the
same call, against the two calls it replaces (fss_render_forward, then
fss_loss_l2_l1 on its outputs) on the same binning:

  - every forward output (F, rgb, T, Top-K ids, the saved positions,
    weights and traversal lengths) and both gradients (dL/dF, dL/drgb) are
    identical bit for bit: the fused kernel forms d = F - F_t from F as it
    stores it, with the loss kernel's operations;
  - the loss differs by the summation order only (1e-5 relative, also
    against its float64 definition on the rendered outputs).

The fused path (the plain Top-K selection with 0 < K <= 8 and the output in
the feature type) runs on BF16 and F32 features, tile sizes 8, 16 and 32,
the grid and persistent schedules, two views of ragged sizes and the
640x480 room view; K = 0, K = 16, the first-K selection and a BF16 output
of F32 features take the two-kernel path inside the call and must agree
the same way."""
import numpy as np
import pytest
import torch

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import _ptr, _stream
from tests.gpu_util import GpuRun, dev

pytestmark = pytest.mark.gpu


def _two_views():
    scene, cam = scenes.tiny_scene(seed=7, n=3000, C=32)
    vm2 = np.array([[0.96, 0.0, 0.28, -0.2], [0.0, 1.0, 0.0, 0.1], [-0.28, 0.0, 0.96, 3.2]], dtype=np.float32)
    cam2 = scenes.Camera(90.0, 90.0, 50.0, 37.0, 100, 75, vm2)  # ragged in both directions
    return scene, [cam, cam2]


def _run_both(scene, cams, wf=1.0, wc=0.5, seed=11, **kw):
    run = GpuRun(scene, cams, render=False, **kw)
    fr, p = run.frame, run.params
    npx = fr.total_pix
    Ft, rgbt = scenes.targets(seed, npx, p.C)
    odt = torch.bfloat16 if p.out_dtype == L.FSS_BF16 else torch.float32
    Ft, rgbt = dev(Ft, odt), dev(rgbt)
    res = []
    for fused in (False, True):
        F, rgb, T, ids = fr.new_outputs()
        dF = torch.full_like(F, float("nan"))
        drgb = torch.full_like(rgb, float("nan"))
        loss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        fr.saved.fill_(0xAB)
        if fused:
            fr.render_forward_loss(run.rgb, run.feats, F, rgb, T, ids, Ft, rgbt, wf, wc, dF, drgb, loss)
        else:
            fr.render_forward(run.rgb, run.feats, F, rgb, T, ids)
            L.fss_loss_l2_l1(p, npx, _ptr(F), _ptr(rgb), _ptr(Ft), _ptr(rgbt), wf, wc, _ptr(dF), _ptr(drgb),
                             _ptr(loss), _stream())
        torch.cuda.synchronize()
        s, _ = fr.read_status()
        assert s == 0
        res.append(dict(F=F, rgb=rgb, T=T, ids=ids, saved=fr.saved.clone(), dF=dF, drgb=drgb, loss=loss.item()))
    a, b = res
    for k in ("F", "rgb", "T", "ids", "saved", "dF", "drgb"):
        if a[k] is None:
            assert b[k] is None
            continue
        x, y = a[k].cpu(), b[k].cpu()
        if x.dtype == torch.bfloat16:
            x, y = x.view(torch.int16), y.view(torch.int16)
        elif x.dtype == torch.float32:
            x, y = x.view(torch.int32), y.view(torch.int32)
        assert torch.equal(x, y), k
    # the loss: the two summation orders and the float64 definition on the rendered outputs
    d = b["F"].double() - Ft.double()
    dc = b["rgb"].double() - rgbt.double()
    ref = wf * float((d * d).mean()) + wc * float(dc.abs().mean())
    assert np.isfinite(b["loss"]) and abs(b["loss"] - ref) <= 1e-5 * ref
    assert abs(a["loss"] - ref) <= 1e-5 * ref
    return a, b


@pytest.mark.parametrize("feat_dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("ts", [8, 16, 32])
def test_two_ragged_views_fused(feat_dtype, ts):
    scene, cams = _two_views()
    _run_both(scene, cams, K=8, tile_size=ts, feat_dtype=feat_dtype, stop_rule="exact_topk")


@pytest.mark.parametrize("K", [1, 4, 8])
def test_k_up_to_8_persistent_schedule(K):
    scene, cams = _two_views()
    _run_both(scene, cams, K=K, feat_dtype=torch.bfloat16, schedule="persistent", wf=0.3, wc=2.0)


@pytest.mark.parametrize("kw", [dict(K=0), dict(K=16), dict(K=8, select="front"),
                                dict(K=8, feat_dtype=torch.float32, out_dtype=torch.bfloat16),
                                dict(K=8, renorm=True)])
def test_two_kernel_and_variant_cases(kw):
    scene, cams = _two_views()
    kw = dict(dict(feat_dtype=torch.bfloat16), **kw)
    _run_both(scene, cams, **kw)


def test_room_view_bf16_k8():
    """The 640x480 room view of the forward+backward workload (200k surfels)."""
    scene = scenes.room_scene(n=200_000, C=64, seed=3)
    cam = scenes.circle_poses(16)[5]
    _run_both(scene, [cam], K=8, feat_dtype=torch.bfloat16, stop_rule="exact_topk", cap=1 << 20)


def test_zero_weights_give_zero_loss_and_gradients():
    scene, cams = _two_views()
    a, b = _run_both(scene, cams, K=8, feat_dtype=torch.bfloat16, wf=0.0, wc=0.0)
    assert b["loss"] == 0.0
    assert not b["dF"].float().abs().any() and not b["drgb"].abs().any()


def test_empty_scene_with_background():
    """No surfels: F = 0, rgb = background, T = 1 everywhere; the loss of those."""
    from tests._scenes import make_scene
    _, cams = _two_views()
    empty = make_scene(np.zeros((0, 3)), np.zeros((0, 2)), np.zeros((0, 4)), np.zeros(0), C=32)
    a, b = _run_both(empty, cams, K=8, feat_dtype=torch.bfloat16, bg=(0.25, 0.5, 0.75))
    assert not b["F"].float().abs().any() and bool((b["T"] == 1.0).all())


def test_graph_replay_equals_the_eager_call():
    """The call captured in a CUDA graph (as the training step replays it) and
    replayed on new targets gives the eager call's outputs on those targets."""
    scene, cams = _two_views()
    run = GpuRun(scene, cams, render=False, K=8, feat_dtype=torch.bfloat16, stop_rule="exact_topk")
    fr = run.frame
    npx, C = fr.total_pix, run.params.C
    tgt = [tuple(dev(x, dt) for x, dt in zip(scenes.targets(s, npx, C), (torch.bfloat16, torch.float32)))
           for s in (21, 22)]
    Ft, rgbt = (torch.empty_like(t) for t in tgt[0])
    outs = fr.new_outputs()
    dF, drgb = torch.empty_like(outs[0]), torch.empty_like(outs[1])
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    call = lambda: fr.render_forward_loss(run.rgb, run.feats, *outs, Ft, rgbt, 1.0, 0.5, dF, drgb, loss)
    Ft.copy_(tgt[0][0])
    rgbt.copy_(tgt[0][1])
    call()  # outside the capture first (kernel attributes)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call()
    Ft.copy_(tgt[1][0])
    rgbt.copy_(tgt[1][1])
    g.replay()
    torch.cuda.synchronize()
    got = [t.clone() for t in (*outs[:3], dF, drgb)] + [loss.item()]
    call()
    torch.cuda.synchronize()
    ref = [t.clone() for t in (*outs[:3], dF, drgb)] + [loss.item()]
    for x, y in zip(got[:-1], ref[:-1]):
        assert torch.equal(x.view(torch.int16) if x.dtype == torch.bfloat16 else x,
                           y.view(torch.int16) if y.dtype == torch.bfloat16 else y)
    assert got[-1] == pytest.approx(ref[-1], rel=1e-6)


def _run_sorted(scene, cams, wf=1.0, wc=0.5, seed=11, **kw):
    """fss_sort then fss_render_forward_loss, against fss_sort_render_forward_loss,
    each on a fresh binning of the same frame: identical lists, warp masks,
    forward outputs, saved buffers and gradients; the loss up to its order."""
    run = GpuRun(scene, cams, render=False, **kw)
    fr, p = run.frame, run.params
    npx = fr.total_pix
    Ft, rgbt = scenes.targets(seed, npx, p.C)
    odt = torch.bfloat16 if p.out_dtype == L.FSS_BF16 else torch.float32
    Ft, rgbt = dev(Ft, odt), dev(rgbt)
    res = []
    for fused in (False, True):
        fr.project_bin(run.means, run.scales, run.quats, run.opac)
        F, rgb, T, ids = fr.new_outputs()
        dF = torch.full_like(F, float("nan"))
        drgb = torch.full_like(rgb, float("nan"))
        loss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        fr.saved.fill_(0xAB)
        if fused:
            fr.sort_render_forward_loss(run.rgb, run.feats, F, rgb, T, ids, Ft, rgbt, wf, wc, dF, drgb, loss)
        else:
            fr.sort()
            fr.render_forward_loss(run.rgb, run.feats, F, rgb, T, ids, Ft, rgbt, wf, wc, dF, drgb, loss)
        torch.cuda.synchronize()
        s, _ = fr.read_status()
        assert s == 0
        res.append(dict(F=F, rgb=rgb, T=T, ids=ids, saved=fr.saved.clone(), dF=dF, drgb=drgb, loss=loss.item(),
                        lists=run.lists().copy(), masks=run.masks().copy()))
    a, b = res
    np.testing.assert_array_equal(a["lists"], b["lists"])
    np.testing.assert_array_equal(a["masks"], b["masks"])
    for k in ("F", "rgb", "T", "ids", "saved", "dF", "drgb"):
        if a[k] is None:
            assert b[k] is None
            continue
        x, y = a[k].cpu(), b[k].cpu()
        if x.dtype == torch.bfloat16:
            x, y = x.view(torch.int16), y.view(torch.int16)
        elif x.dtype == torch.float32:
            x, y = x.view(torch.int32), y.view(torch.int32)
        assert torch.equal(x, y), k
    assert b["loss"] == pytest.approx(a["loss"], rel=1e-6)
    return run


@pytest.mark.parametrize("feat_dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("ts", [8, 16, 32])
def test_sort_in_the_forward_two_ragged_views(feat_dtype, ts):
    scene, cams = _two_views()
    _run_sorted(scene, cams, K=8, tile_size=ts, feat_dtype=feat_dtype, stop_rule="exact_topk")


@pytest.mark.parametrize("kw", [dict(K=4, schedule="persistent"), dict(K=16), dict(K=8, select="front"),
                                dict(K=8, renorm=True), dict(K=0)])
def test_sort_in_the_forward_schedules_and_variants(kw):
    scene, cams = _two_views()
    _run_sorted(scene, cams, **dict(dict(feat_dtype=torch.bfloat16), **kw))


@pytest.mark.parametrize("n_small,views", [(1000, 1), (5200, 2)])
def test_sort_in_the_forward_long_tile_lists(n_small, views):
    """A tile of nearly 1,024 pairs (the shared-memory sort's last chunks) and
    of over 4,096 (the radix sort in global scratch), the latter in two views."""
    from tests.test_gpu_binning import _dense_tile_scene
    sc, cam = _dense_tile_scene(n_small=n_small, seed=1)
    run = _run_sorted(sc, [cam] * views, K=8, feat_dtype=torch.bfloat16)
    r = run.ranges()
    assert r[0, 1] - r[0, 0] > (4096 if n_small > 1024 else 960)


def test_sort_in_the_forward_room_view():
    scene = scenes.room_scene(n=200_000, C=64, seed=3)
    cam = scenes.circle_poses(16)[9]
    _run_sorted(scene, [cam], K=8, feat_dtype=torch.bfloat16, stop_rule="exact_topk", cap=1 << 20)

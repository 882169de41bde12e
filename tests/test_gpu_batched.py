"""Batched multi-view rendering: many cameras of mixed size in one call
(global tiles across views), one-CTA-per-tile or persistent schedule,
replayed from a CUDA graph, with the autotuner's choices.

Per view the batched outputs equal single-view calls bit for bit; tile size
and schedule never change the rendered features.
"""
import numpy as np
import pytest
import torch

from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import Frame, make_params
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def _mixed_cams(scale=0.25):
    sizes = ((int(320 * scale * 2), int(240 * scale * 2), 262.5 * scale * 2),
             (int(640 * scale), int(480 * scale), 525.0 * scale),
             (int(1280 * scale), int(720 * scale), 900.0 * scale))
    return scenes.batched_cameras(sizes=sizes, per_size=4)


def _inputs(sc, dtype=torch.bfloat16):
    return [dev(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb)] + [dev(sc.feats, dtype)]


def _run(frame, ins):
    means, scales, quats, opac, rgb, feats = ins
    frame.bin_and_sort(means, scales, quats, opac)
    F, rgb_o, T, ids = frame.new_outputs()
    frame.render_forward(rgb, feats, F, rgb_o, T, ids)
    torch.cuda.synchronize()
    return F, rgb_o, T, ids


@pytest.mark.parametrize("schedule", ["grid", "persistent"])
def test_batched_views_equal_single_view_calls(schedule):
    sc = scenes.room_scene(n=100_000, C=16, seed=6)
    cams = _mixed_cams()
    ins = _inputs(sc)
    p = make_params(C=16, K=8, feat_dtype=torch.bfloat16, schedule=schedule)
    fr = Frame(cams, sc.n, p, pair_capacity=1 << 20)
    F, rgb, T, ids = _run(fr, ins)
    for v, cam in enumerate(cams):
        one = Frame([cam], sc.n, make_params(C=16, K=8, feat_dtype=torch.bfloat16), pair_capacity=1 << 18)
        F1, rgb1, T1, ids1 = _run(one, ins)
        a, b = fr.pix_off[v], fr.pix_off[v + 1]
        assert torch.equal(F[a:b], F1) and torch.equal(rgb[a:b], rgb1)
        assert torch.equal(T[a:b], T1) and torch.equal(ids[a:b], ids1)


def test_tile_size_and_schedule_do_not_change_features():
    sc = scenes.room_scene(n=60_000, C=16, seed=7)
    cams = _mixed_cams()
    ins = _inputs(sc)
    ref = None
    for ts in (8, 16, 32):
        for schedule in ("grid", "persistent"):
            fr = Frame(cams, sc.n, make_params(C=16, K=8, tile_size=ts, feat_dtype=torch.bfloat16,
                                               schedule=schedule), pair_capacity=1 << 20)
            out = _run(fr, ins)
            if ref is None:
                ref = out
            else:
                for x, y in zip(out, ref):
                    assert torch.equal(x, y), (ts, schedule)


def test_graph_replay_of_batched_fwd_bwd_matches_eager():
    sc = scenes.room_scene(n=60_000, C=16, seed=8)
    cams = _mixed_cams()
    means, scales, quats, opac, rgb, feats = _inputs(sc)
    fr = Frame(cams, sc.n, make_params(C=16, K=8, feat_dtype=torch.bfloat16, schedule="persistent"),
               pair_capacity=1 << 20)
    fr.bin_and_sort(means, scales, quats, opac)
    fr._alloc(int(fr.num_pairs * 1.3) + 1024)
    F, rgb_o, T, ids = fr.new_outputs()
    g = torch.Generator(device="cuda").manual_seed(0)
    dF = torch.randn(F.shape, generator=g, device="cuda").bfloat16()
    drgb = torch.randn(rgb_o.shape, generator=g, device="cuda")
    grads = [torch.empty_like(x) for x in (means, scales, quats, opac, rgb, feats)]

    def step():
        fr.project_bin(means, scales, quats, opac)
        fr.sort()
        fr.render_forward(rgb, feats, F, rgb_o, T, ids)
        fr.render_backward(means, scales, quats, opac, rgb, feats, T, dF, drgb, None, *grads)

    step()
    torch.cuda.synchronize()
    eager = [x.clone() for x in (F, rgb_o, T, ids)] + [x.clone() for x in grads]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for x in (F, rgb_o, T, grads[0]):
        x.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert fr.read_status()[0] == 0
    got = [F, rgb_o, T, ids] + grads
    for k in range(4):
        assert torch.equal(got[k], eager[k])
    for x, y in zip(got[4:], eager[4:]):  # gradient sums use atomics: equal up to rounding order
        scale = y.float().abs().max().item()
        # A gradient entry sums up to (pixels x views) terms of both signs in an
        # order the atomics decide; reordering a binary32 sum of n terms moves it
        # by up to ~n 2^-24 times the sum of the terms' magnitudes, which under
        # cancellation is a few 1e-4 of the tensor's largest entry.  A BF16
        # result may in addition round one BF16 ulp (2^-8 relative) apart.
        rel = 2.0 ** -7 if x.dtype == torch.bfloat16 else 0.0
        tol = rel * y.float().abs() + 2e-3 * scale + 1e-12
        assert bool(((x.float() - y.float()).abs() <= tol).all())


def test_autotuner_picks_a_valid_configuration(tmp_path):
    from paper_2604_10951_gb300.tune import Autotuner
    sc = scenes.room_scene(n=40_000, C=16, seed=9)
    cams = _mixed_cams(scale=0.125)
    means, scales, quats, opac, rgb, feats = _inputs(sc)
    tuner = Autotuner(str(tmp_path / "tune.json"))
    best = tuner.tune(cams, means, scales, quats, opac, rgb, feats, K=8, reps=2)
    assert best["tile_size"] in (8, 16, 32) and best["schedule"] in ("grid", "persistent")
    assert len(best["all"]) == 12 and best["ms"] == min(c["ms"] for c in best["all"])
    again = Autotuner(str(tmp_path / "tune.json")).tune(cams, means, scales, quats, opac, rgb, feats, K=8)
    assert again["tile_size"] == best["tile_size"]

"""GPU parity of the 2DGS screen-space low-pass filter (alpha = o exp(-rho/2),
rho = min(u^2 + v^2, 2 |x - c|^2)): binning bit-exact against the oracle's
binary32 mirror with the screen disc (every bin mode), warp masks that keep
every pixel of the disc, the forward against the FP64 oracle (features,
colour, ids, the sensor depth with the centre depth for the screen term),
and the gradients, whose screen-term part runs through the projected centre.
Borderline decisions are resolved against the oracle's outcomes as in the
other parity tests.  The switch between the two terms leaves the values
continuous but not the derivative, so the sensor depth and the upstream
gradients skip pixels within rounding distance of it (the oracle's low-pass
flag).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import make_scene
from tests.gpu_util import GpuRun, dev
from tests.outcomes import oracle_ref
from tests.test_gpu_backward import _assert_close, _gpu_backward, _resolved, _upstream
from tests.test_gpu_binning import _check_lists, _check_masks, _check_view
from tests.test_gpu_render import _compare

pytestmark = pytest.mark.gpu


def _small(seed=0, n=2000, f=0.05):
    sc, cam = scenes.tiny_scene(seed=seed, n=n)
    return make_scene(sc.means, sc.scales * f, sc.quats, sc.opacities, sc.rgb, sc.feats), cam


@pytest.mark.parametrize("mode", ["aabb", "snug", "accu"])
def test_binning_bit_exact(mode):
    sc, cam = _small()
    run = GpuRun(sc, [cam], K=4, bin_mode=mode, render=False, lowpass=True)
    _check_view(run, sc, cam, 16, mode, lowpass=1)
    _check_lists(run, sc, [cam], 16, mode, lowpass=1)
    b = O.binning(sc, cam, O.make_params(lowpass=1), {"aabb": O.AABB, "snug": O.SNUG, "accu": O.ACCU}[mode])
    assert run.P == b["P"]
    assert run.P > O.binning(sc, cam, O.make_params(), {"aabb": O.AABB, "snug": O.SNUG, "accu": O.ACCU}[mode])["P"]


def test_room_view_binning_and_masks():
    sc = scenes.room_scene(n=200_000, C=8, seed=2)
    cam = scenes.circle_poses(16)[4]
    run = GpuRun(sc, [cam], K=8, render=False, cap=1 << 20, lowpass=True)
    _check_view(run, sc, cam, 16, "accu", lowpass=1)
    _check_lists(run, sc, [cam], 16, "accu", lowpass=1)
    _check_masks(run, sc, cam, 16, lowpass=1)


def test_masks_tiny():
    sc, cam = _small(seed=1)
    run = GpuRun(sc, [cam], K=4, render=False, lowpass=True)
    _check_masks(run, sc, cam, 16, lowpass=1)


@pytest.mark.parametrize("K", [4, 0])
def test_forward_against_oracle(K):
    sc, cam = _small(seed=2, f=0.15)
    run = GpuRun(sc, [cam], K=K, lowpass=True)
    p = O.make_params(K=K, lowpass=1)
    ref, S = oracle_ref(sc, cam, p)
    ok = _compare(run.view(0), ref, S, 1e-4, K)
    plain = GpuRun(sc, [cam], K=K).view(0)
    assert np.abs(run.view(0)["T"] - plain["T"]).max() > 1e-2  # the filter changes the image
    # sensor depth: the screen term takes the centre's depth
    fr = run.frame
    depth = torch.zeros(fr.total_pix, device="cuda")
    F, rgb, T, ids = fr.new_outputs()
    fr.render_forward_aux(run.rgb, run.feats, F, rgb, T, ids, depth)
    torch.cuda.synchronize()
    d = depth.cpu().numpy().reshape(cam.height, cam.width)
    okd = ok & ((ref["flags"] & O.FLAG_LOWPASS) == 0)
    assert (np.abs(d - ref["depth"])[okd] <= 1e-4 * ref["depth"][okd] + 1e-6).all()
    assert torch.equal(F, run.F) and torch.equal(T, run.T)


@pytest.mark.parametrize("K", [4, 0])
def test_gradients_against_oracle(K):
    sc, cam = _small(seed=3, n=1500, f=0.15)
    run = GpuRun(sc, [cam], K=K, lowpass=True)
    p = O.make_params(K=K, lowpass=1)
    ref = _resolved(run, sc, cam, p)
    gF, grgb, gT = _upstream(ref, sc.C, seed=4, extra_flags=O.FLAG_LOWPASS)
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, binned=ref["binned"], flip=ref["flip"])
    g = _gpu_backward(run, gF, grgb, gT)
    _assert_close(g, g_ref)

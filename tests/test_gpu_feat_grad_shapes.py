"""GPU parity of the feature-gradient kernel on the shapes its template and
pass logic branch on, against the oracle's FP64 analytic gradients:

- lanes per feature row G = 1, 2, 4 (with idle lanes: C = 24 BF16 is three
  16-byte chunks in a group of four), 8, 16, 32;
- K that does not divide the thread block (per-entry division) and K that does;
- tile sizes 8 and 32;
- full accumulation (K = 0) with 64- and 128-channel instances;
- a tile whose list is longer than one pass of list positions (2048), with
  selected entries in both passes, and chunks with more distinct surfels than
  one pass of staged feature rows holds.

Tolerances as in test_gpu_backward: FP32 1e-4 relative + 1e-5 of the
largest magnitude; BF16 feature gradients 2^-8 relative.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests.gpu_util import GpuRun
from tests.test_gpu_backward import _assert_close, _gpu_backward, _resolved, _upstream

pytestmark = pytest.mark.gpu


def _check(sc, cam, K, feat_dtype, tile_size=16, seed=0):
    run = GpuRun(sc, [cam], K=K, tile_size=tile_size, feat_dtype=feat_dtype)
    p = O.make_params(K=K, tile_size=tile_size)
    if feat_dtype == torch.bfloat16:
        feats = torch.as_tensor(sc.feats).bfloat16().double().numpy()
    else:
        feats = None
    ref = _resolved(run, sc, cam, p, tol=2e-2 if feat_dtype == torch.bfloat16 else 1e-4, feats=feats)
    b = ref["binned"]
    gF, grgb, gT = _upstream(ref, sc.C, seed=seed)
    if feat_dtype == torch.bfloat16:
        gF = torch.as_tensor(gF).bfloat16().double().numpy()
    g_ref = O.render_backward(sc, cam, p, gF, grgb, gT, feats=feats, binned=b, flip=ref["flip"])
    g = _gpu_backward(run, gF, grgb, gT, feat_dtype=feat_dtype)
    if feat_dtype == torch.bfloat16:
        _assert_close(g, g_ref, names=("means", "scales", "quats", "opac", "rgb"))
        _assert_close(g, g_ref, rel=8e-3, floor=1e-4, names=("feat",))
    else:
        _assert_close(g, g_ref)
    return b


@pytest.mark.parametrize("C,dtype,K,ts", [
    (4, torch.float32, 3, 16),      # G = 1, K does not divide the block
    (8, torch.float32, 5, 16),      # G = 2
    (24, torch.bfloat16, 6, 16),    # G = 4, one idle lane per group
    (64, torch.bfloat16, 8, 8),     # G = 8, tile size 8
    (64, torch.float32, 7, 32),     # G = 16, tile size 32
    (128, torch.float32, 4, 16),    # G = 32
    (256, torch.bfloat16, 2, 16),   # G = 32, BF16
])
def test_feature_gradients_across_group_widths(C, dtype, K, ts):
    sc, cam = scenes.tiny_scene(seed=11 + C, n=1200, C=C)
    _check(sc, cam, K, dtype, tile_size=ts, seed=C)


def _long_list_scene(C, seed=0):
    """32x32 camera at the origin looking +z (f = 32).  2,100 small surfels
    facing the camera at depths 2..3 project into the left half of tile
    (0, 0); one large surfel at depth 5 covers its right half, so that tile's
    list is longer than 2048 and its right-half pixels select an entry at a
    position past 2048."""
    rng = np.random.default_rng(seed)
    n_small = 2100
    z = rng.uniform(2.0, 3.0, n_small)
    px = rng.uniform(0.5, 7.5, n_small)
    py = rng.uniform(0.5, 15.5, n_small)
    f, c = 32.0, 16.0
    means = np.stack([(px - c) / f * z, (py - c) / f * z, z], axis=1)
    # about 0.8 pixel standard deviation
    log_scales = np.log(np.stack([0.8 * z / f, 0.8 * z / f], axis=1) * rng.uniform(0.8, 1.25, (n_small, 2)))
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (n_small, 1))
    logits = rng.normal(0.0, 0.5, n_small)
    zb = 5.0
    big_mean = np.array([[(12.0 - c) / f * zb, (8.0 - c) / f * zb, zb]])
    big_scale = np.log(np.array([[3.0 * zb / f, 5.0 * zb / f]]))
    means = np.concatenate([means, big_mean])
    log_scales = np.concatenate([log_scales, big_scale])
    quats = np.concatenate([quats, [[1.0, 0.0, 0.0, 0.0]]])
    logits = np.concatenate([logits, [2.0]])
    n = n_small + 1
    feats = rng.normal(0.0, 1.0, (n, C))
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sc = scenes.Scene(means, log_scales, quats, logits, rgb, feats)
    vm = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], dtype=np.float32)
    cam = scenes.Camera(f, f, c, c, 32, 32, vm)
    return sc, cam


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_feature_gradients_long_tile_list(dtype):
    sc, cam = _long_list_scene(C=64)
    b = _check(sc, cam, 8, dtype)
    # the scene does what it is for: tile (0, 0) lists more than 2048 surfels
    r = np.asarray(b["ranges"])
    assert r[0, 1] - r[0, 0] > 2048
    p = O.make_params(K=8)
    ref = O.render(sc, cam, p, binned=b)
    pos = np.asarray(ref["pos"])[:16, :16]
    assert (pos >= 2048).any() and ((pos >= 0) & (pos < 2048)).any()


@pytest.mark.parametrize("C,dtype,ts", [
    (64, torch.float32, 16),     # full accumulation, 64-channel instance
    (128, torch.float32, 16),    # 128-channel instance
    (96, torch.bfloat16, 32),    # 128-channel instance, tile size 32, BF16
])
def test_full_accumulation_gradients_wide_features(C, dtype, ts):
    sc, cam = scenes.tiny_scene(seed=31 + C, n=1000, C=C)
    _check(sc, cam, 0, dtype, tile_size=ts, seed=C + 1)

"""GPU parity of the forward render (Eq. 2) and Top-K Hard Selection (Eq. 7).

Features: |F_gpu - F_ref| <= tol * S with S = sum_i w_i |c_i| + 1e-6 (the
magnitude the sum is built from), tol = 1e-4 for FP32 storage and 2e-2 for
BF16 storage.  RGB and T within 2e-5 absolute.  Top-K ids, list positions
and traversal lengths exact.  At pixels where a decision lies within
rounding distance of its threshold (alpha_min, the near plane, the T_min
and exact stops, the K-th place of the Top-K set), both outcomes are
correct: the GPU's result must equal one of the oracle's outcomes there
(tests/outcomes.py), and at most 0.1 % of the pixels may equal none.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene
from tests.gpu_util import GpuRun
from tests.outcomes import oracle_ref, settle

pytestmark = pytest.mark.gpu


def _oracle(scene, cam, K, ts=16, feats=None, stop=O.TMIN, bg=(0, 0, 0), **kw):
    p = O.make_params(K=K, tile_size=ts, stop_rule=stop, bg=bg, **kw)
    return oracle_ref(scene, cam, p, feats=feats)


def _compare(g, ref, S, tol, K):
    """Every pixel against the oracle's outcome the GPU took (ref and S are
    updated in place); returns the compared pixels."""
    ok = settle(g, ref, S, tol, K)
    err = np.abs(g["F"] - ref["F"]) / S
    assert err[ok].max() <= tol, err[ok].max()
    np.testing.assert_allclose(g["rgb"][ok], ref["rgb"][ok], atol=2e-5, rtol=0)
    np.testing.assert_allclose(g["T"][ok], ref["T"][ok], atol=2e-5, rtol=1e-4)
    if K:
        for k in ("ids", "pos", "nstop"):
            if k in g:
                np.testing.assert_array_equal(g[k][ok], ref[k][ok], err_msg=k)
    return ok


@pytest.mark.parametrize("K", [0, 1, 4, 8])
def test_tiny_scene_fp32(K):
    sc, cam = scenes.tiny_scene(seed=0)
    run = GpuRun(sc, [cam], K=K)
    ref, S = _oracle(sc, cam, K)
    _compare(run.view(0), ref, S, 1e-4, K)


def test_tiny_scene_large_K_matches_full_bit_for_bit():
    sc, cam = scenes.tiny_scene(seed=1, n=800)
    full = GpuRun(sc, [cam], K=0).view(0)
    big = GpuRun(sc, [cam], K=32).view(0)
    ref = O.render(sc, cam, O.make_params(K=0))
    small = ref["ncontrib"] <= 32
    assert small.mean() > 0.9
    np.testing.assert_array_equal(big["F"][small], full["F"][small])
    np.testing.assert_array_equal(big["T"], full["T"])
    np.testing.assert_array_equal(big["rgb"], full["rgb"])


@pytest.mark.parametrize("out_dtype", [torch.bfloat16, torch.float32])
def test_bf16_features(out_dtype):
    sc, cam = scenes.tiny_scene(seed=2, C=32)
    run = GpuRun(sc, [cam], K=4, feat_dtype=torch.bfloat16, out_dtype=out_dtype)
    f_bf16 = torch.as_tensor(sc.feats).bfloat16().double().numpy()
    ref, S = _oracle(sc, cam, 4, feats=f_bf16)
    tol = 2e-2 if out_dtype == torch.bfloat16 else 1e-4
    _compare(run.view(0), ref, S, tol, 4)


@pytest.mark.parametrize("ts", [8, 32])
def test_tile_sizes(ts):
    sc, cam = scenes.tiny_scene(seed=3)
    run = GpuRun(sc, [cam], K=4, tile_size=ts)
    ref, S = _oracle(sc, cam, 4, ts=ts)
    g = run.view(0)
    _compare(g, ref, S, 1e-4, 4)
    base = GpuRun(sc, [cam], K=4, tile_size=16).view(0)
    for k in ("F", "rgb", "T", "ids"):
        np.testing.assert_array_equal(g[k], base[k])


def test_renders_identical_across_bin_modes():
    sc, cam = scenes.tiny_scene(seed=4)
    outs = [GpuRun(sc, [cam], K=4, bin_mode=m).view(0) for m in ("aabb", "snug", "accu")]
    for o in outs[1:]:
        for k in ("F", "rgb", "T", "ids"):
            np.testing.assert_array_equal(o[k], outs[0][k])


def test_exact_topk_stop_keeps_features():
    sc, cam = scenes.tiny_scene(seed=5)
    a = GpuRun(sc, [cam], K=4, stop_rule="tmin")
    b = GpuRun(sc, [cam], K=4, stop_rule="exact_topk")
    ga, gb = a.view(0), b.view(0)
    np.testing.assert_array_equal(ga["F"], gb["F"])
    np.testing.assert_array_equal(ga["ids"], gb["ids"])
    assert b.counters()[0] < a.counters()[0]
    ref, S = _oracle(sc, cam, 4, stop=O.EXACT_TOPK)
    _compare(gb, ref, S, 1e-4, 4)


def test_room_view_full_resolution():
    sc = scenes.room_scene(n=500_000, C=64, seed=1)
    cam = scenes.circle_poses(16)[3]
    for K in (8, 0):
        run = GpuRun(sc, [cam], K=K, cap=1 << 20)
        ref, S = _oracle(sc, cam, K)
        _compare(run.view(0), ref, S, 1e-4, K)


def test_ragged_image_background_and_empty_scene():
    sc, _ = scenes.tiny_scene(seed=6, n=400)
    cam = ident_cam(W=100, H=75, f=90.0)
    cam.viewmat[2, 3] = 3.0
    bg = (0.25, 0.5, 0.75)
    run = GpuRun(sc, [cam], K=4, bg=bg)
    ref, S = _oracle(sc, cam, 4, bg=bg)
    _compare(run.view(0), ref, S, 1e-4, 4)
    empty = make_scene(np.zeros((0, 3)), np.zeros((0, 2)), np.zeros((0, 4)), np.zeros(0), C=8)
    e = GpuRun(empty, [cam], K=4, bg=bg).view(0)
    assert np.all(e["T"] == 1.0) and np.all(e["F"] == 0.0) and np.all(e["ids"] == -1)
    np.testing.assert_allclose(e["rgb"], np.broadcast_to(np.array(bg, np.float32), e["rgb"].shape))


def test_counters_match_oracle_contributions():
    sc, cam = scenes.tiny_scene(seed=7)
    run = GpuRun(sc, [cam], K=0)
    ref, _ = _oracle(sc, cam, 0)
    ctr = run.counters()
    assert abs(int(ctr[1]) - int(ref["counters"][1])) <= 0.001 * int(ref["counters"][1])


@pytest.mark.parametrize("K,stop", [(1, "tmin"), (4, "tmin"), (4, "exact_topk"), (12, "exact_topk")])
def test_front_k_selection(K, stop):
    """The first K contributors in depth order (the other reading of Eq. 7)."""
    sc, cam = scenes.tiny_scene(seed=4)
    run = GpuRun(sc, [cam], K=K, stop_rule=stop, select="front")
    p = O.make_params(K=K, stop_rule=O.EXACT_TOPK if stop == "exact_topk" else O.TMIN, select=1)
    ref, S = oracle_ref(sc, cam, p)
    _compare(run.view(0), ref, S, 1e-4, K)


@pytest.mark.parametrize("K,select,feat_dtype", [(4, "topw", torch.float32), (8, "topw", torch.bfloat16),
                                                 (4, "front", torch.float32)])
def test_renormalised_topk(K, select, feat_dtype):
    """The Top-K feature sum divided by the selected weights' sum (a variant of
    Eq. 7); colour, transmittance and ids are those of the plain Top-K call."""
    sc, cam = scenes.tiny_scene(seed=9, C=32)
    run = GpuRun(sc, [cam], K=K, select=select, renorm=True, feat_dtype=feat_dtype)
    feats = torch.as_tensor(sc.feats).to(feat_dtype).double().numpy()
    p = O.make_params(K=K, select=1 if select == "front" else 0, renorm=1)
    ref, S = oracle_ref(sc, cam, p, feats=feats)
    _compare(run.view(0), ref, S, 1e-4 if feat_dtype == torch.float32 else 2e-2, K)
    plain = GpuRun(sc, [cam], K=K, select=select, feat_dtype=feat_dtype).view(0)
    g = run.view(0)
    for k in ("rgb", "T", "ids", "w"):
        np.testing.assert_array_equal(g[k], plain[k])

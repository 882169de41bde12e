"""GPU parity of the sensor outputs of the forward render: expected depth
sum_i w_i z_i, median depth (the hit at which the transmittance first drops
below 1/2, else 0) and the facing normal sum_i w_i n_i, over the same
contributors that composite colour (Eq. 2).

Tolerances follow the FP32 arithmetic of the kernels: the depth sum within
1e-4 of itself (every term is positive), each normal component within
1e-4 (1 - T) + 1e-6 (|n_i| = 1, so the sum of |w_i n_i| is at most
sum w_i = 1 - T), the median depth within 1e-5 relative (one FP32 quotient
det / c2).  Borderline decisions are resolved against the oracle's outcomes
(tests/outcomes.py), and where the transmittance passes within 1e-6 of 1/2
the median depth must equal one of the two outcomes of that switch.
Requesting the sensor outputs changes none of the other outputs: they are
compared bit for bit with the plain forward call.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests.gpu_util import GpuRun
from tests.outcomes import oracle_ref, settle

pytestmark = pytest.mark.gpu


def _aux_run(run):
    fr = run.frame
    n = fr.total_pix
    F, rgb, T, ids = fr.new_outputs()
    depth = torch.full((n,), -7.0, device="cuda")
    med = torch.full((n,), -7.0, device="cuda")
    nrm = torch.full((n, 3), -7.0, device="cuda")
    fr.render_forward_aux(run.rgb, run.feats, F, rgb, T, ids, depth, med, nrm)
    torch.cuda.synchronize()
    assert fr.read_status()[0] == 0
    assert bool((depth != -7).all()) and bool((med != -7).all()) and bool((nrm != -7).all())
    return dict(F=F, rgb=rgb, T=T, ids=ids, depth=depth, med=med, nrm=nrm)


def _ref(run, sc, cam, p, v=0, feats=None, tol=1e-4):
    """The oracle's outputs with the outcomes the GPU took at borderline pixels."""
    ref, S = oracle_ref(sc, cam, p, feats=feats)
    settle(run.view(v), ref, S, tol, p.K)
    return ref


def _check(run, aux, ref, v=0):
    h, w = run.frame.sizes[v]
    a, b = run.frame.pix_off[v], run.frame.pix_off[v + 1]
    for k, plain in (("F", run.F), ("rgb", run.rgb_out), ("T", run.T), ("ids", run.ids)):
        if plain is not None:
            assert torch.equal(aux[k][a:b], plain[a:b]), k
    ok = ~ref["unmatched"]
    d = aux["depth"][a:b].cpu().numpy().reshape(h, w)
    m = aux["med"][a:b].cpu().numpy().reshape(h, w)
    n = aux["nrm"][a:b].cpu().numpy().reshape(h, w, 3)
    T = ref["T"]
    e_d = np.abs(d - ref["depth"])[ok]
    assert (e_d <= 1e-4 * ref["depth"][ok] + 1e-6).all(), e_d.max()
    e_n = np.abs(n - ref["normal"])[ok]
    assert (e_n <= 1e-4 * (1.0 - T[ok])[:, None] + 1e-6).all(), e_n.max()
    # the median switch: one outcome, or either of two where T passes within 1e-6 of 1/2
    med = ref["depth_med"].copy()
    sw = ok & ((ref["flags"] & O.FLAG_MEDIAN) != 0)
    if sw.any():
        c = ref["_ctx"]
        alt = O.render(c["scene"], c["cam"], c["params"], feats=c["feats"], binned=c["binned"],
                       flip=ref["flip"] | np.uint32(O.FLIP_MEDIAN), only=sw)["depth_med"]
        close = lambda x, y: (np.abs(x - y) <= 1e-5 * np.abs(y)) & ((x == 0) == (y == 0))
        take = sw & ~close(m, med) & close(m, alt)
        med[take] = alt[take]
    e_m = np.abs(m - med)[ok]
    assert (e_m <= 1e-5 * med[ok]).all(), e_m.max()
    assert ((m[ok] == 0) == (med[ok] == 0)).all()
    print(f"depth max rel {np.max(e_d / (ref['depth'][ok] + 1e-6)):.2e}, normal max abs {e_n.max():.2e}, "
          f"median max abs {e_m.max() if e_m.size else 0:.2e}, median switches {int(sw.sum())}, "
          f"outcomes {ref['outcomes']}")
    return ok


@pytest.mark.parametrize("K,select,stop", [(0, "topw", "tmin"), (4, "topw", "tmin"), (8, "topw", "exact_topk"),
                                           (4, "front", "exact_topk"), (12, "topw", "tmin")])
def test_sensor_outputs_tiny_scene(K, select, stop):
    sc, cam = scenes.tiny_scene(seed=11)
    run = GpuRun(sc, [cam], K=K, stop_rule=stop, select=select)
    p = O.make_params(K=K, stop_rule=O.EXACT_TOPK if stop == "exact_topk" else O.TMIN,
                      select=1 if select == "front" else 0)
    ref = _ref(run, sc, cam, p)
    aux = _aux_run(run)
    ok = _check(run, aux, ref)
    assert ok.mean() >= 0.999
    assert (ref["depth"] > 0).mean() > 0.3  # the tiny scene covers much of the view


def test_sensor_outputs_room_view_bf16():
    """The bench's launch configuration (BF16 rows, K = 8, exact stop) on a
    full 640x480 room view."""
    sc = scenes.room_scene(n=500_000, C=64, seed=4)
    cam = scenes.circle_poses(16)[5]
    run = GpuRun(sc, [cam], K=8, feat_dtype=torch.bfloat16, stop_rule="exact_topk", cap=1 << 20)
    p = O.make_params(K=8, stop_rule=O.EXACT_TOPK)
    ref = _ref(run, sc, cam, p, feats=torch.as_tensor(sc.feats).bfloat16().double().numpy(), tol=2e-2)
    aux = _aux_run(run)
    ok = _check(run, aux, ref)
    assert ok.mean() >= 0.999


def test_sensor_outputs_batched_views_and_partial_requests():
    """Three views in one launch (persistent schedule) equal each single-view
    call; a call that asks for the normal alone gets the same normals."""
    sc = scenes.room_scene(n=200_000, C=16, seed=5)
    cams = scenes.circle_poses(8, 320, 240, 262.5)[:3]
    run = GpuRun(sc, cams, K=8, stop_rule="exact_topk", schedule="persistent", cap=1 << 20)
    aux = _aux_run(run)
    p = O.make_params(K=8, stop_rule=O.EXACT_TOPK)
    for v, cam in enumerate(cams):
        _check(run, aux, _ref(run, sc, cam, p, v), v)
    fr = run.frame
    nrm = torch.zeros(fr.total_pix, 3, device="cuda")
    F, rgb, T, ids = fr.new_outputs()
    fr.render_forward_aux(run.rgb, run.feats, F, rgb, T, ids, None, None, nrm)
    torch.cuda.synchronize()
    assert torch.equal(nrm, aux["nrm"])
    assert torch.equal(F, aux["F"]) and torch.equal(ids, aux["ids"])

"""GPU parity of the query-guided instance labels (Sec. 3.3) and of the
per-pixel instance mask rendered from them.

Labels: the tensor-core kernel against the FP64 oracle on the same BF16
inputs.  The logits sum exact BF16 products in FP32 (at most dim 2^-24 of
sum |f_q f_ins| off), and the proximity, exponentials and softmax run in
FP32, so each label is within 5e-5 of itself (plus 1e-7); BF16 storage adds
2^-8 relative rounding.  Shapes cover ragged Gaussian counts (not multiples
of the 128-row tile), every query and feature width class up to 256 x 128,
and the full 500k-Gaussian room workload.

Mask: the labels rendered by the Top-K (and full) renderer with C = n_queries
and the per-pixel argmax output, against the argmax of the oracle's render
of its own labels, with the outcome the GPU took at borderline decisions
(tests/outcomes.py); pixels whose two largest channels lie within 2e-4 of
the larger one (1e-2 with BF16 label storage, twice its rounding) have two
correct argmaxes and are left out of the mask comparison, and counted.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import query_labels
from tests._scenes import make_scene
from tests.gpu_util import GpuRun, dev
from tests.outcomes import oracle_ref, settle

pytestmark = pytest.mark.gpu


def _bf(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).bfloat16()


def _run(means, f_ins, f_q, p_q, prec, out_dtype=torch.float32):
    out = query_labels(_bf(f_ins).cuda(), dev(means), _bf(f_q).cuda(), dev(p_q), dev(prec), out_dtype=out_dtype)
    torch.cuda.synchronize()
    ref = O.query_labels(_bf(f_ins).double().numpy(), means, _bf(f_q).double().numpy(), p_q, prec)
    return out.float().cpu().numpy(), ref


@pytest.mark.parametrize("n,nq,dim", [(1000, 32, 32), (777, 16, 16), (2049, 48, 64), (300, 256, 128),
                                      (130, 128, 32)])
def test_labels_against_oracle(n, nq, dim):
    sc = scenes.room_scene(n=max(n, 5000), C=4, seed=n)
    means = sc.means[:n]
    f_ins, f_q, p_q, prec = scenes.room_queries(means, nq, dim, seed=nq + dim)
    got, ref = _run(means, f_ins, f_q, p_q, prec)
    err = np.abs(got - ref)
    assert (err <= 5e-5 * ref + 1e-7).all(), (err / ref).max()
    gotb, _ = _run(means, f_ins, f_q, p_q, prec, torch.bfloat16)
    assert (np.abs(gotb - ref) <= (2.0 ** -8 + 5e-5) * ref + 1e-7).all()  # BF16: 8 significant bits
    print(f"N={n} nq={nq} dim={dim}: max rel err {(err / ref).max():.2e}")


def test_labels_full_room_workload():
    """500k Gaussians, 32 queries, 32-d instance features (the paper's widths)."""
    sc = scenes.room_scene(n=500_000, C=4, seed=3)
    f_ins, f_q, p_q, prec = scenes.room_queries(sc.means, 32, 32, seed=0)
    got, ref = _run(sc.means, f_ins, f_q, p_q, prec)
    err = np.abs(got - ref) / ref
    assert err.max() <= 5e-5, err.max()
    # the rows are distributions, and the labels separate the instances
    np.testing.assert_allclose(got.sum(1), 1.0, atol=1e-5)
    assert (got.argmax(1) == ref.argmax(1)).mean() > 0.999
    print(f"500k x 32 labels: max rel err {err.max():.2e}")


def test_empty_input_and_argument_checks():
    f_q = _bf(np.zeros((16, 16))).cuda()
    z3 = torch.zeros(16, 3, device="cuda")
    z6 = torch.zeros(16, 6, device="cuda")
    out = query_labels(torch.zeros(0, 16, dtype=torch.bfloat16, device="cuda"), torch.zeros(0, 3, device="cuda"),
                       f_q, z3, z6)
    assert out.shape == (0, 16)
    with pytest.raises(RuntimeError):
        query_labels(torch.zeros(4, 24, dtype=torch.bfloat16, device="cuda"), torch.zeros(4, 3, device="cuda"),
                     _bf(np.zeros((16, 24))).cuda(), z3, z6)


def _label_scene(n, nq, C_dtype, seed):
    sc = scenes.room_scene(n=n, C=4, seed=seed)
    f_ins, f_q, p_q, prec = scenes.room_queries(sc.means, nq, 32, seed=seed)
    gpu_l = query_labels(_bf(f_ins).cuda(), dev(sc.means), _bf(f_q).cuda(), dev(p_q), dev(prec), out_dtype=C_dtype)
    ref_l = O.query_labels(_bf(f_ins).double().numpy(), sc.means, _bf(f_q).double().numpy(), p_q, prec)
    return sc, gpu_l, ref_l


@pytest.mark.parametrize("K,feat_dtype", [(8, torch.bfloat16), (4, torch.float32), (0, torch.float32)])
def test_rendered_instance_mask(K, feat_dtype):
    nq = 32
    sc, gpu_l, ref_l = _label_scene(200_000, nq, feat_dtype, seed=5)
    cam = scenes.circle_poses(8, 320, 240, 262.5)[2]
    lab_sc = make_scene(sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, ref_l.astype(np.float32))
    run = GpuRun(lab_sc, [cam], K=K, feat_dtype=feat_dtype, stop_rule="exact_topk" if K else "tmin", cap=1 << 20,
                 render=False)
    fr = run.frame
    F, rgb, T, ids = fr.new_outputs()
    label = torch.full((fr.total_pix,), -7, dtype=torch.int32, device="cuda")
    fr.render_forward_aux(run.rgb, gpu_l, F, rgb, T, ids, label=label)
    torch.cuda.synchronize()
    # the argmax call without features gives the same mask
    label2 = torch.full_like(label, -7)
    fr.render_forward_aux(run.rgb, gpu_l, None, None, None, None, label=label2)
    torch.cuda.synchronize()
    assert torch.equal(label, label2)
    p = O.make_params(K=K, stop_rule=O.EXACT_TOPK if K else O.TMIN)
    tol = 1e-4 if feat_dtype == torch.float32 else 2e-2
    h, w = fr.sizes[0]
    g_lab = label.cpu().numpy().reshape(h, w)
    g_F = F.float().cpu().numpy().reshape(h, w, nq)
    g = dict(F=g_F, rgb=rgb.cpu().numpy().reshape(h, w, 3), T=T.cpu().numpy().reshape(h, w))
    if K:
        g["ids"] = ids.cpu().numpy().reshape(h, w, K)
    ref, S = oracle_ref(lab_sc, cam, p, feats=ref_l)
    okf = settle(g, ref, S, tol, K)  # the GPU's outcome at borderline pixels
    Fr = ref["F"]
    srt = np.sort(Fr, -1)
    # BF16 label storage moves each rendered channel by up to 2^-8 of itself
    gap = 2e-4 if feat_dtype == torch.float32 else 1e-2
    gap_ok = (srt[..., -1] - srt[..., -2]) > gap * srt[..., -1]
    none = (ref["ids"][..., 0] < 0) if K else (ref["ncontrib"] == 0)
    want = np.where(none, -1, Fr.argmax(-1))
    ok = okf & (gap_ok | none)
    assert ok.mean() > (0.97 if feat_dtype == torch.float32 else 0.8), ok.mean()
    np.testing.assert_array_equal(g_lab[ok], want[ok])
    assert (g_lab >= -1).all() and (g_lab < nq).all()
    # the rendered label features themselves (S = F: every label is positive)
    assert (np.abs(g_F - Fr)[okf] <= tol * Fr[okf] + 1e-6).all()
    print(f"K={K} {feat_dtype}: mask equal on all {ok.mean():.4f} of the pixels compared, {(want[ok] >= 0).mean():.3f} of them covered")

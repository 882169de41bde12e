"""fss_forward_static: the forward frame on the library's static device
scratch array, called through the C ABI, against the ordinary entry points
(fss_project_bin, fss_sort, fss_render_forward on a caller workspace).

The forward pass is deterministic (each tile's list is in a total order and
every pixel's arithmetic is fixed), so the outputs must match bit for bit on
every call, and a call must not depend on what the previous one left in the
shared array.  This file is collected last so that it also runs after every
other GPU test in the same process.
"""
import ctypes as C

import pytest
import torch

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import Frame, _ptr, _stream, make_params
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def _inputs(sc, feat_dtype):
    return [dev(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb)] + [dev(sc.feats, feat_dtype)]


def _reference(cams, sc, params, ins):
    fr = Frame(cams, sc.n, params, pair_capacity=1 << 16)
    means, scales, quats, opac, rgb, feats = ins
    fr.bin_and_sort(means, scales, quats, opac)
    outs = fr.new_outputs()
    fr.render_forward(rgb, feats, *outs)
    torch.cuda.synchronize()
    return fr, outs


def _static(fr, params, ins, cap):
    """One fss_forward_static call into fresh NaN/-2-filled outputs."""
    F, rgb_o, T, ids = fr.new_outputs()
    for x in (F, rgb_o, T):
        x.fill_(float("nan"))
    if ids is not None:
        ids.fill_(-2)
    saved = torch.full_like(fr.saved, 0xAB)
    means, scales, quats, opac, rgb, feats = ins
    st, n = L.fss_forward_static(params, fr.cams, fr.n_cams, fr.N, cap, _ptr(means), _ptr(scales), _ptr(quats),
                                 _ptr(opac), _ptr(rgb), _ptr(feats), _ptr(F), _ptr(rgb_o), _ptr(T), _ptr(ids),
                                 _ptr(saved), _stream())
    return st, n, (F, rgb_o, T, ids), saved


def _assert_same(got, ref, saved, ref_saved):
    for x, y in zip(got, ref):
        if y is None:
            assert x is None
        else:
            assert torch.equal(x, y)
    assert torch.equal(saved, ref_saved)


@pytest.mark.parametrize("case", ["tiny_f32_k4", "two_views_bf16_k8", "full_accumulation"])
def test_static_forward_matches_workspace_forward_twice(case):
    if case == "tiny_f32_k4":
        sc, cam = scenes.tiny_scene(seed=0, n=2000, C=16)
        cams, params = [cam], make_params(C=16, K=4)
        feat_dtype = torch.float32
    elif case == "two_views_bf16_k8":
        sc = scenes.room_scene(n=20_000, C=16, seed=4)
        cams = scenes.circle_poses(n_poses=2, width=160, height=120, f=131.25)
        feat_dtype = torch.bfloat16
        params = make_params(C=16, K=8, feat_dtype=feat_dtype, stop_rule="exact_topk", schedule="persistent")
    else:
        sc, cam = scenes.tiny_scene(seed=1, n=3000, C=32)
        cams, params = [cam], make_params(C=32, K=0, tile_size=8)
        feat_dtype = torch.float32
    ins = _inputs(sc, feat_dtype)
    fr, ref = _reference(cams, sc, params, ins)
    cap = fr.num_pairs + 64
    assert L.fss_workspace_size(params, fr.cams, fr.n_cams, fr.N, cap) <= L.FSS_STATIC_SCRATCH_BYTES
    for _ in range(2):  # two calls in a row on the same static array
        st, n, got, saved = _static(fr, params, ins, cap)
        assert st == L.FSS_OK and n == fr.num_pairs
        _assert_same(got, ref, saved, fr.saved)


def test_static_forward_reports_capacity_then_recovers():
    sc, cam = scenes.tiny_scene(seed=2, n=2000, C=16)
    params = make_params(C=16, K=4)
    ins = _inputs(sc, torch.float32)
    fr, ref = _reference([cam], sc, params, ins)
    st, need, _, _ = _static(fr, params, ins, cap=fr.num_pairs // 2)
    assert st == L.FSS_ERR_CAPACITY and need == fr.num_pairs
    st, n, got, saved = _static(fr, params, ins, cap=need)  # the error word must not carry over
    assert st == L.FSS_OK and n == need
    _assert_same(got, ref, saved, fr.saved)


def test_static_forward_rejects_frames_over_the_limit():
    sc, cam = scenes.tiny_scene(seed=0, n=2000, C=16)
    params = make_params(C=16, K=4)
    ins = _inputs(sc, torch.float32)
    fr = Frame([cam], sc.n, params, pair_capacity=1 << 10)
    big_cap = L.FSS_STATIC_SCRATCH_BYTES // 16
    assert L.fss_workspace_size(params, fr.cams, 1, sc.n, big_cap) > L.FSS_STATIC_SCRATCH_BYTES
    with pytest.raises(L.FssError) as ei:
        _static(fr, params, ins, cap=big_cap)
    assert ei.value.status == L.FSS_ERR_UNSUPPORTED and "FSS_STATIC_SCRATCH_BYTES" in str(ei.value)
    # the rejected call launched nothing; the next one works
    fr2, ref = _reference([cam], sc, params, ins)
    st, n, got, saved = _static(fr2, params, ins, cap=fr2.num_pairs)
    assert st == L.FSS_OK
    _assert_same(got, ref, saved, fr2.saved)


def test_static_forward_calls_leave_device_memory_unchanged():
    """After a first call (which loads the module and looks up the array),
    further calls change neither the device's free memory (cudaMemGetInfo:
    no allocation by the library, the runtime or a library it calls) nor
    torch's allocated bytes; outputs are allocated before the calls."""
    sc, cam = scenes.tiny_scene(seed=3, n=2000, C=16)
    params = make_params(C=16, K=4)
    ins = _inputs(sc, torch.float32)
    fr, ref = _reference([cam], sc, params, ins)
    cap = fr.num_pairs + 64
    F, rgb_o, T, ids = fr.new_outputs()
    saved = torch.empty_like(fr.saved)
    means, scales, quats, opac, rgb, feats = ins

    def call():
        return L.fss_forward_static(params, fr.cams, fr.n_cams, fr.N, cap, _ptr(means), _ptr(scales), _ptr(quats),
                                    _ptr(opac), _ptr(rgb), _ptr(feats), _ptr(F), _ptr(rgb_o), _ptr(T), _ptr(ids),
                                    _ptr(saved), _stream())

    assert call()[0] == L.FSS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(5):
        assert call()[0] == L.FSS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    _assert_same((F, rgb_o, T, ids), ref, saved, fr.saved)

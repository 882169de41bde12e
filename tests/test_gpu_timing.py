"""The kernel-event hook: one event per launched kernel, in launch order, on
the launch stream, also inside a captured CUDA graph."""
import pytest
import torch

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import Frame, make_params
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu

N_KERNELS = 2 + 1 + 1 + 4 + 1  # binning (project; emit with the tile scan), sort, forward, backward, rows


def _frame():
    sc = scenes.room_scene(n=50_000, C=16, seed=11)
    cam = scenes.circle_poses(16)[2]
    ins = [dev(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb)] + [dev(sc.feats, torch.bfloat16)]
    fr = Frame([cam], sc.n, make_params(C=16, K=8, feat_dtype=torch.bfloat16), pair_capacity=1 << 20)
    fr.bin_and_sort(*ins[:4])
    return fr, ins


def _step(fr, ins, outs, grads, dF, drgb):
    means, scales, quats, opac, rgb, feats = ins
    F, rgb_o, T, ids = outs
    fr.project_bin(means, scales, quats, opac)
    fr.sort()
    fr.render_forward(rgb, feats, F, rgb_o, T, ids)
    fr.render_backward(means, scales, quats, opac, rgb, feats, T, dF, drgb, None, *grads)


@pytest.mark.parametrize("graph", [False, True])
def test_one_event_per_kernel_in_order(graph):
    fr, ins = _frame()
    outs = fr.new_outputs()
    dF = torch.randn(outs[0].shape, device="cuda").bfloat16()
    drgb = torch.randn(outs[1].shape, device="cuda")
    grads = [torch.empty_like(x) for x in ins]
    ev = [torch.cuda.Event(enable_timing=True, external=True)] + \
         [torch.cuda.Event(enable_timing=True) for _ in range(N_KERNELS + 2)]
    for e in ev:
        e.record()
    torch.cuda.synchronize()
    try:
        if graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                ev[0].record()
                L.fss_set_kernel_events(ev[1:N_KERNELS + 1])
                _step(fr, ins, outs, grads, dF, drgb)
                L.fss_set_kernel_events([])
            end = torch.cuda.Event(enable_timing=True)
            g.replay()
            end.record()
        else:
            ev[0].record()
            L.fss_set_kernel_events(ev[1:N_KERNELS + 1])
            _step(fr, ins, outs, grads, dF, drgb)
            L.fss_set_kernel_events([])
            end = torch.cuda.Event(enable_timing=True)
            end.record()
    finally:
        L.fss_set_kernel_events([])
    torch.cuda.synchronize()
    assert fr.read_status()[0] == L.FSS_OK
    t = [ev[k].elapsed_time(ev[k + 1]) for k in range(N_KERNELS)]
    assert all(x >= 0.0 for x in t)
    total = ev[0].elapsed_time(end)
    assert sum(t) <= total + 1e-3 and sum(t) >= 0.5 * total
    # no event beyond the n given is recorded: the spare ones keep their time from
    # before the step, so they lie at least the whole step before its end
    for k in (N_KERNELS + 1, N_KERNELS + 2):
        assert ev[k].elapsed_time(end) >= total - 1e-3

"""The autograd path without host synchronisation: a Frame with deferred
status checks renders and differentiates through render() without waiting
for the device, so a whole training step (forward, loss, backward) can be
captured in a CUDA graph and replayed.  Capacity overflow surfaces at the
explicit check after the step.

The replayed gradients equal the eager ones up to the order of the atomic
sums (each gradient entry sums terms over pixels in arrival order: within
1e-5 of the tensor's largest entry); the forward outputs are equal bit for
bit.
"""
import numpy as np
import pytest
import torch

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import Frame, make_params, render
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def _setup(cap=1 << 18, seed=0):
    sc, cam = scenes.tiny_scene(seed=seed, n=1500, C=8)
    frame = Frame([cam], sc.n, make_params(C=sc.C, K=4, stop_rule="exact_topk"), pair_capacity=cap, deferred=True)
    params = [dev(x).requires_grad_() for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb, sc.feats)]
    F_t, rgb_t = scenes.targets(4, frame.total_pix, sc.C)
    return sc, frame, params, dev(F_t), dev(rgb_t)


def _step(frame, params, F_t, rgb_t):
    F, rgb, T, ids = render(*params, frame)
    loss = ((F - F_t) ** 2).mean() + (rgb - rgb_t).abs().mean()
    loss.backward()
    return F, rgb, T, ids, loss


def _close(a, b, name):
    scale = b.abs().max().item()
    assert scale > 0, name
    assert (a - b).abs().max().item() <= 1e-5 * scale, name


def test_render_forward_backward_replays_from_a_cuda_graph():
    sc, frame, params, F_t, rgb_t = _setup()
    # eager reference; its autograd graph is dropped (detached outputs), so the capture
    # below builds its own gradient-accumulation nodes on the capturing stream
    F0, rgb0, T0, ids0, _ = (x.detach() for x in _step(frame, params, F_t, rgb_t))
    assert frame.check() > 0
    g_eager = [p.grad.clone() for p in params]
    for p in params:
        p.grad = None
    # warm up on a side stream, then capture forward + loss + backward
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            for p in params:
                p.grad = None
            _step(frame, params, F_t, rgb_t)
    torch.cuda.current_stream().wait_stream(s)
    for p in params:
        p.grad = None
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        F, rgb, T, ids, loss = _step(frame, params, F_t, rgb_t)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    frame.check()
    assert torch.equal(F, F0) and torch.equal(T, T0) and torch.equal(ids, ids0) and torch.equal(rgb, rgb0)
    for p, g, name in zip(params, g_eager, ("means", "scales", "quats", "opac", "rgb", "feat")):
        _close(p.grad, g, name)
    # the replay follows new inputs written into the captured parameters
    with torch.no_grad():
        params[4].mul_(0.5)
    graph.replay()
    torch.cuda.synchronize()
    assert not torch.equal(rgb, rgb0)


def test_deferred_overflow_is_reported_by_check_and_recovers_after_grow():
    sc, frame, params, F_t, rgb_t = _setup(cap=64)
    _step(frame, params, F_t, rgb_t)  # no synchronisation: the overflow stays on the device
    with pytest.raises(L.FssError) as ei:
        frame.check()
    assert ei.value.status == L.FSS_ERR_CAPACITY
    need = ei.value.needed
    assert need > 64
    frame.grow(need)
    for p in params:
        p.grad = None
    F, rgb, T, ids, _ = _step(frame, params, F_t, rgb_t)
    assert frame.check() == need
    # the same step through a frame with the status read at every forward
    ref = Frame(frame.cams_py, sc.n, frame.params, pair_capacity=1 << 18)
    params2 = [p.detach().clone().requires_grad_() for p in params]
    F2, rgb2, T2, ids2, _ = _step(ref, params2, F_t, rgb_t)
    assert torch.equal(F, F2) and torch.equal(ids, ids2)
    for a, b, name in zip(params, params2, ("means", "scales", "quats", "opac", "rgb", "feat")):
        _close(a.grad, b.grad, name)

"""Torch-facing wrapper over the C ABI: device buffers, streams, autograd.

Every step of the rasterizer runs in ``libfss.so``; this module only owns
torch tensors (workspace, outputs), passes their pointers and the current
stream, and wires the backward call into ``torch.autograd``.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import torch

from . import _lib as L

BIN_MODES = {"aabb": L.FSS_BIN_AABB, "snug": L.FSS_BIN_SNUG, "accu": L.FSS_BIN_ACCU}
STOP_RULES = {"tmin": L.FSS_STOP_TMIN, "exact_topk": L.FSS_STOP_EXACT_TOPK}
SCHEDULES = {"grid": L.FSS_SCHED_GRID, "persistent": L.FSS_SCHED_PERSISTENT}
SELECTS = {"topw": L.FSS_SELECT_TOPW, "front": L.FSS_SELECT_FRONT}
DTYPES = {torch.float32: L.FSS_F32, torch.bfloat16: L.FSS_BF16}
TORCH_DTYPES = {L.FSS_F32: torch.float32, L.FSS_BF16: torch.bfloat16}


def make_params(C: int, K: int = 8, tile_size: int = 16, bin_mode="accu", stop_rule="tmin",
                alpha_min: float = 1.0 / 255.0, alpha_max: float = 0.99, T_min: float = 1e-4,
                feat_dtype=torch.float32, out_dtype=None, bg=(0.0, 0.0, 0.0),
                schedule="grid", select="topw", renorm=False, sh_degree=None, lowpass=False) -> L.fss_params:
    p = L.fss_default_params()
    p.tile_size, p.K, p.C = int(tile_size), int(K), int(C)
    p.bin_mode = BIN_MODES[bin_mode] if isinstance(bin_mode, str) else int(bin_mode)
    p.stop_rule = STOP_RULES[stop_rule] if isinstance(stop_rule, str) else int(stop_rule)
    p.alpha_min, p.alpha_max, p.T_min = float(alpha_min), float(alpha_max), float(T_min)
    p.feat_dtype = DTYPES[feat_dtype] if isinstance(feat_dtype, torch.dtype) else int(feat_dtype)
    od = feat_dtype if out_dtype is None else out_dtype
    p.out_dtype = DTYPES[od] if isinstance(od, torch.dtype) else int(od)
    for k in range(3):
        p.bg_rgb[k] = float(bg[k])
    p.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    p.select = SELECTS[select] if isinstance(select, str) else int(select)
    p.renorm = int(bool(renorm))
    p.lowpass = int(bool(lowpass))
    if sh_degree is not None:  # view-dependent colours: rgb arguments hold [N, (d+1)^2, 3] coefficients
        p.color_mode, p.sh_degree = L.FSS_COLOR_SH, int(sh_degree)
    return p


def make_cams(cams: Sequence) -> "C.Array":
    """ctypes array of fss_camera from objects with fx, fy, cx, cy, width,
    height, viewmat (3x4) and near."""
    arr = (L.fss_camera * len(cams))()
    for c, src in zip(arr, cams):
        c.fx, c.fy, c.cx, c.cy = float(src.fx), float(src.fy), float(src.cx), float(src.cy)
        c.width, c.height = int(src.width), int(src.height)
        vm = torch.as_tensor(src.viewmat, dtype=torch.float32).reshape(12).tolist()
        for k in range(12):
            c.viewmat[k] = vm[k]
        c.near_plane = float(getattr(src, "near", 0.2))
    return arr


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Frame:
    """Workspace and per-pixel buffers for one set of cameras, N surfels and
    one parameter block.  One forward may be in flight per frame (the
    backward pass reads the binning and the saved buffer it left).

    ``deferred=True`` makes :meth:`forward` (and so :func:`render` under
    autograd) asynchronous: it never waits for the device, so a training
    step can run ahead of the host or be captured in a CUDA graph.  The pair
    capacity is then fixed at construction; the caller calls :meth:`check`
    after the step (or after several), which raises ``FssError`` with status
    ``FSS_ERR_CAPACITY`` and the needed pair count if a frame overflowed.
    The outputs and gradients of an overflowed step are incomplete: grow
    the frame (:meth:`grow`) and run the step again."""

    def __init__(self, cams: Sequence, N: int, params: L.fss_params, pair_capacity: int = 1 << 20,
                 device: Optional[torch.device] = None, deferred: bool = False):
        if not torch.cuda.is_available():
            raise RuntimeError("the rasterizer needs a CUDA device (sm_103a)")
        L.lib()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.cams_py = list(cams)
        self.cams = make_cams(self.cams_py)
        self.n_cams = len(self.cams_py)
        self.N = int(N)
        self.params = params
        self.sizes = [(int(c.height), int(c.width)) for c in self.cams_py]
        self.total_pix = sum(h * w for h, w in self.sizes)
        self.pix_off = [0]
        for h, w in self.sizes:
            self.pix_off.append(self.pix_off[-1] + h * w)
        self.saved = torch.empty(L.fss_saved_size(params, self.cams, self.n_cams), dtype=torch.uint8,
                                 device=self.device)
        self.deferred = bool(deferred)
        self._alloc(pair_capacity)

    # -- workspace ------------------------------------------------------------
    def _alloc(self, cap: int):
        self.cap = int(cap)
        nbytes = L.fss_workspace_size(self.params, self.cams, self.n_cams, self.N, self.cap)
        self.ws = torch.zeros(max(nbytes, 256), dtype=torch.uint8, device=self.device)

    def region(self, which: int) -> torch.Tensor:
        off, size = L.fss_workspace_region(self.params, self.cams, self.n_cams, self.N, self.cap, which)
        return self.ws[off:off + size]

    def args(self):
        return self.params, self.cams, self.n_cams, self.N

    # -- pipeline steps (one C call each) -------------------------------------
    def project_bin(self, means, scales, quats, opac, stream=None):
        L.fss_project_bin(*self.args(), _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac),
                          _ptr(self.ws), self.cap, _stream(stream))

    def sort(self, stream=None):
        L.fss_sort(*self.args(), _ptr(self.ws), self.cap, _stream(stream))

    def render_forward(self, rgb, feats, out_feat=None, out_rgb=None, out_T=None, out_ids=None, stream=None):
        L.fss_render_forward(*self.args(), _ptr(self.ws), self.cap, _ptr(rgb), _ptr(feats), _ptr(out_feat),
                             _ptr(out_rgb), _ptr(out_T), _ptr(out_ids), _ptr(self.saved), _stream(stream))

    def render_forward_aux(self, rgb, feats, out_feat=None, out_rgb=None, out_T=None, out_ids=None, depth=None,
                           depth_median=None, normal=None, stream=None, label=None):
        """render_forward plus the sensor outputs (expected depth [pix], median depth [pix],
        facing normal [pix, 3]; float32 tensors or None) and the per-pixel argmax over the
        rendered channels (label [pix] int32 or None)."""
        L.fss_render_forward_aux(*self.args(), _ptr(self.ws), self.cap, _ptr(rgb), _ptr(feats), _ptr(out_feat),
                                 _ptr(out_rgb), _ptr(out_T), _ptr(out_ids), _ptr(self.saved), _ptr(depth),
                                 _ptr(depth_median), _ptr(normal), _stream(stream), label=_ptr(label))

    def render_forward_loss(self, rgb, feats, out_feat, out_rgb, out_T, out_ids, feat_target, rgb_target, w_feat,
                            w_rgb, d_feat, d_rgb, loss, stream=None):
        """render_forward and the L2-feature/L1-RGB loss with its gradients in one call
        (loss: one float64 tensor; see fss_render_forward_loss)."""
        L.fss_render_forward_loss(*self.args(), _ptr(self.ws), self.cap, _ptr(rgb), _ptr(feats), _ptr(out_feat),
                                  _ptr(out_rgb), _ptr(out_T), _ptr(out_ids), _ptr(self.saved), _ptr(feat_target),
                                  _ptr(rgb_target), w_feat, w_rgb, _ptr(d_feat), _ptr(d_rgb), _ptr(loss),
                                  _stream(stream))

    def sort_render_forward_loss(self, rgb, feats, out_feat, out_rgb, out_T, out_ids, feat_target, rgb_target,
                                 w_feat, w_rgb, d_feat, d_rgb, loss, stream=None):
        """sort + render_forward_loss in one call, after project_bin (see fss_sort_render_forward_loss)."""
        L.fss_sort_render_forward_loss(*self.args(), _ptr(self.ws), self.cap, _ptr(rgb), _ptr(feats), _ptr(out_feat),
                                       _ptr(out_rgb), _ptr(out_T), _ptr(out_ids), _ptr(self.saved),
                                       _ptr(feat_target), _ptr(rgb_target), w_feat, w_rgb, _ptr(d_feat), _ptr(d_rgb),
                                       _ptr(loss), _stream(stream))

    def render_backward(self, means, scales, quats, opac, rgb, feats, out_T, d_feat, d_rgb, d_T, g_means, g_scales,
                        g_quats, g_opac, g_rgb, g_feat, stream=None):
        L.fss_render_backward(*self.args(), _ptr(self.ws), self.cap, _ptr(means), _ptr(scales), _ptr(quats),
                              _ptr(opac), _ptr(rgb), _ptr(feats), _ptr(self.saved), _ptr(out_T), _ptr(d_feat),
                              _ptr(d_rgb), _ptr(d_T), _ptr(g_means), _ptr(g_scales), _ptr(g_quats), _ptr(g_opac),
                              _ptr(g_rgb), _ptr(g_feat), _stream(stream))

    def read_status(self, stream=None):
        return L.fss_read_status(*self.args(), _ptr(self.ws), self.cap, _stream(stream))

    # -- conveniences -----------------------------------------------------------
    def new_outputs(self):
        p = self.params
        dev = self.device
        F = torch.empty(self.total_pix, p.C, dtype=TORCH_DTYPES[p.out_dtype], device=dev)
        rgb = torch.empty(self.total_pix, 3, dtype=torch.float32, device=dev)
        T = torch.empty(self.total_pix, dtype=torch.float32, device=dev)
        ids = torch.empty(self.total_pix, max(p.K, 1), dtype=torch.int32, device=dev) if p.K else None
        return F, rgb, T, ids

    def bin_and_sort(self, means, scales, quats, opac, grow: bool = True):
        """Binning with automatic capacity growth (synchronises once)."""
        while True:
            self.project_bin(means, scales, quats, opac)
            status, need = self.read_status()
            if status == L.FSS_OK:
                break
            if status != L.FSS_ERR_CAPACITY or not grow:
                raise L.FssError(status, L.last_error())
            self._alloc(int(need * 1.25) + 1024)
        self.num_pairs = need
        self.sort()
        return need

    def forward(self, means, scales, quats, opac, rgb, feats, grow: bool = True):
        if self.deferred:  # no host synchronisation: capacity is checked later by check()
            self.project_bin(means, scales, quats, opac)
            self.sort()
        else:
            self.bin_and_sort(means, scales, quats, opac, grow)
        F, rgb_o, T, ids = self.new_outputs()
        self.render_forward(rgb, feats, F, rgb_o, T, ids)
        return F, rgb_o, T, ids

    def check(self, stream=None):
        """Waits for the frame's last calls and reads the device status
        (fss_read_status); raises FssError on capacity overflow (with the
        needed pair count as ``.needed``) or a device-side error.  Returns
        the pair count of the last binning."""
        status, n = self.read_status(stream)
        if status != L.FSS_OK:
            err = L.FssError(status, L.last_error())
            err.needed = n
            raise err
        self.num_pairs = n
        return n

    def grow(self, pairs: int):
        """A new workspace for at least ``pairs`` tile-surfel pairs (with 25 %
        margin).  Not while a step that uses the old one is in flight or
        captured in a graph."""
        self._alloc(int(pairs * 1.25) + 1024)

    def counters(self) -> torch.Tensor:
        return self.region(L.REG_COUNTERS).view(torch.int64)

    def split(self, t: torch.Tensor):
        """Per-view [H, W, ...] views of a concatenated per-pixel output."""
        return [t[a:b].view(h, w, *t.shape[1:]) for (h, w), a, b in zip(self.sizes, self.pix_off, self.pix_off[1:])]


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opac, rgb, feats, frame: Frame):
        means, scales, quats, opac, rgb, feats = (x.contiguous() for x in (means, scales, quats, opac, rgb, feats))
        F, rgb_o, T, ids = frame.forward(means, scales, quats, opac, rgb, feats)
        ctx.frame = frame
        ctx.save_for_backward(means, scales, quats, opac, rgb, feats, T)
        ctx.mark_non_differentiable(*([ids] if ids is not None else []))
        return F, rgb_o, T, ids

    @staticmethod
    def backward(ctx, dF, drgb, dT, _dids):
        frame: Frame = ctx.frame
        means, scales, quats, opac, rgb, feats, T = ctx.saved_tensors
        dev = means.device
        dF = torch.zeros_like(frame.new_outputs()[0]) if dF is None else dF.contiguous()
        drgb = torch.zeros(frame.total_pix, 3, device=dev) if drgb is None else drgb.contiguous().float()
        dT = None if dT is None else dT.contiguous().float()
        g_means, g_scales = torch.empty_like(means), torch.empty_like(scales)
        g_quats, g_opac, g_rgb = torch.empty_like(quats), torch.empty_like(opac), torch.empty_like(rgb)
        g_feat = torch.empty_like(feats)
        frame.render_backward(means, scales, quats, opac, rgb, feats, T, dF.to(feats.dtype), drgb, dT, g_means,
                              g_scales, g_quats, g_opac, g_rgb, g_feat)
        return g_means, g_scales, g_quats, g_opac, g_rgb, g_feat, None


def query_labels(f_ins, means, f_q, p_q, prec_q, out_dtype=torch.float32, err=None, stream=None):
    """Per-Gaussian instance label distributions [N, n_queries] (fss_query_labels):
    f_ins [N, dim] and f_q [n_queries, dim] BF16, means [N, 3], p_q [n_queries, 3],
    prec_q [n_queries, 6] float32 on the device.  `err` (int32 [1], zeroed) receives
    the kernel's wait-expiry flag; by default a fresh one is checked after the call."""
    N, dim = f_ins.shape
    nq = f_q.shape[0]
    out = torch.empty(N, nq, dtype=out_dtype, device=f_ins.device)
    own = err is None
    if own:
        err = torch.zeros(1, dtype=torch.int32, device=f_ins.device)
    L.fss_query_labels(N, nq, dim, _ptr(f_ins), _ptr(means), _ptr(f_q), _ptr(p_q), _ptr(prec_q), _ptr(out),
                       DTYPES[out_dtype], _ptr(err), _stream(stream))
    if own and int(err.item()) != 0:
        raise RuntimeError("query_labels: a wait on the tensor cores expired")
    return out


def render(means, scales, quats, opacities, rgb, feats, frame: Frame):
    """Differentiable render of activated surfel parameters; returns
    (features [pix, C], rgb [pix, 3], T [pix], topk ids [pix, K] or None)."""
    return _RenderFn.apply(means, scales, quats, opacities, rgb, feats, frame)


def render_raw(means, log_scales, quats, opacity_logits, rgb, feats, frame: Frame):
    """Same as :func:`render` for raw training parameters: scales =
    exp(log_scales), opacities = sigmoid(logits) (activations in torch)."""
    return render(means, torch.exp(log_scales), quats, torch.sigmoid(opacity_logits), rgb, feats, frame)

"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on
numpy inputs and read its outputs and workspace regions back."""
import numpy as np
import torch

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300.raster import Frame, make_params


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


class GpuRun:
    """One binning + render of `scene` for `cams` through the C ABI."""

    def __init__(self, scene, cams, K=4, tile_size=16, bin_mode="accu", stop_rule="tmin", feat_dtype=torch.float32,
                 out_dtype=None, cap=1 << 18, render=True, **kw):
        self.scene = scene
        self.cams = list(cams)
        self.params = make_params(C=scene.C, K=K, tile_size=tile_size, bin_mode=bin_mode, stop_rule=stop_rule,
                                  feat_dtype=feat_dtype, out_dtype=out_dtype, **kw)
        self.frame = Frame(self.cams, scene.n, self.params, pair_capacity=cap)
        self.means, self.scales = dev(scene.means), dev(scene.scales)
        self.quats, self.opac = dev(scene.quats), dev(scene.opacities)
        self.rgb = dev(scene.rgb)
        self.feats = dev(scene.feats, feat_dtype)
        self.P = self.frame.bin_and_sort(self.means, self.scales, self.quats, self.opac)
        if render:
            self.F, self.rgb_out, self.T, self.ids = self.frame.new_outputs()
            self.frame.render_forward(self.rgb, self.feats, self.F, self.rgb_out, self.T, self.ids)
            torch.cuda.synchronize()

    # per-view numpy outputs
    def view(self, v=0):
        h, w = self.frame.sizes[v]
        a, b = self.frame.pix_off[v], self.frame.pix_off[v + 1]
        out = dict(F=self.F[a:b].float().cpu().numpy().reshape(h, w, -1),
                   rgb=self.rgb_out[a:b].cpu().numpy().reshape(h, w, 3),
                   T=self.T[a:b].cpu().numpy().reshape(h, w))
        if self.ids is not None:
            out["ids"] = self.ids[a:b].cpu().numpy().reshape(h, w, -1)
        K = self.params.K
        sv = self.frame.saved
        npx = self.frame.total_pix
        a256 = lambda n: (n + 255) // 256 * 256
        nst = sv[2 * a256(npx * K * 4):].view(torch.int32)[:npx]
        out["nstop"] = nst[a:b].cpu().numpy().reshape(h, w)
        if K:
            pos = sv[:npx * K * 4].view(torch.int32).view(npx, K)
            wt = sv[a256(npx * K * 4):a256(npx * K * 4) + npx * K * 4].view(torch.float32).view(npx, K)
            out["pos"] = pos[a:b].cpu().numpy().reshape(h, w, K)
            out["w"] = wt[a:b].cpu().numpy().reshape(h, w, K)
        return out

    def rec(self):
        return self.frame.region(L.REG_REC).view(torch.float32).view(-1, 16).cpu().numpy()

    def binrec(self):
        raw = self.frame.region(L.REG_BINREC).cpu().numpy().view(np.uint8).reshape(-1, 80)
        f = raw[:, :48].copy().view(np.float32)
        i16 = raw[:, 48:64].copy().view(np.int16)
        flags = raw[:, 64:68].copy().view(np.int32)[:, 0]
        return f, i16, flags

    def count(self):
        return self.frame.region(L.REG_COUNT).view(torch.int32).cpu().numpy()

    def ranges(self):
        return self.frame.region(L.REG_RANGES).view(torch.int32).view(-1, 2).cpu().numpy()

    def lists(self):
        return self.frame.region(L.REG_LIST).view(torch.int32)[:self.P].cpu().numpy()

    def masks(self):
        return self.frame.region(L.REG_MASK).view(torch.int32)[:self.P].cpu().numpy().view(np.uint32)

    def counters(self):
        return self.frame.counters().cpu().numpy()


def tol_scale(oracle_mod, scene, cam, params, binned):
    """S(x, ch) = sum over the accumulated set of w_i |c_i,ch| + 1e-6."""
    abs_out = oracle_mod.render(scene, cam, params, feats=np.abs(scene.feats.astype(np.float64)), binned=binned)
    return abs_out["F"] + 1e-6

"""Autotuner for the batched multi-view rasterizer.

For one workload (cameras, surfel count, channels, K, feature dtype) it
times every candidate of
  tile size     8, 16, 32 pixels;
  CTA schedule  one CTA per tile, or one persistent wave pulling tiles from
                a device work queue (evens out views of mixed size);
  Top-K stop    TMIN, or EXACT_TOPK when only the features are needed (the
                features are the same; RGB and T then cover the traversed
                prefix only)
on the real inputs and keeps the fastest.  K itself is the caller's choice
and never changed.  Tile size and stop rule do not change the rendered
features, so any choice is safe; results are cached per workload key.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Optional, Sequence

import torch

from .raster import Frame, make_params


def workload_key(cams: Sequence, N: int, C: int, K: int, feat_dtype, backward: bool) -> str:
    sizes = ",".join(f"{c.width}x{c.height}" for c in cams)
    return f"N{N}-C{C}-K{K}-{str(feat_dtype).split('.')[-1]}-{'fb' if backward else 'f'}-{sizes}"


class Autotuner:
    def __init__(self, cache_path: Optional[str] = None):
        self.cache_path = cache_path
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def _save(self):
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def candidates(self, allow_exact_stop: bool):
        stops = ["tmin", "exact_topk"] if allow_exact_stop else ["tmin"]
        return [dict(tile_size=ts, schedule=sc, stop_rule=st)
                for ts, sc, st in itertools.product((8, 16, 32), ("grid", "persistent"), stops)]

    def tune(self, cams: Sequence, means, scales, quats, opac, rgb, feats, K: int, backward: bool = True,
             allow_exact_stop: bool = True, reps: int = 5, force: bool = False, **param_kw):
        """Times each candidate on these inputs; returns the best as a dict
        (tile_size, schedule, stop_rule, ms) and caches it."""
        N, C = int(means.shape[0]), int(feats.shape[1])
        key = workload_key(cams, N, C, K, feats.dtype, backward)
        if not force and key in self.cache:
            return self.cache[key]
        results = []
        for cand in self.candidates(allow_exact_stop):
            params = make_params(C=C, K=K, feat_dtype=feats.dtype, **cand, **param_kw)
            fr = Frame(cams, N, params, pair_capacity=1 << 20, device=means.device)
            fr.bin_and_sort(means, scales, quats, opac)
            F, rgb_o, T, ids = fr.new_outputs()
            dF = torch.randn_like(F) if backward else None
            drgb = torch.randn_like(rgb_o) if backward else None
            grads = [torch.empty_like(x) for x in (means, scales, quats, opac, rgb, feats)] if backward else None

            def step():
                fr.project_bin(means, scales, quats, opac)
                fr.sort()
                fr.render_forward(rgb, feats, F, rgb_o, T, ids)
                if backward:
                    fr.render_backward(means, scales, quats, opac, rgb, feats, T, dF, drgb, None, *grads)

            step()
            torch.cuda.synchronize()
            times = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                step()
                b.record()
                b.synchronize()
                times.append(a.elapsed_time(b))
            status, _ = fr.read_status()
            if status != 0:
                continue
            times.sort()
            results.append((times[len(times) // 2], cand))
            del fr
        ms, best = min(results, key=lambda r: r[0])
        out = dict(best, ms=ms, all=[dict(c, ms=m) for m, c in results])
        self.cache[key] = out
        self._save()
        return out

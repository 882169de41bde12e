"""Precision of the GPU path against the FP64 oracle, per output and per
gradient, for FP32 and BF16 feature storage (test infrastructure: it runs
the oracle).

Workloads (seeded synthetic stand-ins for the paper's rooms):
  room   500k surfels, C = 64, one 640x480 view (f = 525), the
         forward+backward workload;
  large  1.5M surfels, C = 128, one 1280x720 view (f = 900).
Both with Top-K K = 8 (Eq. 7), AccuTile binning, exact stop, 16x16 tiles.

Per workload and storage type: the error of the rendered features F (against
the tolerance scale S = sum w |c| + 1e-6, and absolute), of the colour and of
the transmittance T; the Top-K id agreement (before and after resolving the
borderline pixels, see tests/outcomes.py); and per gradient (means, scales,
quaternions, opacity, colour, features; upstream gradients N(0, 1), BF16
rounded for BF16 storage) the largest and mean error relative to the
gradient's largest entry and the 99th percentile of the element-wise
relative error over entries above 1e-3 of the largest.  ``band_rows``
restricts the comparison (and the upstream gradients) to one band of tile
rows, which keeps the oracle's share short.

  python -m tests.precision_report [--band ROWS] [--workloads room,large]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "room": dict(n=500_000, C=64, seed=3, poses=(16, 640, 480, 525.0), pose=0),
    "large": dict(n=1_500_000, C=128, seed=2, poses=(32, 1280, 720, 900.0), pose=7),
}
GRADS = ("means", "scales", "quats", "opac", "rgb", "feat")


def _grad_err(g, r):
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    scale = float(np.abs(r).max())
    d = np.abs(g - r)
    big = np.abs(r) > 1e-3 * scale
    el = d[big] / np.abs(r[big]) if big.any() else np.zeros(1)
    return {"max_rel_to_max": float(d.max() / scale) if scale > 0 else 0.0,
            "mean_rel_to_max": float(d.mean() / scale) if scale > 0 else 0.0,
            "p99_rel": float(np.percentile(el, 99)), "entries": int(d.size)}


def report(names=("room", "large"), dtypes=("f32", "bf16"), band_rows=None, band=0, K=8, seed=0, log=None):
    import torch

    import oracle as O
    from paper_2604_10951_gb300 import scenes
    from paper_2604_10951_gb300.raster import Frame, make_params
    from tests.outcomes import oracle_ref, settle, upstream_mask

    O.build()
    out = {}
    for name in names:
        w = WORKLOADS[name]
        t0 = time.perf_counter()
        sc = scenes.room_scene(n=w["n"], C=w["C"], seed=w["seed"])
        cam = scenes.circle_poses(*w["poses"])[w["pose"]]
        H, W, C = cam.height, cam.width, sc.C
        p = O.make_params(K=K, stop_rule=O.EXACT_TOPK)
        b = O.binning(sc, cam, p)
        if band_rows:
            r0, r1 = band * band_rows, min(H, (band + 1) * band_rows)
            tx = (W + 15) // 16
            bcam = dataclasses.replace(cam, height=r1 - r0, cy=np.float32(cam.cy - r0))
            bb = dict(b, ranges=b["ranges"][(r0 // 16) * tx:((r1 + 15) // 16) * tx])
        else:
            r0, r1, bcam, bb = 0, H, cam, b
        dev = torch.device("cuda")
        t32 = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
        means, scales, quats, opac, rgb = (t32(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb))
        rng = np.random.default_rng(seed)
        gF_full = rng.normal(size=(H, W, C))
        grgb_full = rng.normal(size=(H, W, 3))
        for dt in dtypes:
            tdt = torch.bfloat16 if dt == "bf16" else torch.float32
            feats = t32(sc.feats).to(tdt)
            f64 = feats.double().cpu().numpy()
            fr = Frame([cam], sc.n, make_params(C=C, K=K, stop_rule="exact_topk", feat_dtype=tdt), device=dev)
            fr.bin_and_sort(means, scales, quats, opac)
            F, rgb_o, T, ids = fr.new_outputs()
            fr.render_forward(rgb, feats, F, rgb_o, T, ids)
            torch.cuda.synchronize()
            rows = slice(r0 * W, r1 * W)
            g = dict(F=F[rows].float().cpu().numpy().reshape(r1 - r0, W, C),
                     rgb=rgb_o[rows].cpu().numpy().reshape(r1 - r0, W, 3),
                     T=T[rows].cpu().numpy().reshape(r1 - r0, W),
                     ids=ids[rows].cpu().numpy().reshape(r1 - r0, W, K))
            tol = 2e-2 if dt == "bf16" else 1e-4
            ref, S = oracle_ref(sc, bcam, p, binned=bb, feats=f64)
            ids_plain = float((g["ids"] == ref["ids"]).all(-1).mean())
            ok = settle(g, ref, S, tol, K)
            eF = np.abs(g["F"] - ref["F"])[ok]
            eS = (np.abs(g["F"] - ref["F"]) / S)[ok]
            e_rgb = np.abs(g["rgb"] - ref["rgb"])[ok]
            e_T = np.abs(g["T"] - ref["T"])[ok]
            row = {"F_rel_S_max": float(eS.max()), "F_rel_S_mean": float(eS.mean()),
                   "F_abs_max": float(eF.max()), "F_abs_mean": float(eF.mean()),
                   "rgb_abs_max": float(e_rgb.max()), "rgb_abs_mean": float(e_rgb.mean()),
                   "T_abs_max": float(e_T.max()), "T_abs_mean": float(e_T.mean()),
                   "ids_agree_plain": ids_plain, "ids_agree_resolved": float((g["ids"] == ref["ids"]).all(-1)[ok].mean()),
                   "pixels": int(ok.size), "outcomes": ref["outcomes"]}
            # gradients of sum(gF . F) + sum(grgb . rgb) over the band
            gF = gF_full.copy()
            grgb = grgb_full.copy()
            keep = np.zeros((H, W), bool)
            keep[r0:r1] = ~upstream_mask(ref)
            gF[~keep] = 0.0
            grgb[~keep] = 0.0
            if dt == "bf16":
                gF = torch.as_tensor(gF).bfloat16().double().numpy()
            gr = O.render_backward(sc, bcam, p, gF[r0:r1], grgb[r0:r1], None, feats=f64, binned=bb, flip=ref["flip"])
            outs = [torch.empty(sc.n, k, device=dev) for k in (3, 2, 4)] + \
                   [torch.empty(sc.n, device=dev), torch.empty(sc.n, 3, device=dev),
                    torch.empty(sc.n, C, device=dev, dtype=tdt)]
            fr.render_backward(means, scales, quats, opac, rgb, feats, T,
                               t32(gF.reshape(-1, C)).to(tdt), t32(grgb.reshape(-1, 3)).float(), None, *outs)
            torch.cuda.synchronize()
            row["grad"] = {k: _grad_err(o.float().cpu().numpy(), gr[k]) for k, o in zip(GRADS, outs)}
            out[f"{name}_{dt}"] = row
            del fr, F, rgb_o, T, ids, outs
            torch.cuda.empty_cache()
        out[f"{name}_seconds"] = round(time.perf_counter() - t0, 1)
        if log:
            log(f"{name}: {out[f'{name}_seconds']} s")
    out["band_rows"] = band_rows
    return out


def markdown(rep):
    lines = ["| workload | storage | F err / S max (mean) | F abs max | rgb abs max | T abs max | ids agree (plain / resolved) |",
             "|---|---|---|---|---|---|---|"]
    for k, r in rep.items():
        if not isinstance(r, dict) or "grad" not in r:
            continue
        name, dt = k.rsplit("_", 1)
        lines.append(f"| {name} | {dt} | {r['F_rel_S_max']:.2e} ({r['F_rel_S_mean']:.1e}) | {r['F_abs_max']:.1e} | "
                     f"{r['rgb_abs_max']:.1e} | {r['T_abs_max']:.1e} | {r['ids_agree_plain']:.5f} / "
                     f"{r['ids_agree_resolved']:.5f} |")
    lines += ["", "| workload | storage | " + " | ".join(GRADS) + " |", "|---|---|" + "---|" * len(GRADS)]
    for k, r in rep.items():
        if not isinstance(r, dict) or "grad" not in r:
            continue
        name, dt = k.rsplit("_", 1)
        cells = [f"{r['grad'][g]['max_rel_to_max']:.1e} / {r['grad'][g]['p99_rel']:.1e}" for g in GRADS]
        lines.append(f"| {name} | {dt} | " + " | ".join(cells) + " |")
    return "\n".join(lines)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--band", type=int, default=0, help="rows of the compared band (0: whole frames)")
    ap.add_argument("--workloads", default="room,large")
    a = ap.parse_args()
    rep = report(tuple(a.workloads.split(",")), band_rows=a.band or None, log=lambda m: print(m, file=sys.stderr))
    print(json.dumps(rep))
    print(markdown(rep), file=sys.stderr)

#!/usr/bin/env python
"""Benchmark of the 2DGS Top-K feature rasterizer on the GB300.

Workload (one step = the whole hot path for one 640x480 frame): room scene
stand-in with 500k surfels and 64-channel BF16 features (K = 8), camera
cycling over the 16 poses of the circular trajectory; per step:
project + Precise Tile Intersection binning, per-tile depth sort, Top-K
forward render, fused L2-feature/L1-RGB loss and gradient, backward render
(geometric and feature gradients).  Metric: frames/s of forward+backward.

Also reported: the plain FP32 full-accumulation path on the same frames,
per-call times, the roofline of the dominant kernel, an end-to-end number
through the C ABI with host buffers, and the FP64 checker on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s & fwd+bwd ms at 640x480 C=64 K=8; % HBM roofline vs plain FP32 path"
N_SPLATS, C_FEAT, K_TOP, SEED = 500_000, 64, 8, 3
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=256)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip baseline/e2e/cpu legs (profiling runs)")
    ap.add_argument("--queries-only", action="store_true",
                    help="only the query-guided instance-label measurement (profiling runs)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing: one process per GPU, views sharded, no collective on
# the data path (weak scaling); a barrier and a max-reduce of the time only
# ---------------------------------------------------------------------------
def shard_pose(step, rank, world, n_poses):
    """Pose of a rank's step: the ranks take interleaved poses of the camera
    stream (rank r renders poses r, r + world, ...), so together they render
    different views and every pose equally often."""
    return (step * world + rank) % n_poses


class Dist:
    def __init__(self, backend):
        import torch
        import torch.distributed as dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = dist if self.world > 1 else None
        if self.dist:
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend)
        self.torch = torch

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, v: float) -> float:
        if not self.dist:
            return v
        t = self.torch.tensor([v], dtype=self.torch.float64,
                              device="cuda" if self.dist.get_backend() == "nccl" else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.lines = gpu, None, []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_bf16_tflops():
    """Burst cuBLAS bf16 TFLOP/s (a kernel timed alone), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    D = Dist("nccl")
    torch.cuda.set_device(D.local)
    from paper_2604_10951_gb300 import _lib as L
    from paper_2604_10951_gb300 import scenes
    from paper_2604_10951_gb300.build import build
    from paper_2604_10951_gb300.raster import Frame, make_cams, make_params

    build()
    dev = torch.device("cuda", D.local)
    sc = scenes.room_scene(n=N_SPLATS, C=C_FEAT, seed=SEED)
    poses = scenes.circle_poses(16)
    cams_c = [make_cams([c]) for c in poses]
    H, W = poses[0].height, poses[0].width
    npx = H * W
    t32 = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
    means, scales, quats, opac, rgb = (t32(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb))
    feats = {torch.bfloat16: t32(sc.feats).bfloat16(), torch.float32: t32(sc.feats)}
    F_tgt_np, rgb_tgt_np = scenes.targets(4, npx, C_FEAT)
    rgb_tgt = t32(rgb_tgt_np)
    F_tgt = {torch.bfloat16: t32(F_tgt_np).bfloat16(), torch.float32: t32(F_tgt_np)}
    stream = torch.cuda.current_stream()
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    if args.queries_only:
        if D.rank == 0:
            print(json.dumps({"query_labels": queries(torch, dev, sc, means, scales, quats, opac, rgb, poses, flush)}))
        D.close()
        return

    names = ["project_bin", "sort", "render_forward", "loss", "render_backward"]

    def make_events():
        try:  # events that become graph nodes, so per-call times survive graph replay
            return [torch.cuda.Event(enable_timing=True, external=True) for _ in range(6)]
        except TypeError:
            return None

    class Path:
        """Buffers and the step of one configuration (all calls via the C ABI),
        replayed as one CUDA graph per camera pose."""

        def __init__(self, K, dtype, stop):
            self.dtype = dtype
            self.params = make_params(C=C_FEAT, K=K, tile_size=16, bin_mode="accu", stop_rule=stop,
                                      feat_dtype=dtype, out_dtype=dtype)
            self.frame = Frame([poses[0]], N_SPLATS, self.params, pair_capacity=1 << 20, device=dev)
            cap = 0
            for c in cams_c:  # size the pair capacity from the 16 poses, with margin
                self.frame.cams = c
                cap = max(cap, self.frame.bin_and_sort(means, scales, quats, opac))
            self.frame._alloc(int(cap * 1.3) + 4096)
            self.max_pairs = cap
            self.F, self.rgb_o, self.T, self.ids = self.frame.new_outputs()
            self.dF = torch.empty_like(self.F)
            self.drgb = torch.empty_like(self.rgb_o)
            self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
            self.g = [torch.empty(N_SPLATS, k, device=dev) for k in (3, 2, 4)] + \
                     [torch.empty(N_SPLATS, device=dev), torch.empty(N_SPLATS, 3, device=dev)]
            self.gfeat = torch.empty(N_SPLATS, C_FEAT, dtype=dtype, device=dev)
            self.feats = feats[dtype]
            self.F_tgt = F_tgt[dtype]
            self.rgb_tgt = rgb_tgt
            self.graphs, self.gevents = [], []

        def step(self, i, events=None):
            fr, p, ws = self.frame, self.params, ptr(self.frame.ws)
            sp = C.c_void_p(torch.cuda.current_stream().cuda_stream)
            cams = cams_c[shard_pose(i, D.rank, D.world, len(cams_c))]
            a = (p, cams, 1, N_SPLATS)
            rec = (lambda k: events[k].record()) if events else (lambda k: None)
            rec(0)
            L.fss_project_bin(*a, ptr(means), ptr(scales), ptr(quats), ptr(opac), ws, fr.cap, sp)
            rec(1)
            L.fss_sort(*a, ws, fr.cap, sp)
            rec(2)
            L.fss_render_forward(*a, ws, fr.cap, ptr(rgb), ptr(self.feats), ptr(self.F), ptr(self.rgb_o),
                                 ptr(self.T), ptr(self.ids), ptr(fr.saved), sp)
            rec(3)
            L.fss_loss_l2_l1(p, npx, ptr(self.F), ptr(self.rgb_o), ptr(self.F_tgt), ptr(self.rgb_tgt), 1.0, 1.0,
                             ptr(self.dF), ptr(self.drgb), ptr(self.loss), sp)
            rec(4)
            L.fss_render_backward(*a, ws, fr.cap, ptr(means), ptr(scales), ptr(quats), ptr(opac), ptr(rgb),
                                  ptr(self.feats), ptr(fr.saved), ptr(self.T), ptr(self.dF), ptr(self.drgb), None,
                                  *(ptr(g) for g in self.g), ptr(self.gfeat), sp)
            rec(5)

        def capture(self):
            """One graph per pose: the whole step, 11 kernels and 4 memsets."""
            for i in range(len(cams_c)):
                self.step(i)  # sets kernel attributes outside capture
            torch.cuda.synchronize()
            for i in range(len(cams_c)):
                g = torch.cuda.CUDAGraph()
                ev = make_events()
                with torch.cuda.graph(g):
                    self.step(i, ev)
                self.graphs.append(g)
                self.gevents.append(ev)
            torch.cuda.synchronize()

        def check(self):
            for c in cams_c:
                self.frame.cams = c
                s, n = self.frame.read_status()
                if s != L.FSS_OK:
                    raise RuntimeError(f"device status {s}: {L.last_error()}")

        def time_steps(self, steps, warmup):
            if not self.graphs:
                self.capture()
            for i in range(warmup):
                self.graphs[i % len(self.graphs)].replay()
            torch.cuda.synchronize()
            D.barrier()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(steps):
                flush.zero_()  # L2 flush between timed steps (outside the events)
                ev[i][0].record()
                self.graphs[i % len(self.graphs)].replay()
                ev[i][1].record()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            step_ms = [a.elapsed_time(b) for a, b in ev]
            calls = {}
            if self.gevents[0] is not None:  # last replay of each pose's graph
                used = self.gevents[:min(steps, len(self.gevents))]
                for k, n in enumerate(names):
                    calls[n] = float(np.mean([e[k].elapsed_time(e[k + 1]) for e in used]))
            self.check()
            return step_ms, calls, wall

    ours = Path(K_TOP, torch.bfloat16, "exact_topk")
    with ClockSampler(D.local) as clk:
        step_ms, calls, wall = ours.time_steps(args.steps, args.warmup)
    total_ms = D.max(float(np.sum(step_ms)))
    ms_step = total_ms / args.steps
    frames = args.steps * D.world
    value = frames / (total_ms / 1e3)
    # kernels per step: project_bin 3 (project, scan, emit), sort 1, forward 1, loss 1,
    # backward 5 (clear, feature grads + dots, geometry replay, projection, feature rows)
    launches_per_step = 3 + 1 + 1 + 1 + 5

    out = {"metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": D.world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
           "data": "synthetic (seeded room stand-in for the paper's ScanNet scenes)",
           "config": {"workload": "room 500k surfels, 640x480 (fx=fy=525), C=64 BF16 features, K=8 Top-K "
                                  "(exact early stop), 16x16 tiles, AccuTile binning, forward+backward incl. "
                                  "L2-feature/L1-RGB loss; one frame per step over 16 poses, each step one "
                                  "CUDA-graph replay",
                      "global_batch": D.world, "seq_len": npx, "parallelism": f"views sharded x{D.world}",
                      "l2": "flushed between timed steps (512 MB write)"},
           "gpu_launches": launches_per_step * args.steps,
           "step_ms": {q: round(float(np.percentile(step_ms, v)), 4) for q, v in (("p10", 10), ("p50", 50), ("p90", 90))},
           "calls_ms": {k: round(v, 4) for k, v in calls.items()},
           "pairs_per_frame_max": ours.max_pairs}
    clocks = clk.summary()
    if clocks:
        out["clocks"] = clocks
    if not args.no_extras:
        # the plain FP32 full-accumulation path on the same frames
        base = Path(0, torch.float32, "tmin")
        b_ms, b_calls, _ = base.time_steps(max(8, args.steps // 4), 3)
        b_ms_step = D.max(float(np.sum(b_ms))) / len(b_ms)
        out["fp32_full_path"] = {"ms_per_step": round(b_ms_step, 4), "frames_per_s": round(1e3 / b_ms_step, 2),
                                 "calls_ms": {k: round(v, 4) for k, v in b_calls.items()},
                                 "speedup_of_bf16_topk": round(b_ms_step / ms_step, 3)}
        if calls:
            fwd_ms = calls["project_bin"] + calls["sort"] + calls["render_forward"]
            out["forward_only"] = {"ms": round(fwd_ms, 4), "frames_per_s": round(1e3 / fwd_ms, 2)}
            out["roofline"], out["roofline_kernels"], out["kernel_us"], out["roofline_frame"] = \
                roofline(ours, torch, L, flush)
        out["e2e"] = e2e(ours, torch, dev, ptr, L, args)
        del base
        out["ablation_fwd"] = ablation(torch, L, dev, means, scales, quats, opac, rgb, feats[torch.float32], poses,
                                       flush)
        out["variants_render_ms"] = variants(torch, dev, means, scales, quats, opac, rgb, feats[torch.bfloat16],
                                             poses, flush)
        out["query_labels"] = queries(torch, dev, sc, means, scales, quats, opac, rgb, poses, flush)
    if D.rank == 0 and not args.no_extras:
        out["cpu_baseline"] = cpu_baseline(sc, poses)
    if D.rank == 0:
        print(json.dumps(out))
    D.close()


KERNELS = ["k_project", "k_scan", "k_emit", "k_tile_sort", "k_render_topk", "k_loss", "k_bwd_clear", "k_bwd_feat",
           "k_bwd_geo", "k_bwd_project", "k_feat_out"]
# dram__bytes_read.sum + dram__bytes_write.sum of one launch (camera pose 1) from the
# ncu capture summarised in profiles/<kernel>_room500k_640x480_c64_k8.md; to be set
# to None whenever the kernel changes after that capture
NCU_TRAFFIC = {"k_render_topk": 27040768, "k_bwd_feat": 70487808, "k_bwd_geo": 38011904}
# (smsp__inst_executed.sum, gpu__time_duration.sum in us) of the same captures
NCU_ISSUE = {"k_render_topk": (85133445, 98.88), "k_bwd_feat": (67462191, 85.376), "k_bwd_geo": (88911244, 106.4)}
# the query-label kernel's capture (profiles/k_query_labels_room500k_nq32_dim32.md): DRAM read + write
NCU_QUERY_TRAFFIC = {"nq32_dim32_f32": 47276544}


def kernel_times(path, torch, L, flush, rounds=4):
    """Per-kernel durations (ms) over the 16 poses, from events that the library
    records after each of its launches (fss_set_kernel_events), captured into
    one graph per pose; L2 flushed before every replay."""
    graphs, evs = [], []
    for i in range(16):
        # the first event is recorded by torch inside the capture (an external event
        # becomes a graph node); the others by the library after each launch
        ev = [torch.cuda.Event(enable_timing=True, external=True)] + \
             [torch.cuda.Event(enable_timing=True) for _ in range(len(KERNELS))]
        for e in ev:  # creates the CUDA events
            e.record()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ev[0].record()
            L.fss_set_kernel_events(ev[1:])
            path.step(i)
            L.fss_set_kernel_events([])
        graphs.append(g)
        evs.append(ev)
    sums = np.zeros(len(KERNELS))
    n = 0
    nbytes, sizes = {}, {}
    for r in range(rounds):
        for i, (g, ev) in enumerate(zip(graphs, evs)):
            flush.zero_()
            g.replay()
            torch.cuda.synchronize()
            sums += [ev[k].elapsed_time(ev[k + 1]) for k in range(len(KERNELS))]
            n += 1
            if r == 0:  # the pose's algorithmic bytes, averaged over the 16 poses
                b, z = algorithmic_bytes(path, torch, L)
                b.update(z.pop("rest"))
                for k in b:
                    nbytes[k] = nbytes.get(k, 0.0) + b[k] / len(graphs)
                for k in z:
                    sizes[k] = sizes.get(k, 0.0) + z[k] / len(graphs)
    return dict(zip(KERNELS, (sums / n).tolist())), nbytes, {k: int(round(v)) for k, v in sizes.items()}


def algorithmic_bytes(path, torch, L):
    """Unique bytes each of the three render kernels must move per launch for
    the frame last rendered by `path`: reads of their inputs and writes of
    their outputs once, nothing re-read."""
    fr = path.frame
    ranges = fr.region(L.REG_RANGES).view(torch.int32).view(-1, 2).cpu().numpy()
    P = int((ranges[:, 1] - ranges[:, 0]).sum())
    tiles = ranges.shape[0]
    st = fr.region(L.REG_STATUS).view(torch.int32)[:28].cpu().numpy()
    cnt = fr.region(L.REG_STATUS).view(torch.int64)[2:10].cpu().numpy()
    nslot = int(st[22])
    nvis = int(st[20]) + int(st[25])  # bounded visible items (narrow + wide)
    n_eval, n_contrib = int(cnt[0]), int(cnt[1])
    H, W, ts = fr.sizes[0][0], fr.sizes[0][1], 16
    ids = path.ids.cpu().numpy().reshape(H, W, -1)
    U = 0
    for ty in range(0, H, ts):
        for tx in range(0, W, ts):
            blk = ids[ty:ty + ts, tx:tx + ts].reshape(-1)
            U += np.unique(blk[blk >= 0]).size
    s, K, Cc, npx = 2, K_TOP, C_FEAT, H * W
    N = N_SPLATS
    # the other kernels of the step, for the per-frame total
    rest = {
        "k_project": N * 16 + nvis * (24 + 64 + 80 + 8),  # centres and opacities of all, the rest of the visible
        "k_scan": tiles * 12,
        "k_emit": nvis * (80 + 64 + 4) + P * 4,
        "k_tile_sort": P * (4 + 4 + 64 + 4 + 4),
        "k_loss": npx * (2 * Cc * s + 24) + npx * (Cc * s + 12),
        "k_bwd_clear": nslot * (64 + 4 * Cc),
        "k_bwd_project": N * 52 + nslot * (64 + 48 + 40),
        "k_feat_out": N * Cc * s + nslot * 4 * Cc,
    }
    # FP32 operations of the forward: ~20 per evaluation (ray-splat solve,
    # density, opacity, depth test) + ~10 per contribution (compositing, K-set
    # test) + 2 C per selected row (feature accumulation); two MUFU ops per evaluation
    flops_fwd = 20 * n_eval + 10 * n_contrib + 2 * Cc * min(K, 8) * npx
    return {
        # ranges; per pair: list id, warp mask, adjugate rows, opacity, colour;
        # selected rows once per tile; per pixel: features, rgb, T, ids, saved pos/w, nstop
        "k_render_topk": tiles * 8 + P * (4 + 4 + 48 + 4 + 12) + U * Cc * s
        + npx * (Cc * s + 12 + 4 + 4 * K * 3 + 4),
        # per pixel: saved pos/w, dL/dF, dots written; selected rows (+ list id, slot) once
        # per tile; the FP32 feature-gradient accumulators written once
        "k_bwd_feat": tiles * 8 + npx * (8 * K + Cc * s + 4 * K) + U * (Cc * s + 8) + nslot * Cc * 4,
        # per pixel: nstop, T, dL/drgb, saved pos, dots; per pair: list id, mask, record
        # rows, colour; the per-(view, slot) gradient rows written once
        "k_bwd_geo": tiles * 8 + npx * (4 + 4 + 12 + 8 * K) + P * (4 + 4 + 64 + 12) + nslot * 64,
    }, {"pairs": P, "unique_rows": U, "slots": nslot, "evaluations": n_eval, "contributions": n_contrib,
        "flops_fwd": flops_fwd, "rest": rest}


def roofline(path, torch, L, flush):
    """Roofline of the dominant kernel (largest average duration): algorithmic
    bytes per launch / its event-timed duration (both averaged over the 16
    poses), against the measured HBM copy bandwidth; the other render kernels
    alongside."""
    peak, src = measured_peaks()
    kt, nbytes, sizes = kernel_times(path, torch, L, flush)
    rows = {}
    for k, b in nbytes.items():
        if k not in ("k_render_topk", "k_bwd_feat", "k_bwd_geo"):
            continue
        ach = b / (kt[k] * 1e-3) / 1e9
        rows[k] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                   "traffic": NCU_TRAFFIC.get(k), "algorithmic_bytes": int(b), "ms": round(kt[k], 5)}
    # the forward's arithmetic against the FP32 peak: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
    fp32_peak = 152 * 128 * 2 * 2.07e9
    rows["k_render_topk"]["alu"] = {"flops": int(sizes["flops_fwd"]),
                                    "achieved_tflops": round(sizes["flops_fwd"] / (kt["k_render_topk"] * 1e-3) / 1e12, 2),
                                    "peak_tflops": round(fp32_peak / 1e12, 1),
                                    "frac": round(sizes["flops_fwd"] / (kt["k_render_topk"] * 1e-3) / fp32_peak, 4)}
    # warp-instruction issue of the ncu captures against 152 SMs x 4 schedulers x 2.07 GHz
    for k, v in NCU_ISSUE.items():
        if k in rows and v is not None:
            rows[k]["issue_frac_ncu"] = round(v[0] / (v[1] * 1e-6) / (152 * 4 * 2.07e9), 3)
    dom = max(kt, key=kt.get)
    main = dict(rows.get(dom, {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                               "traffic": None}), kernel=dom, peak_source=f"{src} (MEASURED_PEAKS.json hbm_gbs)")
    main.update({k: v for k, v in sizes.items() if k != "flops_fwd"})
    # per frame: all kernels' algorithmic bytes over the summed kernel times
    tot_b = sum(nbytes.get(k, 0.0) for k in KERNELS)
    tot_t = sum(kt.values()) * 1e-3
    frame = {"algorithmic_bytes": int(tot_b), "kernel_ms": round(tot_t * 1e3, 4),
             "achieved": round(tot_b / tot_t / 1e9, 1), "peak": peak, "unit": "GB/s",
             "frac": round(tot_b / tot_t / 1e9 / peak, 4)}
    return main, rows, {k: round(v * 1e3, 2) for k, v in kt.items()}, frame


def ablation(torch, L, dev, means, scales, quats, opac, rgb, feats, poses, flush, reps=3):
    """Forward-only ablation in the layout of the paper's Table 2 on the same
    frames, FP32 features: (A) square box + full accumulation, (B) AccuTile +
    full, (C) square box + Top-K (K=8), (D) AccuTile + Top-K.  Per row: mean
    over the 16 poses of the binning + sort + render time (CUDA events, L2
    flushed before each frame), tile-surfel pairs per frame (the paper's
    RN-Total) and pairs per tile."""
    from paper_2604_10951_gb300.raster import Frame, make_cams, make_params

    rows = {}
    for name, mode, K in (("A", "aabb", 0), ("B", "accu", 0), ("C", "aabb", K_TOP), ("D", "accu", K_TOP)):
        p = make_params(C=C_FEAT, K=K, tile_size=16, bin_mode=mode, stop_rule="exact_topk" if K else "tmin")
        fr = Frame([poses[0]], N_SPLATS, p, pair_capacity=1 << 21, device=dev)
        F, rgb_o, T, ids = fr.new_outputs()
        ms, pairs = [], []
        for cam in poses:
            fr.cams = make_cams([cam])
            fr.bin_and_sort(means, scales, quats, opac)
            pairs.append(fr.num_pairs)
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fr.project_bin(means, scales, quats, opac)
                fr.sort()
                fr.render_forward(rgb, feats, F, rgb_o, T, ids)
                b.record()
                b.synchronize()
                ms.append(a.elapsed_time(b))
        s, n = fr.read_status()
        tiles = fr.region(L.REG_RANGES).shape[0] // 8
        rows[name] = {"bin_mode": mode, "K": K, "fwd_ms": round(float(np.mean(ms)), 4),
                      "fps": round(1e3 / float(np.mean(ms)), 1), "pairs_per_frame": int(np.mean(pairs)),
                      "pairs_per_tile": round(float(np.mean(pairs)) / tiles, 1), "status": int(s)}
        del fr
    return rows


def variants(torch, dev, means, scales, quats, opac, rgb, feats, poses, flush, reps=3):
    """Render-call time (mean over the 16 poses, L2 flushed, CUDA events) of
    the bench's forward configuration and of its variants on the same binned
    frames: the sensor outputs (expected and median depth, normal), the
    first-K selection and the renormalised Top-K."""
    from paper_2604_10951_gb300.raster import Frame, make_cams, make_params

    rows = {}
    for name, sel, rn, aux in (("topw", "topw", False, False), ("topw_sensors", "topw", False, True),
                               ("front", "front", False, False), ("renorm", "topw", True, False)):
        p = make_params(C=C_FEAT, K=K_TOP, feat_dtype=torch.bfloat16, stop_rule="exact_topk", select=sel, renorm=rn)
        fr = Frame([poses[0]], N_SPLATS, p, pair_capacity=1 << 21, device=dev)
        F, rgb_o, T, ids = fr.new_outputs()
        depth = torch.empty(fr.total_pix, device=dev) if aux else None
        med = torch.empty(fr.total_pix, device=dev) if aux else None
        nrm = torch.empty(fr.total_pix, 3, device=dev) if aux else None
        ms = []
        for cam in poses:
            fr.cams = make_cams([cam])
            fr.bin_and_sort(means, scales, quats, opac)
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fr.render_forward_aux(rgb, feats, F, rgb_o, T, ids, depth, med, nrm)
                b.record()
                b.synchronize()
                ms.append(a.elapsed_time(b))
        rows[name] = round(float(np.mean(ms)), 4)
        del fr
    return rows


def queries(torch, dev, sc, means, scales, quats, opac, rgb, poses, flush, reps=20):
    """Query-guided instance labels (Sec. 3.3) on the bench's 500k Gaussians:
    the tensor-core label kernel (32 queries and 32-d instance features as in
    the paper, plus 128 queries) timed alone with CUDA events, L2 flushed
    before each launch, against the HBM roofline of its algorithmic bytes
    (instance features, centres, labels out) and the bf16 tensor peak of its
    2 N nq dim flops; and the instance-mask render (the labels blended by the
    K = 8 Top-K renderer with the per-pixel argmax output, C = 32 BF16) over
    the 16 poses."""
    from paper_2604_10951_gb300 import scenes
    from paper_2604_10951_gb300.raster import Frame, make_cams, make_params, query_labels

    peak, src = measured_peaks()
    tpeak, tsrc = measured_bf16_tflops()
    N = sc.n
    rows = {}
    for nq, dim, od in ((32, 32, torch.float32), (32, 32, torch.bfloat16), (128, 32, torch.bfloat16)):
        f_ins, f_q, p_q, prec = scenes.room_queries(sc.means, nq, dim, seed=0)
        fi = torch.as_tensor(f_ins).to(dev, torch.bfloat16)
        fq = torch.as_tensor(f_q).to(dev, torch.bfloat16)
        pq, pr = torch.as_tensor(p_q).to(dev), torch.as_tensor(prec).to(dev)
        err = torch.zeros(1, dtype=torch.int32, device=dev)
        lab = query_labels(fi, means, fq, pq, pr, out_dtype=od, err=err)
        ms = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            lab = query_labels(fi, means, fq, pq, pr, out_dtype=od, err=err)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        if int(err.item()):
            raise RuntimeError("query_labels: a tensor-core wait expired")
        t = float(np.median(ms)) * 1e-3
        sz = 2 if od == torch.bfloat16 else 4
        nbytes = N * dim * 2 + N * 12 + N * nq * sz + nq * (dim * 2 + 36)
        flops = 2.0 * N * nq * dim
        key = f"nq{nq}_dim{dim}_{'bf16' if sz == 2 else 'f32'}"
        rows[key] = {"us": round(t * 1e6, 2), "bound": "hbm", "algorithmic_bytes": int(nbytes),
                     "achieved_gbs": round(nbytes / t / 1e9, 1), "peak_gbs": peak,
                     "frac": round(nbytes / t / 1e9 / peak, 4), "tensor_tflops": round(flops / t / 1e12, 2),
                     "tensor_frac": round(flops / t / 1e12 / tpeak, 5), "traffic": NCU_QUERY_TRAFFIC.get(key)}
        if key == "nq32_dim32_bf16":
            mask_lab = lab
    rows["peaks"] = {"hbm": src, "bf16_tflops": tpeak, "bf16_source": tsrc}
    # the instance mask: labels blended by the Top-K renderer, argmax per pixel
    p = make_params(C=32, K=K_TOP, feat_dtype=torch.bfloat16, stop_rule="exact_topk")
    fr = Frame([poses[0]], N_SPLATS, p, pair_capacity=1 << 21, device=dev)
    label = torch.empty(fr.total_pix, dtype=torch.int32, device=dev)
    F = torch.empty(fr.total_pix, 32, dtype=torch.bfloat16, device=dev)
    ms = []
    for cam in poses:
        fr.cams = make_cams([cam])
        fr.bin_and_sort(means, scales, quats, opac)
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fr.render_forward_aux(rgb, mask_lab, F, None, None, None, label=label)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
    rows["mask_render_ms"] = round(float(np.mean(ms)), 4)
    rows["mask_covered"] = round(float((label >= 0).float().mean().item()), 4)
    del fr
    return rows


def e2e(path, torch, dev, ptr, L, args):
    """Same step through the C ABI with host buffers: per step the targets go
    host->device from pinned memory and the loss comes back.  The copies run
    on a second stream into two alternating device buffers, so step i+1's
    targets travel while step i computes (the compute stream waits for its
    buffer's copy, and a copy waits until the step two back has released its
    buffer).  The compute of a step is the same CUDA graph of C ABI calls as
    the device-timed step, captured once per (pose, buffer); the waits on the
    copies sit between the replays, on the compute stream."""
    F_h = path.F_tgt.cpu().pin_memory()
    r_h = torch.empty(path.frame.total_pix, 3).pin_memory()
    r_h.copy_(torch.rand(path.frame.total_pix, 3))
    loss_h = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    F_d = [torch.empty_like(path.F_tgt) for _ in range(2)]
    r_d = [torch.empty(path.frame.total_pix, 3, device=dev) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    released = [torch.cuda.Event() for _ in range(2)]
    compute = torch.cuda.current_stream()
    old_F, old_r = path.F_tgt, path.rgb_tgt
    n_poses = len(path.graphs) or 1
    graphs = [[], []]
    for b in range(2):  # one graph per (pose, buffer): the graph reads that buffer's targets
        path.F_tgt, path.rgb_tgt = F_d[b], r_d[b]
        for i in range(n_poses):
            path.step(i)
        torch.cuda.synchronize()
        for i in range(n_poses):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                path.step(i)
            graphs[b].append(g)
    torch.cuda.synchronize()
    for e in released:
        e.record(compute)
    steps = max(8, args.steps // 4)

    def step(i):
        b = i & 1
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(released[b])
            F_d[b].copy_(F_h, non_blocking=True)
            r_d[b].copy_(r_h, non_blocking=True)
            copied[b].record(copy_stream)
        compute.wait_event(copied[b])
        graphs[b][i % n_poses].replay()
        released[b].record(compute)
        loss_h[b].copy_(path.loss, non_blocking=True)

    for i in range(3):
        step(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        step(i)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    path.F_tgt, path.rgb_tgt = old_F, old_r
    del graphs
    return {"value": round(steps / dt, 2), "unit": "frames/s",
            "h2d_bytes_per_step": int(F_h.numel() * F_h.element_size() + r_h.numel() * 4),
            "d2h_bytes_per_step": 8,
            "copies": "second stream, two alternating buffers; compute as CUDA-graph replays of the C ABI calls"}


BAND = 160  # rows per oracle step: ten 16-row tile rows, a third of a 640x480 frame


class OracleSteps:
    """The FP64 checker as it stands, stepping through the bench's frames in
    bands of BAND rows (each call of the checker also prepares the whole
    scene, so a frame in three bands costs a little more than in one call):
    step i renders (forward, OpenMP over the host cores)
    and differentiates (backward, one thread) rows [b BAND, (b+1) BAND) of
    pose f, with f, b = divmod(i, bands per frame); a frame's binning runs
    at its first band and counts in that step.  A band camera is the pose
    with height BAND and cy - b BAND, whose tiles are the frame's tile rows,
    so its lists are a slice of the frame's: every frame costs one binning
    and all its rows, as a whole frame does."""

    def __init__(self, sc, poses):
        import oracle as O

        O.build()
        self.O, self.sc, self.poses = O, sc, poses
        self.p = O.make_params(K=K_TOP, stop_rule=O.EXACT_TOPK)
        self.threads = O.num_threads()
        self.nb = poses[0].height // BAND
        self.frame, self.binned = None, None
        self.rng = np.random.default_rng(0)

    def step(self, i):
        import dataclasses

        O = self.O
        f, b = divmod(i, self.nb)
        cam = self.poses[f % len(self.poses)]
        if self.frame != f:
            self.binned = O.binning(self.sc, cam, self.p)
            self.frame = f
        bcam = dataclasses.replace(cam, height=BAND, cy=np.float32(cam.cy - b * BAND))
        tx = (cam.width + 15) // 16
        tr0 = b * BAND // 16
        rng = self.binned["ranges"][tr0 * tx:(tr0 + BAND // 16) * tx]
        bb = dict(self.binned, ranges=rng)
        ref = O.render(self.sc, bcam, self.p, binned=bb, threads=self.threads)
        gF = self.rng.normal(size=ref["F"].shape) * 1e-3
        grgb = self.rng.normal(size=ref["rgb"].shape) * 1e-3
        O.render_backward(self.sc, bcam, self.p, gF, grgb, None, binned=bb)

    def sample(self, steps, warmup=0):
        for i in range(warmup):
            self.step(i)
        self.frame = None  # the timed steps start with a fresh frame (its binning included)
        t0 = time.perf_counter()
        for i in range(steps):
            self.step(i)
        dt = time.perf_counter() - t0
        frames = steps / self.nb
        return {"value": round(frames / dt, 4), "unit": "frames/s", "cores": self.threads, "kind": "oracle",
                "sample": f"{steps} bands of {BAND} rows ({frames:.1f} frames of 640x480 over the 16 poses, each "
                          f"frame's binning once) of the same workload, FP64 forward (OpenMP, {self.threads} threads) "
                          f"+ backward (1 thread)", "seconds": round(dt, 2)}


def cpu_baseline(sc, poses, steps=15):
    """The checker on a bounded sample of the bench's workload (about ten
    seconds of CPU work: five frames in 160-row bands)."""
    return OracleSteps(sc, poses).sample(steps)


# ---------------------------------------------------------------------------
# reference arm: the FP64 checker on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    """The reference arm: the FP64 checker, W untimed and K timed steps of
    160-row bands of the bench's frames (OracleSteps), on rank 0 only (the
    other ranks of a torchrun launch exit without work)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2604_10951_gb300 import scenes

    sc = scenes.room_scene(n=N_SPLATS, C=C_FEAT, seed=SEED)
    poses = scenes.circle_poses(16)
    res = OracleSteps(sc, poses).sample(args.steps, args.warmup)
    out = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": "frames/s",
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(res["seconds"] * 1e3 / max(1, args.steps), 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "room 500k surfels, 640x480 (fx=fy=525), C=64, K=8 Top-K, forward+backward "
                                  "(FP64 checker, one step = a 160-row band of a frame)"},
           "cpu_baseline": res,
           "e2e": {"value": res["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)

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
def make_events(torch, n):
    try:  # events that become graph nodes, so per-call times survive graph replay
        return [torch.cuda.Event(enable_timing=True, external=True) for _ in range(n)]
    except TypeError:
        return None


FWD_CALLS = ["project_bin", "sort", "render_forward"]
STEP_CALLS = ["project_bin", "sort_render_forward_loss", "render_backward"]
FWD_KERNELS = ["k_project", "k_emit", "k_tile_sort"]
# kernels per fwd+bwd step: project_bin 2 (project; emit, whose first CTA scans the tile counts), then the
# sort, forward and loss in one kernel (Top-K, K <= 8: each CTA sorts its tile, renders it and evaluates the
# loss on it), backward 5 (clear, feature grads + dots, geometry replay, projection, feature rows)
BWD_KERNELS = ["k_bwd_clear", "k_bwd_feat", "k_bwd_geo", "k_bwd_project", "k_feat_out"]
KERNELS = FWD_KERNELS[:2] + ["k_render_topk"] + BWD_KERNELS


def step_kernels(K, backward):
    """The kernels one step of StepPath launches, in order: the forward path
    (binning, sort, render), or the training step, where for the plain Top-K
    selection with K <= 8 the render kernel also sorts its tile and
    evaluates the loss, else the sort and the loss run as kernels of their own."""
    render = "k_render_topk" if K else "k_render_full"
    if not backward:
        return FWD_KERNELS + [render]
    fwd = [render] if 0 < K <= 8 else ["k_tile_sort", render, "k_loss"]
    return FWD_KERNELS[:2] + fwd + [k for k in BWD_KERNELS if K or k != "k_bwd_feat"]


class StepPath:
    """Buffers and the step of one configuration, every call through the C
    ABI, replayed as one CUDA graph per camera set: binning, sort, forward
    render, and (``backward``) the L2-feature/L1-RGB loss (in the forward
    call, fss_render_forward_loss) and the backward render.  ``cam_sets`` lists the camera sets the steps cycle over (one
    view each, or several views rendered in one call)."""

    def __init__(self, torch, L, dev, scene_t, cam_sets, N, C, K, dtype, stop, backward=True, ts=16,
                 schedule="grid", rank=0, world=1, targets_seed=4):
        from paper_2604_10951_gb300 import scenes
        from paper_2604_10951_gb300.raster import Frame, make_cams, make_params

        self.torch, self.L, self.dev = torch, L, dev
        self.means, self.scales, self.quats, self.opac, self.rgb = scene_t["geo"]
        self.feats = scene_t["feats"][dtype]
        self.N, self.C, self.K, self.dtype = N, C, K, dtype
        self.s = 2 if dtype == torch.bfloat16 else 4
        self.ts, self.backward, self.rank, self.world = ts, backward, rank, world
        self.params = make_params(C=C, K=K, tile_size=ts, bin_mode="accu", stop_rule=stop, feat_dtype=dtype,
                                  out_dtype=dtype, schedule=schedule)
        self.cam_sets = cam_sets
        self.cams_c = [make_cams(cs) for cs in cam_sets]
        self.n_cams = len(cam_sets[0])
        self.frame = Frame(cam_sets[0], N, self.params, pair_capacity=1 << 20, device=dev)
        cap = 0
        for c in self.cams_c:  # size the pair capacity from every camera set, with margin
            self.frame.cams = c
            cap = max(cap, self.frame.bin_and_sort(self.means, self.scales, self.quats, self.opac))
        self.frame._alloc(int(cap * 1.3) + 4096)
        self.max_pairs = cap
        self.F, self.rgb_o, self.T, self.ids = self.frame.new_outputs()
        npx = self.frame.total_pix
        self.npx = npx
        self.render_kernel = "k_render_topk" if K else "k_render_full"
        self.fused_loss = False
        self.kernels = step_kernels(K, False)
        self.calls = FWD_CALLS
        if backward:
            F_t, rgb_t = scenes.targets(targets_seed, npx, C)
            self.F_tgt = torch.as_tensor(F_t).to(dev).to(dtype)
            self.rgb_tgt = torch.as_tensor(rgb_t).to(dev)
            self.dF = torch.empty_like(self.F)
            self.drgb = torch.empty_like(self.rgb_o)
            self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
            self.g = [torch.empty(N, k, device=dev) for k in (3, 2, 4)] + \
                     [torch.empty(N, device=dev), torch.empty(N, 3, device=dev)]
            self.gfeat = torch.empty(N, C, dtype=dtype, device=dev)
            # the loss runs inside the Top-K kernel for K <= 8, else as its own kernel
            self.fused_loss = 0 < K <= 8
            self.kernels = step_kernels(K, True)
            self.calls = STEP_CALLS
        self.graphs, self.gevents = [], []
        self.ncu = False  # the ncu constants above describe this path's kernels (the main workload only)

    @property
    def n_sets(self):
        return len(self.cams_c)

    def step(self, i, events=None):
        L, torch = self.L, self.torch
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        fr, p, ws = self.frame, self.params, ptr(self.frame.ws)
        sp = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        cams = self.cams_c[shard_pose(i, self.rank, self.world, self.n_sets)]
        a = (p, cams, self.n_cams, self.N)
        rec = (lambda k: events[k].record()) if events else (lambda k: None)
        rec(0)
        L.fss_project_bin(*a, ptr(self.means), ptr(self.scales), ptr(self.quats), ptr(self.opac), ws, fr.cap, sp)
        rec(1)
        if not self.backward:
            L.fss_sort(*a, ws, fr.cap, sp)
            rec(2)
            L.fss_render_forward(*a, ws, fr.cap, ptr(self.rgb), ptr(self.feats), ptr(self.F), ptr(self.rgb_o),
                                 ptr(self.T), ptr(self.ids), ptr(fr.saved), sp)
            rec(3)
            return
        L.fss_sort_render_forward_loss(*a, ws, fr.cap, ptr(self.rgb), ptr(self.feats), ptr(self.F),
                                       ptr(self.rgb_o), ptr(self.T), ptr(self.ids), ptr(fr.saved), ptr(self.F_tgt),
                                       ptr(self.rgb_tgt), 1.0, 1.0, ptr(self.dF), ptr(self.drgb), ptr(self.loss), sp)
        rec(2)
        L.fss_render_backward(*a, ws, fr.cap, ptr(self.means), ptr(self.scales), ptr(self.quats), ptr(self.opac),
                              ptr(self.rgb), ptr(self.feats), ptr(fr.saved), ptr(self.T), ptr(self.dF),
                              ptr(self.drgb), None, *(ptr(g) for g in self.g), ptr(self.gfeat), sp)
        rec(3)

    def capture(self):
        """One graph per camera set: the whole step."""
        torch = self.torch
        for i in range(self.n_sets):
            self.step(i)  # sets kernel attributes outside capture
        torch.cuda.synchronize()
        for i in range(self.n_sets):
            g = torch.cuda.CUDAGraph()
            ev = make_events(torch, len(self.calls) + 1)
            with torch.cuda.graph(g):
                self.step(i, ev)
            self.graphs.append(g)
            self.gevents.append(ev)
        torch.cuda.synchronize()

    def check(self):
        for c in self.cams_c:
            self.frame.cams = c
            s, n = self.frame.read_status()
            if s != self.L.FSS_OK:
                raise RuntimeError(f"device status {s}: {self.L.last_error()}")

    def time_steps(self, steps, warmup, flush, barrier=lambda: None):
        torch = self.torch
        if not self.graphs:
            self.capture()
        for i in range(warmup):
            self.graphs[i % len(self.graphs)].replay()
        torch.cuda.synchronize()
        barrier()
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
        if self.gevents[0] is not None:  # last replay of each set's graph
            used = self.gevents[:min(steps, len(self.gevents))]
            for k, n in enumerate(self.calls):
                calls[n] = float(np.mean([e[k].elapsed_time(e[k + 1]) for e in used]))
        self.check()
        return step_ms, calls, wall


def percentiles(ms):
    return {q: round(float(np.percentile(ms, v)), 4) for q, v in (("p10", 10), ("p50", 50), ("p90", 90))}


def run_ours(args):
    import torch

    D = Dist("nccl")
    torch.cuda.set_device(D.local)
    from paper_2604_10951_gb300 import _lib as L
    from paper_2604_10951_gb300 import scenes
    from paper_2604_10951_gb300.build import build

    build()
    dev = torch.device("cuda", D.local)
    sc = scenes.room_scene(n=N_SPLATS, C=C_FEAT, seed=SEED)
    poses = scenes.circle_poses(16)
    H, W = poses[0].height, poses[0].width
    npx = H * W
    scene_t = device_scene(torch, dev, sc)
    means, scales, quats, opac, rgb = scene_t["geo"]
    feats = scene_t["feats"]
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    if args.queries_only:
        if D.rank == 0:
            print(json.dumps({"query_labels": queries(torch, dev, sc, means, scales, quats, opac, rgb, poses, flush)}))
        D.close()
        return

    ours = StepPath(torch, L, dev, scene_t, [[c] for c in poses], N_SPLATS, C_FEAT, K_TOP, torch.bfloat16,
                    "exact_topk", rank=D.rank, world=D.world)
    ours.ncu = True
    with ClockSampler(D.local) as clk:
        step_ms, calls, wall = ours.time_steps(args.steps, args.warmup, flush, D.barrier)
    total_ms = D.max(float(np.sum(step_ms)))
    ms_step = total_ms / args.steps
    frames = args.steps * D.world
    value = frames / (total_ms / 1e3)
    launches_per_step = len(KERNELS)

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
           "step_ms": percentiles(step_ms),
           "calls_ms": {k: round(v, 4) for k, v in calls.items()},
           "pairs_per_frame_max": ours.max_pairs}
    clocks = clk.summary()
    if clocks:
        out["clocks"] = clocks
    if not args.no_extras:
        # the plain FP32 full-accumulation path on the same frames
        base = StepPath(torch, L, dev, scene_t, [[c] for c in poses], N_SPLATS, C_FEAT, 0, torch.float32, "tmin",
                        rank=D.rank, world=D.world)
        b_ms, b_calls, _ = base.time_steps(max(32, args.steps // 4), 3, flush)
        b_ms_step = D.max(float(np.sum(b_ms))) / len(b_ms)
        out["fp32_full_path"] = {"ms_per_step": round(b_ms_step, 4), "frames_per_s": round(1e3 / b_ms_step, 2),
                                 "calls_ms": {k: round(v, 4) for k, v in b_calls.items()},
                                 "speedup_of_bf16_topk": round(b_ms_step / ms_step, 3)}
        del base
        # the same frames forward only (binning, sort, render; one graph per pose)
        fwd = StepPath(torch, L, dev, scene_t, [[c] for c in poses], N_SPLATS, C_FEAT, K_TOP, torch.bfloat16,
                       "exact_topk", backward=False, rank=D.rank, world=D.world)
        f_ms, _, _ = fwd.time_steps(max(64, args.steps // 4), 3, flush)
        fwd_ms = D.max(float(np.sum(f_ms))) / len(f_ms)
        out["forward_only"] = {"ms": round(fwd_ms, 4), "frames_per_s": round(1e3 / fwd_ms, 2)}
        del fwd
        rf = path_roofline(ours, torch, L, flush, float(np.mean(step_ms)))
        out["roofline"], out["roofline_kernels"], out["kernel_us"], out["roofline_frame"] = \
            rf["main"], rf["rows"], rf["kernel_us"], rf["frame"]
        out["kernel_us_hooked"], out["hook"] = rf["kernel_us_hooked"], rf["hook"]
        out["e2e"] = e2e(ours, torch, dev, L, args)
        out["e2e_sensor_fwd"] = e2e_sensor(torch, dev, L, scene_t, poses, args)
        out["ablation_fwd"] = ablation(torch, L, dev, means, scales, quats, opac, rgb, feats[torch.float32], poses,
                                       flush)
        out["variants_render_ms"] = variants(torch, dev, means, scales, quats, opac, rgb, feats[torch.bfloat16],
                                             poses, flush)
        out["query_labels"] = queries(torch, dev, sc, means, scales, quats, opac, rgb, poses, flush)
        out["room_fwd_K"] = room_fwd_K(torch, L, dev, args, flush, D)
        del ours
        torch.cuda.empty_cache()
        out["large_fwd"] = large_fwd(torch, L, dev, args, flush, D)
        torch.cuda.empty_cache()
        out["batched_fb"] = batched_fb(torch, L, dev, args, flush, D)
        torch.cuda.empty_cache()
    if D.rank == 0 and D.world == 1 and not args.no_extras:  # the checker's leg: rank 0 at N = 1 only
        out["cpu_baseline"] = cpu_baseline(sc, poses)
        out["precision_vs_oracle"] = precision_sample()
    if D.rank == 0:
        print(json.dumps(out))
    D.close()


def device_scene(torch, dev, sc):
    t32 = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
    geo = tuple(t32(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities, sc.rgb))
    f = t32(sc.feats)
    return {"geo": geo, "feats": {torch.bfloat16: f.bfloat16(), torch.float32: f}}


# dram__bytes_read.sum + dram__bytes_write.sum of one launch inside the step (camera
# pose 0, the L2 contents the step's earlier kernels left; ncu --cache-control none),
# from the in-step traffic summary under profiles/; to be set to None whenever the
# kernel changes after that capture
NCU_TRAFFIC = {"k_render_topk": None, "k_bwd_feat": 12216832 + 21090048, "k_bwd_geo": 12893440 + 9380352}
# (smsp__inst_executed.sum, gpu__time_duration.sum in us) of the one-kernel --set full
# captures summarised under profiles/
NCU_ISSUE = {"k_render_topk": None, "k_bwd_feat": (61610201, 76.096), "k_bwd_geo": (82220205, 101.536)}
# the query-label kernel's capture (summarised under profiles/): DRAM read + write
NCU_QUERY_TRAFFIC = {"nq32_dim32_f32": 47276544}


def kernel_times(path, torch, L, flush, rounds=4):
    """Per-kernel durations (ms) averaged over the path's camera sets, from
    events that the library records after each of its launches
    (fss_set_kernel_events), captured into one graph per set; L2 flushed
    before every replay.  Also the algorithmic bytes of each kernel for
    those sets."""
    graphs, evs = [], []
    names = path.kernels
    for i in range(path.n_sets):
        # the first event is recorded by torch inside the capture (an external event
        # becomes a graph node); the others by the library after each launch
        ev = [torch.cuda.Event(enable_timing=True, external=True)] + \
             [torch.cuda.Event(enable_timing=True) for _ in range(len(names))]
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
    sums = np.zeros(len(names))
    n = 0
    nbytes, sizes = {}, {}
    for r in range(rounds):
        for i, (g, ev) in enumerate(zip(graphs, evs)):
            flush.zero_()
            g.replay()
            torch.cuda.synchronize()
            sums += [ev[k].elapsed_time(ev[k + 1]) for k in range(len(names))]
            n += 1
            if r == 0:  # the set's algorithmic bytes, averaged over the sets
                b, z = algorithmic_bytes(path, torch, L)
                for k in b:
                    nbytes[k] = nbytes.get(k, 0.0) + b[k] / len(graphs)
                for k in z:
                    sizes[k] = sizes.get(k, 0.0) + z[k] / len(graphs)
    return dict(zip(names, (sums / n).tolist())), nbytes, {k: int(round(v)) for k, v in sizes.items()}


def unique_rows(ids, sizes, pix_off, ts):
    """U: per tile, the distinct surfels of its pixels' Top-K sets, summed over tiles."""
    U = 0
    for (h, w), a in zip(sizes, pix_off):
        v = ids[a:a + h * w].reshape(h, w, -1)
        for ty in range(0, h, ts):
            for tx in range(0, w, ts):
                blk = v[ty:ty + ts, tx:tx + ts].reshape(-1)
                U += np.unique(blk[blk >= 0]).size
    return U


def algorithmic_bytes(path, torch, L):
    """Unique bytes each kernel of the step must move per launch for the
    camera set last rendered by `path`: reads of its inputs and writes of its
    outputs once, nothing re-read."""
    fr = path.frame
    ranges = fr.region(L.REG_RANGES).view(torch.int32).view(-1, 2).cpu().numpy()
    P = int((ranges[:, 1] - ranges[:, 0]).sum())
    tiles = ranges.shape[0]
    st = fr.region(L.REG_STATUS).view(torch.int32)[:28].cpu().numpy()
    cnt = fr.region(L.REG_STATUS).view(torch.int64)[2:10].cpu().numpy()
    nslot = int(st[22])
    nvis = int(st[20]) + int(st[25])  # bounded visible items (narrow + wide)
    n_eval, n_contrib = int(cnt[0]), int(cnt[1])
    s, K, Cc, npx, N, ts = path.s, path.K, path.C, path.npx, path.N, path.ts
    V = path.n_cams
    U = unique_rows(path.ids.cpu().numpy(), fr.sizes, fr.pix_off, ts) if K else 0
    b = {
        "k_project": V * N * 16 + nvis * (24 + 64 + 80 + 8),  # centres and opacities of all, the rest of the visible
        "k_emit": tiles * 12 + nvis * (80 + 64 + 4) + P * 4,
        "k_tile_sort": P * (4 + 4 + 64 + 4 + 4),
    }
    if K:
        # ranges; per pair: list id, warp mask, adjugate rows, opacity, colour;
        # selected rows once per tile; per pixel: features, rgb, T, ids, saved pos/w, nstop
        b["k_render_topk"] = tiles * 8 + P * (4 + 4 + 48 + 4 + 12) + U * Cc * s + npx * (Cc * s + 12 + 4 + 4 * K * 3 + 4)
    else:
        # per pair the record and the feature row (staged once per tile); per pixel F, rgb, T, nstop
        b["k_render_full"] = tiles * 8 + P * (4 + 4 + 48 + 4 + 12 + Cc * s) + npx * (Cc * s + 12 + 4 + 4)
    if path.backward:
        loss_b = npx * (2 * Cc * s + 24) + npx * (Cc * s + 12)  # F, F_t, rgb, rgb_t read; dL/dF, dL/drgb written
        if path.fused_loss:  # the sort and the loss in the render kernel: F is not read back
            b["k_render_topk"] += loss_b - npx * (Cc * s + 12) + b.pop("k_tile_sort")
        else:
            b["k_loss"] = loss_b
        b.update({
            "k_bwd_clear": nslot * (64 + 4 * Cc),
            "k_bwd_project": N * 52 + nslot * (V * 64 + 48 + 40),
            "k_feat_out": N * Cc * s + nslot * 4 * Cc,
        })
        if K:
            # per pixel: saved pos/w, dL/dF, dots written; selected rows (+ list id, slot) once
            # per tile; the FP32 feature-gradient accumulators written once
            b["k_bwd_feat"] = tiles * 8 + npx * (8 * K + Cc * s + 4 * K) + U * (Cc * s + 8) + nslot * Cc * 4
            # per pixel: nstop, T, dL/drgb, saved pos, dots; per pair: list id, mask, record
            # rows, colour; the per-(view, slot) gradient rows written once
            b["k_bwd_geo"] = tiles * 8 + npx * (4 + 4 + 12 + 8 * K) + P * (4 + 4 + 64 + 12) + nslot * V * 64
        else:
            b["k_bwd_geo"] = tiles * 8 + npx * (4 + 4 + 12 + Cc * s) + P * (4 + 4 + 64 + 12 + Cc * s) \
                + nslot * V * 64 + nslot * Cc * 4
    # FP32 operations of the forward: ~20 per evaluation (ray-splat solve,
    # density, opacity, depth test) + ~10 per contribution (compositing, K-set
    # test) + 2 C per selected row (feature accumulation); two MUFU ops per evaluation
    flops_fwd = 20 * n_eval + 10 * n_contrib + 2 * Cc * (min(K, 8) * npx if K else n_contrib)
    return b, {"pairs": P, "unique_rows": U, "slots": nslot, "evaluations": n_eval, "contributions": n_contrib,
               "flops_fwd": flops_fwd}


def hook_corrected(kt_raw, step_ms):
    """Per-kernel times without the event hook's own cost: the hooked
    kernel times sum to more than the hook-free step (each recorded event
    adds a gap after its kernel), so the excess over the hook-free step's
    mean is split evenly over the kernels and taken off each."""
    tot = sum(kt_raw.values())
    over = max(0.0, (tot - step_ms) / len(kt_raw))
    return {k: max(v - over, 1e-6) for k, v in kt_raw.items()}, {
        "hooked_sum_ms": round(tot, 5), "hook_free_step_ms": round(step_ms, 5),
        "overhead_us_per_kernel": round(over * 1e3, 3),
        "method": "per-kernel event times minus an even share of (hooked sum - hook-free step mean)"}


def path_roofline(path, torch, L, flush, step_ms, rounds=4):
    """Roofline of the path's dominant kernel (largest average duration):
    algorithmic bytes per launch / its event-timed duration (both averaged
    over the camera sets, the duration corrected for the hook), against the
    measured HBM copy bandwidth; the render kernels alongside, and the frame
    total."""
    peak, src = measured_peaks()
    raw, nbytes, sizes = kernel_times(path, torch, L, flush, rounds)
    kt, hook = hook_corrected(raw, step_ms)
    rows = {}
    for k, b in nbytes.items():
        ach = b / (kt[k] * 1e-3) / 1e9
        rows[k] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                   "traffic": NCU_TRAFFIC.get(k) if path.ncu else None,
                   "algorithmic_bytes": int(b), "ms": round(kt[k], 5)}
    # the forward's arithmetic against the FP32 peak: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
    fp32_peak = 152 * 128 * 2 * 2.07e9
    rk = path.render_kernel
    rows[rk]["alu"] = {"flops": int(sizes["flops_fwd"]),
                       "achieved_tflops": round(sizes["flops_fwd"] / (kt[rk] * 1e-3) / 1e12, 2),
                       "peak_tflops": round(fp32_peak / 1e12, 1),
                       "frac": round(sizes["flops_fwd"] / (kt[rk] * 1e-3) / fp32_peak, 4)}
    # warp-instruction issue of the ncu captures against 152 SMs x 4 schedulers x 2.07 GHz
    for k, v in NCU_ISSUE.items():
        if k in rows and v is not None and path.ncu:
            rows[k]["issue_frac_ncu"] = round(v[0] / (v[1] * 1e-6) / (152 * 4 * 2.07e9), 3)
    dom = max(kt, key=kt.get)
    main = dict(rows[dom], kernel=dom, peak_source=f"{src} (MEASURED_PEAKS.json hbm_gbs)")
    main.update({k: v for k, v in sizes.items() if k != "flops_fwd"})
    # per frame: all kernels' algorithmic bytes over the summed kernel times
    tot_b = sum(nbytes.values())
    tot_t = sum(kt.values()) * 1e-3
    frame = {"algorithmic_bytes": int(tot_b), "kernel_ms": round(tot_t * 1e3, 4),
             "achieved": round(tot_b / tot_t / 1e9, 1), "peak": peak, "unit": "GB/s",
             "frac": round(tot_b / tot_t / 1e9 / peak, 4)}
    render_rows = {k: v for k, v in rows.items() if k.startswith(("k_render", "k_bwd_feat", "k_bwd_geo"))}
    return {"main": main, "rows": render_rows, "kernel_us": {k: round(v * 1e3, 2) for k, v in kt.items()},
            "kernel_us_hooked": {k: round(v * 1e3, 2) for k, v in raw.items()}, "frame": frame, "hook": hook}


def workload_line(path, torch, L, flush, steps, warmup, D, per="frames"):
    """Timed graph replays of a path (L2 flushed between steps), its step
    percentiles and its dominant kernel's roofline."""
    ms, calls, _ = path.time_steps(steps, warmup, flush, D.barrier)
    ms_step = D.max(float(np.sum(ms))) / len(ms)
    rf = path_roofline(path, torch, L, flush, float(np.mean(ms)), rounds=2)
    views = path.n_cams
    return {"ms_per_step": round(ms_step, 4), f"{per}_per_s": round(views * 1e3 / ms_step, 2),
            "steps": steps, "step_ms": percentiles(ms), "calls_ms": {k: round(v, 4) for k, v in calls.items()},
            "roofline": rf["main"], "kernel_us": rf["kernel_us"], "pairs_per_step_max": path.max_pairs}


def room_fwd_K(torch, L, dev, args, flush, D):
    """The room forward workload (500k surfels, seed 1, FP32 C = 64 features,
    640x480 over 16 poses): binning + sort + render, full accumulation and
    Top-K K = 4, 8, 16 (exact stop), each step one graph replay."""
    from paper_2604_10951_gb300 import scenes

    sc = scenes.room_scene(n=N_SPLATS, C=C_FEAT, seed=1)
    scene_t = device_scene(torch, dev, sc)
    poses = [[c] for c in scenes.circle_poses(16)]
    rows = {}
    for K in (0, 4, 8, 16):
        p = StepPath(torch, L, dev, scene_t, poses, N_SPLATS, C_FEAT, K, torch.float32,
                     "exact_topk" if K else "tmin", backward=False, rank=D.rank, world=D.world)
        rows["full" if K == 0 else f"K{K}"] = workload_line(p, torch, L, flush, max(32, args.steps // 4), 3, D)
        del p
    rows["workload"] = "room 500k surfels (seed 1), 640x480 f=525, FP32 C=64, forward (binning, sort, render)"
    return rows


def large_fwd(torch, L, dev, args, flush, D):
    """The large forward workload: 1.5M surfels in the room generator (seed
    2), BF16 C = 128 features, 1280x720 (f = 900) over 32 poses, Top-K K = 8."""
    from paper_2604_10951_gb300 import scenes

    sc = scenes.room_scene(n=1_500_000, C=128, seed=2)
    scene_t = device_scene(torch, dev, sc)
    poses = [[c] for c in scenes.circle_poses(32, 1280, 720, 900.0)]
    p = StepPath(torch, L, dev, scene_t, poses, sc.n, 128, K_TOP, torch.bfloat16, "exact_topk", backward=False,
                 rank=D.rank, world=D.world)
    row = workload_line(p, torch, L, flush, max(64, args.steps // 4), 3, D)
    row["workload"] = "large 1.5M surfels (seed 2), 1280x720 f=900, BF16 C=128, K=8 exact stop, forward"
    return row


def batched_fb(torch, L, dev, args, flush, D):
    """The batched workload: 1M surfels (seed 6), BF16 C = 128, K = 8, 12
    cameras of mixed size (4x 320x240, 4x 640x480, 4x 1280x720) rendered in
    one call per step (forward + loss + backward), with the tile size,
    schedule and stop rule the autotuner picks; one graph replay per step."""
    from paper_2604_10951_gb300 import scenes
    from paper_2604_10951_gb300.tune import Autotuner

    sc = scenes.room_scene(n=1_000_000, C=128, seed=6)
    scene_t = device_scene(torch, dev, sc)
    cams = scenes.batched_cameras()
    means, scales, quats, opac, rgb = scene_t["geo"]
    t0 = time.perf_counter()
    best = Autotuner().tune(cams, means, scales, quats, opac, rgb, scene_t["feats"][torch.bfloat16], K=K_TOP, reps=3)
    tune_s = time.perf_counter() - t0
    p = StepPath(torch, L, dev, scene_t, [cams], sc.n, 128, K_TOP, torch.bfloat16, best["stop_rule"],
                 ts=best["tile_size"], schedule=best["schedule"])
    row = workload_line(p, torch, L, flush, max(32, args.steps // 8), 3, D, per="views")
    row["autotuner"] = {k: v for k, v in best.items() if k != "all"}
    row["autotuner"]["seconds"] = round(tune_s, 1)
    row["autotuner"]["candidates_ms"] = {f"ts{c['tile_size']}_{c['schedule']}_{c['stop_rule']}": round(c["ms"], 3)
                                         for c in best["all"]}
    row["workload"] = ("batched 1M surfels (seed 6), 12 views (4x 320x240, 4x 640x480, 4x 1280x720) in one call, "
                       "BF16 C=128, K=8, forward + loss + backward, autotuned")
    return row


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


def e2e(path, torch, dev, L, args):
    """Same step through the C ABI with host buffers: per step the targets go
    host->device from pinned memory and the loss comes back.  The copies run
    on a second stream into two alternating device buffers, so step i+1's
    targets travel while step i computes (the compute stream waits for its
    buffer's copy, and a copy waits until the step two back has released its
    buffer).  The compute of a step is the same CUDA graph of C ABI calls as
    the device-timed step, captured once per (pose, buffer); the waits on the
    copies sit between the replays, on the compute stream.  At least 100
    timed steps."""
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
    n_poses = path.n_sets
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
    steps = max(100, args.steps)

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
    return {"value": round(steps / dt, 2), "unit": "frames/s", "steps": steps,
            "h2d_bytes_per_step": int(F_h.numel() * F_h.element_size() + r_h.numel() * 4),
            "d2h_bytes_per_step": 8,
            "copies": "second stream, two alternating buffers; compute as CUDA-graph replays of the C ABI calls"}


def e2e_sensor(torch, dev, L, scene_t, poses, args):
    """The simulator's sensor use (Sec. 4.4): per frame a forward render of
    the room workload's view (binning, sort, BF16 Top-K K = 8 features, RGB,
    expected depth through fss_render_forward_aux) whose features, colour
    and depth come back to pinned host buffers.  The device->host copies run
    on a second stream from two alternating output sets, so frame i's
    outputs travel while frame i+1 renders; each frame's compute is one CUDA
    graph of the C ABI calls per (pose, output set).  At least 100 frames."""
    from paper_2604_10951_gb300.raster import Frame, make_cams, make_params

    means, scales, quats, opac, rgb = scene_t["geo"]
    feats = scene_t["feats"][torch.bfloat16]
    p = make_params(C=C_FEAT, K=K_TOP, stop_rule="exact_topk", feat_dtype=torch.bfloat16)
    fr = Frame([poses[0]], N_SPLATS, p, pair_capacity=1 << 20, device=dev)
    cams_c = [make_cams([c]) for c in poses]
    cap = 0
    for c in cams_c:
        fr.cams = c
        cap = max(cap, fr.bin_and_sort(means, scales, quats, opac))
    fr._alloc(int(cap * 1.3) + 4096)
    npx = fr.total_pix
    outs = []
    for b in range(2):
        F, rgb_o, T, ids = fr.new_outputs()
        outs.append((F, rgb_o, T, ids, torch.empty(npx, device=dev)))
    host = [(torch.empty(outs[0][0].shape, dtype=outs[0][0].dtype).pin_memory(), torch.empty(npx, 3).pin_memory(),
             torch.empty(npx).pin_memory()) for _ in range(2)]
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())

    def compute(i, b):
        sp = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        cams = cams_c[i % len(cams_c)]
        a = (p, cams, 1, N_SPLATS)
        ws = ptr(fr.ws)
        F, rgb_o, T, ids, depth = outs[b]
        L.fss_project_bin(*a, ptr(means), ptr(scales), ptr(quats), ptr(opac), ws, fr.cap, sp)
        L.fss_sort(*a, ws, fr.cap, sp)
        L.fss_render_forward_aux(*a, ws, fr.cap, ptr(rgb), ptr(feats), ptr(F), ptr(rgb_o), ptr(T), ptr(ids),
                                 ptr(fr.saved), ptr(depth), None, None, sp)

    graphs = [[], []]
    for b in range(2):
        for i in range(len(cams_c)):
            compute(i, b)
        torch.cuda.synchronize()
        for i in range(len(cams_c)):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                compute(i, b)
            graphs[b].append(g)
    torch.cuda.synchronize()
    copy_stream = torch.cuda.Stream(device=dev)
    rendered = [torch.cuda.Event() for _ in range(2)]
    drained = [torch.cuda.Event() for _ in range(2)]
    main = torch.cuda.current_stream()
    for e in drained:
        e.record(copy_stream)

    def frame(i):
        b = i & 1
        main.wait_event(drained[b])  # the copy of frame i - 2 has left this output set
        graphs[b][i % len(cams_c)].replay()
        rendered[b].record(main)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(rendered[b])
            F, rgb_o, T, ids, depth = outs[b]
            hF, hr, hd = host[b]
            hF.copy_(F, non_blocking=True)
            hr.copy_(rgb_o, non_blocking=True)
            hd.copy_(depth, non_blocking=True)
            drained[b].record(copy_stream)

    for i in range(3):
        frame(i)
    torch.cuda.synchronize()
    steps = max(100, args.steps)
    t0 = time.perf_counter()
    for i in range(steps):
        frame(i)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s, _ = fr.read_status()
    d2h = sum(int(t.numel() * t.element_size()) for t in host[0])
    del graphs
    return {"value": round(steps / dt, 2), "unit": "frames/s", "steps": steps, "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": d2h, "status": int(s),
            "outputs": "features [640x480, 64] BF16, RGB, expected depth to pinned host memory per frame",
            "copies": "second stream, two alternating output sets; compute as CUDA-graph replays of the C ABI calls"}


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


def precision_sample():
    """Part of the checker's leg: the GPU path's error against the FP64
    oracle per output and per gradient (tests/precision_report.py), FP32 and
    BF16 feature storage, on one whole view of the room (500k surfels,
    640x480, C = 64) and large (1.5M surfels, 1280x720, C = 128) workloads."""
    from tests.precision_report import report

    t0 = time.perf_counter()
    out = report(("room", "large"))
    out.pop("band_rows", None)
    out["views"] = {"room": "pose 0 of 16, whole 640x480 frame", "large": "pose 7 of 32, whole 1280x720 frame"}
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


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

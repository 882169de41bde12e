"""Host-side logic of the benchmark, on CPU: the multi-process plumbing of a
torchrun launch (two gloo ranks: the barrier, the max-over-ranks timing
reduce, the interleaved pose shards) and the reference arm's band sampling
of the FP64 checker (a band step renders the frame's rows, to FP64 rounding)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import oracle as O
from paper_2604_10951_gb300 import scenes


def test_pose_shards_cover_the_stream_evenly():
    for world in (1, 2, 4, 8):
        seen = np.zeros(16, int)
        for step in range(32):
            poses = [bench.shard_pose(step, r, world, 16) for r in range(world)]
            assert len(set(poses)) == world  # the ranks render different views at once
            for q in poses:
                seen[q] += 1
        assert (seen == seen[0]).all()


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    D = bench.Dist("gloo")
    D.barrier()
    m = D.max(1.5 + rank)
    D.barrier()
    D.close()
    with open(os.path.join(out, f"r{rank}"), "w") as f:
        f.write(f"{D.rank} {D.world} {m}")


def test_two_gloo_ranks_reduce_the_slowest_time(tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        rank, world, m = open(tmp_path / f"r{r}").read().split()
        assert (int(rank), int(world), float(m)) == (r, 2, 2.5)


def test_reference_band_step_renders_the_frame_rows():
    sc = scenes.room_scene(n=30_000, C=8, seed=4)
    poses = scenes.circle_poses(4, 160, 2 * bench.BAND, 131.25)
    st = bench.OracleSteps(sc, poses)
    assert st.nb == 2
    seen = {}
    real = O.render

    def spy(scene, cam, params, **kw):
        out = real(scene, cam, params, **kw)
        seen[int(round(float(poses[0].cy) - float(cam.cy))) // bench.BAND] = out
        return out

    O.render = spy
    try:
        st.step(0)
        st.step(1)
    finally:
        O.render = real
    full = O.render(sc, poses[0], st.p)
    for b in (0, 1):
        rows = slice(b * bench.BAND, (b + 1) * bench.BAND)
        # the band camera's cy differs by whole rows: the same rays up to FP64 rounding
        for k in ("F", "rgb", "T"):
            np.testing.assert_allclose(seen[b][k], full[k][rows], rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(seen[b]["ids"], full["ids"][rows])
    res = st.sample(4, warmup=1)
    assert res["kind"] == "oracle" and res["value"] > 0 and f"bands of {bench.BAND} rows" in res["sample"]


class _FakeFrame:
    """The workspace regions that the bench's byte model reads, on the CPU:
    tile ranges and the status block's counts."""

    def __init__(self, torch, tiles=12, pairs_per_tile=5, sizes=((32, 48),)):
        import paper_2604_10951_gb300._lib as L
        self.L = L
        r = np.zeros((tiles, 2), np.int32)
        r[:, 0] = np.arange(tiles) * pairs_per_tile
        r[:, 1] = r[:, 0] + pairs_per_tile
        st = np.zeros(32, np.int32)
        st[20], st[22], st[25] = 40, 30, 2  # narrow visible items, slots, wide items
        self.regions = {L.REG_RANGES: torch.from_numpy(r.view(np.uint8).reshape(-1)),
                        L.REG_STATUS: torch.from_numpy(st.view(np.uint8).reshape(-1))}
        self.sizes = list(sizes)
        self.pix_off = [0]
        for h, w in self.sizes:
            self.pix_off.append(self.pix_off[-1] + h * w)

    def region(self, which):
        return self.regions[which]


class _FakePath:
    def __init__(self, torch, K, backward, dtype_bytes=2, C=16):
        self.frame = _FakeFrame(torch)
        self.s, self.K, self.C, self.N, self.ts, self.n_cams = dtype_bytes, K, C, 100, 16, 1
        self.npx = self.frame.pix_off[-1]
        self.ids = torch.zeros(self.npx, max(K, 1), dtype=torch.int32) if K else None
        self.backward = backward
        self.fused_loss = backward and 0 < K <= 8
        self.render_kernel = "k_render_topk" if K else "k_render_full"
        self.kernels = bench.step_kernels(K, backward)  # as StepPath sets them


@pytest.mark.parametrize("K,backward", [(8, True), (4, True), (0, True), (16, True), (8, False), (0, False)])
def test_byte_model_covers_exactly_the_step_kernels(K, backward):
    """Every kernel the step launches has algorithmic bytes and no other key
    appears (the roofline divides one by the other's event time), for the
    fused training step (sort and loss in the render kernel), the two-kernel
    cases and the forward-only paths."""
    import torch
    path = _FakePath(torch, K, backward)
    b, z = bench.algorithmic_bytes(path, torch, path.frame.L)
    assert set(b) == set(path.kernels), (sorted(b), path.kernels)
    assert all(v > 0 for v in b.values())
    assert z["pairs"] == 60 and z["slots"] == 30
    if backward and path.fused_loss:
        assert bench.KERNELS == path.kernels and len(bench.KERNELS) == 8

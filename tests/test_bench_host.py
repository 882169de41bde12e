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

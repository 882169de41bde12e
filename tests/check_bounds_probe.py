"""Probe of the check build (run in a process of its own with
FSS_CHECK_BOUNDS=1; tests/test_gpu_check_bounds.py runs it).

A clean frame (binning, sort, forward, backward) must report FSS_OK.  Then
one corruption per run, each of the device data an index is taken from,
must be refused by the device-side checks (the access skipped) and reported
by fss_read_status as FSS_ERR_BOUNDS naming the check:
  - a tile range reaching past the pair capacity;
  - a pair-list entry naming an item past the view's surfels;
  - a saved Top-K list position past its tile's list;
  - a workspace canary overwritten from the host.
Every corrupted value lies just past its valid range, so that even an
access that missed its check would stay inside the buffers (the inputs are
allocated with spare rows).  Prints one JSON line of (status, message) per case.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2604_10951_gb300 import _lib as L  # noqa: E402
from paper_2604_10951_gb300 import scenes  # noqa: E402
from paper_2604_10951_gb300.raster import Frame, make_params  # noqa: E402


def main():
    assert L.check_build(), "run with FSS_CHECK_BOUNDS=1"
    torch.cuda.set_device(0)
    sc, cam = scenes.tiny_scene(seed=0, n=2000, C=16)
    N, K = sc.n, 4
    spare = 64  # rows past N, so that a missed check would still read inside the allocation

    def padded(a, dtype=torch.float32):
        a = np.ascontiguousarray(a)
        t = torch.zeros((a.shape[0] + spare,) + a.shape[1:], dtype=dtype, device="cuda")
        t[:a.shape[0]] = torch.as_tensor(a).to("cuda", dtype)
        return t

    means, scales, quats, opac, rgb, feats = (padded(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities,
                                                                    sc.rgb, sc.feats))
    fr = Frame([cam], N, make_params(C=sc.C, K=K), pair_capacity=1 << 16)
    F, rgb_o, T, ids = fr.new_outputs()
    grads = [torch.empty_like(x) for x in (means, scales, quats, opac, rgb, feats)]
    dF, drgb = torch.randn_like(F), torch.randn_like(rgb_o)
    out = {}

    def status():
        s, _ = fr.read_status()
        return [int(s), L.last_error() if s else ""]

    def forward():
        fr.bin_and_sort(means, scales, quats, opac)
        fr.render_forward(rgb, feats, F, rgb_o, T, ids)

    def backward():
        fr.render_backward(means, scales, quats, opac, rgb, feats, T, dF, drgb, None, *grads)

    forward()
    backward()
    out["clean"] = status()
    ranges = fr.region(L.REG_RANGES).view(torch.int32).view(-1, 2)
    t = int(torch.argmax(ranges[:, 1] - ranges[:, 0]).item())  # the longest tile list
    r0, r1 = (int(v) for v in ranges[t].tolist())

    # a tile range past the pair capacity
    forward()
    ranges[t, 1] = fr.cap + 5
    fr.render_forward(rgb, feats, F, rgb_o, T, ids)
    out["range"] = status()

    # a pair-list entry naming an item past the surfels
    forward()
    fr.region(L.REG_LIST).view(torch.int32)[r0] = N + 3
    fr.render_forward(rgb, feats, F, rgb_o, T, ids)
    out["item"] = status()

    # a saved list position past its tile's list (pixel (0, 0) of tile t's first pixel)
    forward()
    ts = fr.params.tile_size
    tiles_x = (cam.width + ts - 1) // ts
    pix = (t // tiles_x) * ts * cam.width + (t % tiles_x) * ts
    pos = fr.saved[:fr.total_pix * K * 4].view(torch.int32).view(-1, K)
    pos[pix, 0] = (r1 - r0) + 7
    backward()
    out["position"] = status()

    # a canary overwritten on the host (the one after the pair list)
    forward()
    off, size = L.fss_workspace_region(*fr.args(), fr.cap, L.REG_LIST)
    guard = off + (size + 255) // 256 * 256
    torch.cuda.synchronize()
    fr.ws[guard + 17] = 0
    out["canary"] = status()

    # and a clean frame again afterwards
    forward()
    backward()
    out["clean_after"] = status()
    print(json.dumps(out))


if __name__ == "__main__":
    main()

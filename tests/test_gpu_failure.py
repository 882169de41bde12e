"""Failure detection on the GPU without a fault: the bounded device wait of
the binning (the emission kernel's CTAs wait for the one that scans the tile
counts) runs out when the scan withholds its result, the status block
reports FSS_ERR_TIMEOUT, and the same frame bins normally afterwards, bit
for bit as a fresh one."""
import numpy as np
import pytest
import torch

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300 import scenes
from paper_2604_10951_gb300.raster import Frame, make_params
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def test_binning_wait_runs_out_reports_timeout_and_recovers():
    sc, cam = scenes.tiny_scene(seed=4, n=3000, C=8)
    ins = [dev(x) for x in (sc.means, sc.scales, sc.quats, sc.opacities)]
    params = make_params(C=8, K=4)
    fr = Frame([cam], sc.n, params, pair_capacity=1 << 16)
    L.fss_test_hold_scan(True)
    try:
        fr.project_bin(*ins)
        status, _ = fr.read_status()
    finally:
        L.fss_test_hold_scan(False)
    assert status == L.FSS_ERR_TIMEOUT
    n = fr.bin_and_sort(*ins)  # the status was read (and cleared): the frame works again
    ref = Frame([cam], sc.n, params, pair_capacity=1 << 16)
    assert ref.bin_and_sort(*ins) == n > 0
    for r in (L.REG_RANGES, L.REG_LIST, L.REG_MASK):
        a, b = fr.region(r), ref.region(r)
        m = n * 4 if r != L.REG_RANGES else a.numel()
        assert torch.equal(a[:m], b[:m]), r

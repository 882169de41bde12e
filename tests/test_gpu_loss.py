"""fss_loss_l2_l1, the training loss of the forward+backward step, through
the C ABI against its definition evaluated in float64 on the host:

  L = w_f mean((F - F_t)^2) + w_c mean(|rgb - rgb_t|),
  dL/dF = 2 w_f (F - F_t) / (n C),  dL/drgb = w_c sign(rgb - rgb_t) / (3 n).

The kernel forms each difference and product in FP32 (the difference of two
BF16 values is exact in FP32) and rounds dL/dF once to the output type, so
dL/dF matches the float64 value rounded to FP32 and then to the output type
within one unit in the last place of the output type; dL/drgb is exact; L is
an FP32 sum of n C terms per thread, within 1e-5 relative.  Sizes span
several grid-stride steps and a ragged tail (n C / 8 not a multiple of the
grid)."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300.raster import _ptr, _stream, make_params

pytestmark = pytest.mark.gpu


def _run(n, Cc, dtype, wf, wc, seed):
    rng = np.random.default_rng(seed)
    F = torch.as_tensor(rng.normal(0.0, 1.0, (n, Cc)), dtype=torch.float32).to(dtype).cuda()
    Ft = torch.as_tensor(rng.normal(0.0, 1.0, (n, Cc)), dtype=torch.float32).to(dtype).cuda()
    rgb = torch.as_tensor(rng.uniform(0.0, 1.0, (n, 3)), dtype=torch.float32).cuda()
    rgbt = rgb.clone()
    rgbt[: n // 2] = torch.as_tensor(rng.uniform(0.0, 1.0, (n // 2, 3)), dtype=torch.float32).cuda()  # half equal: sign 0
    dF = torch.full_like(F, float("nan"))
    drgb = torch.full_like(rgb, float("nan"))
    loss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    p = make_params(C=Cc, K=8, feat_dtype=dtype, out_dtype=dtype)
    L.fss_loss_l2_l1(p, n, _ptr(F), _ptr(rgb), _ptr(Ft), _ptr(rgbt), wf, wc, _ptr(dF), _ptr(drgb), _ptr(loss),
                     _stream())
    torch.cuda.synchronize()
    return F, Ft, rgb, rgbt, dF, drgb, loss


@pytest.mark.parametrize("n,Cc,dtype", [(1237, 64, torch.bfloat16), (40_001, 64, torch.bfloat16),
                                        (777, 32, torch.float32), (307_200, 64, torch.bfloat16)])
def test_loss_and_gradients_match_the_definition(n, Cc, dtype):
    wf, wc = 1.0, 0.25
    F, Ft, rgb, rgbt, dF, drgb, loss = _run(n, Cc, dtype, wf, wc, seed=n)
    d = F.double().cpu().numpy() - Ft.double().cpu().numpy()
    dc = rgb.double().cpu().numpy() - rgbt.double().cpu().numpy()
    L_ref = wf * np.mean(d * d) + wc * np.mean(np.abs(dc))
    assert abs(loss.item() - L_ref) <= 1e-5 * L_ref
    # dL/dF: float64 value, rounded to FP32, then to the output type; one ulp of the output type
    g_ref = torch.as_tensor(2.0 * wf * d / (n * Cc)).float().to(dtype).float().numpy()
    g = dF.float().cpu().numpy()
    ulp = np.spacing(np.abs(g_ref).astype(np.float32)) * (2.0 ** 16 if dtype == torch.bfloat16 else 1.0)
    assert np.all(np.abs(g - g_ref) <= ulp)
    # dL/drgb: exact
    sc = np.float32(wc / np.float32(3 * n))
    np.testing.assert_array_equal(drgb.cpu().numpy(), (np.sign(dc) * sc).astype(np.float32))


def test_repeated_calls_overwrite_the_loss():
    a = _run(5000, 64, torch.bfloat16, 1.0, 1.0, seed=3)[-1].item()
    b = _run(5000, 64, torch.bfloat16, 1.0, 1.0, seed=3)[-1].item()
    assert a == pytest.approx(b, rel=1e-6) and np.isfinite(a)

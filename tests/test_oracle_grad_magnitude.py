"""Pins for the oracle's gradient magnitude chain (the tolerance scale of the
GPU gradient tests): the same chain as the analytic gradients with every
operand taken by magnitude.  It bounds each gradient entry, is positively
homogeneous in the upstream gradients, vanishes with them, and equals the
gradient's magnitude where a single term with no inner cancellation makes
up the entry."""
import numpy as np

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene

COLS = {"means": slice(0, 3), "scales": slice(3, 5), "quats": slice(5, 9), "opac": slice(9, 10)}


def _grads(sc, cam, K, gF, grgb, gT):
    p = O.make_params(K=K)
    return O.render_backward(sc, cam, p, gF, grgb, gT, binned=O.binning(sc, cam, p))


def test_magnitudes_bound_every_gradient_entry_and_scale_with_the_upstream():
    sc, cam = scenes.tiny_scene(seed=3, n=600)
    rng = np.random.default_rng(1)
    H, W = cam.height, cam.width
    gF, grgb, gT = rng.normal(size=(H, W, sc.C)), rng.normal(size=(H, W, 3)), rng.normal(size=(H, W))
    for K in (0, 4):
        g = _grads(sc, cam, K, gF, grgb, gT)
        A = g["abs"]
        assert (A >= 0).all() and A.max() > 0
        for k, c in COLS.items():
            assert (np.abs(g[k]).reshape(len(A), -1) <= A[:, c] * (1 + 1e-12) + 1e-300).all(), k
        # cancellation makes the magnitudes exceed the gradients somewhere by far
        assert (A[:, 3:5] > 10 * np.abs(g["scales"])).any()
        g3 = _grads(sc, cam, K, -3 * gF, -3 * grgb, -3 * gT)
        np.testing.assert_allclose(g3["abs"], 3 * A, rtol=1e-12, atol=1e-300)
        g0 = _grads(sc, cam, K, 0 * gF, 0 * grgb, 0 * gT)
        assert (g0["abs"] == 0).all()


def test_opacity_magnitude_is_exact_for_a_single_term():
    # one fronto-parallel surfel, upstream transmittance gradient on one pixel
    # only: dL/do = -gT T_final / (1 - alpha) * G, a single product
    cam = ident_cam(W=16, H=16, f=16.0)
    sc = make_scene([[0.0, 0.0, 2.0]], [[0.4, 0.4]], [[1, 0, 0, 0]], [0.6], C=3)
    gF = np.zeros((16, 16, 3))
    grgb = np.zeros((16, 16, 3))
    gT = np.zeros((16, 16))
    gT[8, 8] = -1.7
    g = O.render_backward(sc, cam, O.make_params(K=0), gF, grgb, gT, brute=True)
    assert g["opac"][0] != 0
    assert g["abs"][0, 9] == abs(g["opac"][0])

"""Pins for the oracle's view-dependent colour (Sec. 3.1, read as real
spherical harmonics of degree <= 3, as in the 2DGS base model): the basis
against scipy's complex spherical harmonics, orthonormality by quadrature,
its polynomial gradient by central differences, the degree-0 closed form,
and the colour gradients (coefficients and the direction term of the means)
by central differences of the whole FP64 render."""
import types

import numpy as np
import pytest
from scipy import special

import oracle as O
from paper_2604_10951_gb300 import scenes


def _dirs(n, seed=0):
    d = np.random.default_rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_basis_matches_scipy_real_harmonics():
    d = _dirs(200)
    Y, _ = O.sh_basis(3, d)
    theta, phi = np.arccos(np.clip(d[:, 2], -1, 1)), np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            c = special.sph_harm_y(l, abs(m), theta, phi)  # Condon-Shortley phase included
            if m > 0:
                want = np.sqrt(2) * (-1) ** m * c.real
            elif m < 0:
                want = np.sqrt(2) * (-1) ** m * c.imag
            else:
                want = c.real
            np.testing.assert_allclose(Y[:, l * l + l + m], want, atol=1e-12)


def test_basis_is_orthonormal_on_the_sphere():
    z, wz = np.polynomial.legendre.leggauss(16)      # exact for the degree <= 6 products
    phi = np.arange(32) * 2 * np.pi / 32               # trapezoid: exact for |frequency| < 32
    Z, P = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - Z ** 2)
    d = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(32, 2 * np.pi / 32)[None]).reshape(-1)
    Y, _ = O.sh_basis(3, d)
    np.testing.assert_allclose((Y * w[:, None]).T @ Y, np.eye(16), atol=1e-12)


def test_polynomial_gradient_by_central_differences():
    d = _dirs(20, 1) * 0.9  # the polynomials extend off the sphere
    _, G = O.sh_basis(3, d)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3); e[k] = h
        fd = (O.sh_basis(3, d + e)[0] - O.sh_basis(3, d - e)[0]) / (2 * h)
        np.testing.assert_allclose(G[:, :, k], fd, atol=1e-8)


def test_degree_zero_is_a_constant_colour_with_the_half_offset_and_clamp():
    sc, cam = scenes.tiny_scene(seed=2, n=50)
    coef = np.random.default_rng(3).normal(size=(50, 1, 3))
    rgb = O.sh_colors(coef, sc.means, cam)
    np.testing.assert_allclose(rgb, np.maximum(0.0, coef[:, 0] / (2 * np.sqrt(np.pi)) + 0.5), atol=1e-15)


def test_colour_gradients_by_central_differences():
    sc, cam = scenes.fd_subscene(seed=5)
    p = O.make_params(K=4, alpha_min=1e-8, T_min=0.0)
    rng = np.random.default_rng(4)
    sh = rng.normal(0.0, 0.3, (sc.n, 16, 3))
    s64 = types.SimpleNamespace(means=sc.means.astype(np.float64), scales=sc.scales.astype(np.float64),
                                quats=sc.quats.astype(np.float64), opacities=sc.opacities.astype(np.float64),
                                rgb=sc.rgb.astype(np.float64), feats=sc.feats.astype(np.float64))
    H, W = cam.height, cam.width
    gF, grgb = rng.normal(size=(H, W, sc.C)), rng.normal(size=(H, W, 3))

    def loss():
        out = O.render(s64, cam, p, brute=True, sh=sh)
        return (gF * out["F"]).sum() + (grgb * out["rgb"]).sum(), [out["ncontrib"], out["ids"]]

    g = O.render_backward(s64, cam, p, gF, grgb, None, brute=True, sh=sh)
    L0, st0 = loss()
    active = np.nonzero(np.abs(g["rgb"]).sum(1) > 0)[0]
    pick = rng.choice(active, 8, replace=False)
    errs, scale = [], max(np.abs(g["means"][pick]).max(), np.abs(g["sh"][pick]).max())
    for i in pick:
        for arr, name, idxs in ((s64.means, "means", [(i, k) for k in range(3)]),
                                (sh, "sh", [(i, b, c) for b in (0, 3, 8, 15) for c in range(3)])):
            for idx in idxs:
                th = arr[idx]
                h = 1e-6 * max(1.0, abs(th))
                arr[idx] = th + h
                Lp, stp = loss()
                arr[idx] = th - h
                Lm, stm = loss()
                arr[idx] = th
                if any(not np.array_equal(a, b) or not np.array_equal(a, c) for a, b, c in zip(st0, stp, stm)):
                    continue
                an = g[name][idx]
                errs.append(abs((Lp - Lm) / (2 * h) - an) / (abs(an) + 1e-4 * scale))
    assert len(errs) > 80
    assert max(errs) < 1e-6, max(errs)

"""Pins for the oracle's sensor outputs over the traversed contributors:
expected depth sum_i w_i z_i (z_i the camera depth of the ray-surfel hit),
median depth (the hit at which the transmittance first drops below 1/2, else
0) and normal sum_i w_i n_i (camera-space unit normals turned to face the
camera).  Closed forms for fronto-parallel and tilted surfels, the
two-surfel recurrence written out by hand, and bounds that hold for any scene.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene
from tests.test_oracle_composite import _fronto_alpha


def test_fronto_parallel_surfel_depth_and_normal():
    cam = ident_cam(W=24, H=20, f=24.0)
    sc = make_scene([[0.05, -0.02, 2.0]], [[0.3, 0.2]], [[1, 0, 0, 0]], [0.7], C=3)
    out = O.render(sc, cam, O.make_params(K=0), brute=True)
    p = sc.means[0].astype(float)
    for py in range(cam.height):
        for px in range(cam.width):
            a = _fronto_alpha(cam, p, sc.scales[0].astype(float), float(sc.opacities[0]), px + 0.5, py + 0.5)
            if a < 1 / 255:
                a = 0.0
            assert out["depth"][py, px] == pytest.approx(a * p[2], abs=1e-12)  # the plane z = 2
            np.testing.assert_allclose(out["normal"][py, px], [0.0, 0.0, -a], atol=1e-12)  # faces the camera
            assert out["depth_med"][py, px] == (p[2] if 1 - a < 0.5 else 0.0)


def test_surfel_seen_from_behind_still_faces_the_camera():
    cam = ident_cam(W=16, H=16, f=16.0)
    q = [0.0, 1.0, 0.0, 0.0]  # 180 degrees about x: the normal points away from the camera
    sc = make_scene([[0.0, 0.0, 2.0]], [[0.4, 0.4]], [q], [0.9], C=3)
    out = O.render(sc, cam, O.make_params(K=0), brute=True)
    a = out["depth"][8, 8] / 2.0
    assert a > 0.5
    np.testing.assert_allclose(out["normal"][8, 8], [0.0, 0.0, -a], atol=1e-12)


def test_tilted_surfel_hit_depth_matches_a_ray_plane_solve():
    cam = ident_cam(W=32, H=32, f=32.0)
    th = 0.6  # rotation about y
    sc = make_scene([[0.1, -0.05, 2.5]], [[0.5, 0.3]], [[np.cos(th / 2), 0.0, np.sin(th / 2), 0.0]], [0.8], C=3)
    out = O.render(sc, cam, O.make_params(K=0), brute=True)
    c = sc.means[0].astype(float)
    qw, qx, qy, qz = (sc.quats[0].astype(float) / np.linalg.norm(sc.quats[0].astype(float)))
    n = np.array([2 * (qx * qz + qw * qy), 2 * (qy * qz - qw * qx), 1 - 2 * (qx * qx + qy * qy)])  # R(q) e3
    n_face = -n if n @ c > 0 else n
    for py, px in [(16, 16), (14, 18), (17, 12)]:
        d = np.array([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy, 1.0])
        lam = (n @ c) / (n @ d)  # ray x = lam d meets the plane n.(x - c) = 0
        a = 1.0 - out["T"][py, px]
        assert a > 0
        assert out["depth"][py, px] == pytest.approx(a * lam * d[2], rel=1e-10)
        np.testing.assert_allclose(out["normal"][py, px], a * n_face, atol=1e-12)


def test_two_surfels_by_hand():
    cam = ident_cam(W=8, H=8, f=8.0)
    means = [[0.0, 0.0, 3.0], [0.02, 0.01, 2.0]]  # the second is nearer
    sc = make_scene(means, [[0.5, 0.4], [0.3, 0.6]], [[1, 0, 0, 0]] * 2, [0.6, 0.8], C=3)
    out = O.render(sc, cam, O.make_params(K=0), brute=True)
    x, y = 4.5, 3.5
    a_far = _fronto_alpha(cam, sc.means[0].astype(float), sc.scales[0].astype(float), float(sc.opacities[0]), x, y)
    a_near = _fronto_alpha(cam, sc.means[1].astype(float), sc.scales[1].astype(float), float(sc.opacities[1]), x, y)
    w_near, w_far = a_near, a_far * (1 - a_near)
    z_near, z_far = float(sc.means[1][2]), float(sc.means[0][2])
    assert out["depth"][3, 4] == pytest.approx(w_near * z_near + w_far * z_far, abs=1e-13)
    med = z_near if 1 - a_near < 0.5 else (z_far if (1 - a_near) * (1 - a_far) < 0.5 else 0.0)
    assert out["depth_med"][3, 4] == med
    np.testing.assert_allclose(out["normal"][3, 4], [0, 0, -(w_near + w_far)], atol=1e-13)


def test_bounds_on_a_random_scene():
    sc, cam = scenes.tiny_scene(seed=8, n=1500)
    out = O.render(sc, cam, O.make_params(K=4))
    acc = 1.0 - out["T"]
    # |sum w n| <= sum w = 1 - T (unit normals); every normal faces the camera
    assert np.all(np.linalg.norm(out["normal"], axis=-1) <= acc + 1e-12)
    pc_dir = np.stack(np.meshgrid((np.arange(cam.width) + 0.5 - cam.cx) / cam.fx,
                                  (np.arange(cam.height) + 0.5 - cam.cy) / cam.fy), -1)
    ray = np.concatenate([pc_dir, np.ones(pc_dir.shape[:2] + (1,))], -1)
    assert np.all(np.sum(out["normal"] * ray, -1) <= 1e-12)
    # depths: positive hits beyond the near plane; the median is 0 exactly where T stays >= 1/2
    assert np.all(out["depth"] >= 0.2 * acc - 1e-12)
    np.testing.assert_array_equal(out["depth_med"] == 0.0, out["T"] >= 0.5)

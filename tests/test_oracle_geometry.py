"""Pins for the oracle's surfel geometry and ray-splat intersection.

Each check is independent of the oracle's own formulas: scipy's rotation
fixes the quaternion convention, a world-space ray-plane solve fixes the
intersection, and the fronto-parallel case reduces to similar triangles.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2604_10951_gb300 import scenes
from tests._scenes import ident_cam, make_scene


def _rot(q_wxyz):
    w, x, y, z = q_wxyz
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def test_identity_quaternion_frame_gives_axis_aligned_homography():
    # Eq. 1 with t_u = x, t_v = y: T = K [r_u e1 | r_v e2 | p_c]
    cam = ident_cam(W=64, H=48, f=50.0, cx=30.0, cy=20.0)
    sc = make_scene([[0.3, -0.2, 2.5]], [[0.1, 0.05]], [[1, 0, 0, 0]], [0.8])
    T, z, ca, ok = O.geometry(sc, cam, O.make_params())
    p = np.array([0.3, -0.2, 2.5], dtype=np.float32).astype(np.float64)
    ru, rv = float(np.float32(0.1)), float(np.float32(0.05))
    expect = np.array([[50.0 * ru, 0.0, 50.0 * p[0] + 30.0 * p[2]],
                       [0.0, 50.0 * rv, 50.0 * p[1] + 20.0 * p[2]],
                       [0.0, 0.0, p[2]]])
    np.testing.assert_allclose(T[0], expect, rtol=1e-14, atol=1e-14)
    assert z[0] == pytest.approx(p[2], rel=1e-15)
    assert ca[0] == pytest.approx(p[2] / np.linalg.norm(p), rel=1e-12)  # normal . ray to centre
    assert ok[0] == 1


def _ray_plane(cam, mean, scale, quat, x, y):
    """World-space intersection of the pixel ray with the surfel plane."""
    vm = np.asarray(cam.viewmat, np.float64)
    R, t = vm[:, :3], vm[:, 3]
    Kinv = np.linalg.inv(np.array([[cam.fx, 0, cam.cx], [0, cam.fy, cam.cy], [0, 0, 1.0]]))
    Rinv = np.linalg.inv(R)  # the binary32 view rotation is only orthonormal to ~1e-7
    d = Rinv @ (Kinv @ np.array([x, y, 1.0]))
    o = -Rinv @ t
    Rs = _rot(np.asarray(quat, np.float64) / np.linalg.norm(quat))
    tu, tv, n = Rs[:, 0], Rs[:, 1], Rs[:, 2]
    p = np.asarray(mean, np.float64)
    lam = n @ (p - o) / (n @ d)
    X = o + lam * d
    u = tu @ (X - p) / scale[0]
    v = tv @ (X - p) / scale[1]
    zhit = (R @ X + t)[2]
    return u, v, zhit


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ray_splat_matches_world_space_ray_plane_solve(seed):
    rng = np.random.default_rng(seed)
    cams = scenes.circle_poses(4, 96, 64, 80.0)
    for cam in cams:
        n = 20
        means = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
        fwd = np.linalg.inv(np.asarray(cam.viewmat)[:, :3]) @ np.array([0, 0, 1.0])
        campos = -np.asarray(cam.viewmat)[:, :3].T @ np.asarray(cam.viewmat)[:, 3]
        means = (campos + 2.5 * fwd + 0.4 * means).astype(np.float32)
        scales = rng.uniform(0.02, 0.3, (n, 2)).astype(np.float32)
        quats = rng.normal(size=(n, 4)).astype(np.float32)
        sc = make_scene(means, scales, quats, np.full(n, 0.5))
        T, z, ca, ok = O.geometry(sc, cam, O.make_params())
        xy = np.stack([rng.uniform(0, cam.width, 16), rng.uniform(0, cam.height, 16)], 1)
        for i in range(n):
            if abs(ca[i]) < 0.05:
                continue
            uvz, valid = O.ray_splat(T[i], xy)
            for k in range(len(xy)):
                u, v, zh = _ray_plane(cam, sc.means[i], sc.scales[i], sc.quats[i], *xy[k])
                assert valid[k] == 1
                scale = 1.0 + abs(u) + abs(v)
                assert uvz[k, 0] == pytest.approx(u, abs=1e-9 * scale)
                assert uvz[k, 1] == pytest.approx(v, abs=1e-9 * scale)
                assert uvz[k, 2] == pytest.approx(zh, rel=1e-9)


def test_fronto_parallel_intersection_closed_form():
    # u = ((x - cx) d / fx - p_x) / r_u for a surfel facing the camera at depth d
    cam = ident_cam(W=40, H=40, f=40.0)
    d = 2.0
    sc = make_scene([[0.1, -0.05, d]], [[0.2, 0.1]], [[1, 0, 0, 0]], [0.9])
    T, *_ = O.geometry(sc, cam, O.make_params())
    xs = np.array([[3.5, 7.5], [20.5, 20.5], [39.5, 0.5]])
    uvz, valid = O.ray_splat(T[0], xs)
    p = sc.means[0].astype(np.float64)
    r = sc.scales[0].astype(np.float64)
    for k, (x, y) in enumerate(xs):
        assert uvz[k, 0] == pytest.approx(((x - 20.0) * d / 40.0 - p[0]) / r[0], rel=1e-12, abs=1e-12)
        assert uvz[k, 1] == pytest.approx(((y - 20.0) * d / 40.0 - p[1]) / r[1], rel=1e-12, abs=1e-12)
        assert uvz[k, 2] == pytest.approx(d, rel=1e-12)


def test_hit_behind_near_plane_is_invalid():
    # a surfel tilted so that part of its plane lies behind the near plane
    cam = ident_cam(W=32, H=32, f=32.0, near=1.0)
    q = np.array([np.cos(0.6), np.sin(0.6), 0, 0])  # rotate about x
    sc = make_scene([[0.0, 0.0, 1.2]], [[0.5, 0.5]], [q], [0.9])
    T, *_ = O.geometry(sc, cam, O.make_params())
    ys = np.linspace(0.5, 31.5, 32)
    uvz, valid = O.ray_splat(T[0], np.stack([np.full(32, 16.5), ys], 1), near=1.0)
    zh = uvz[:, 2]
    assert np.all((zh > 1.0) == (valid == 1))
    assert valid.min() == 0 and valid.max() == 1


def test_edge_on_surfel_is_culled():
    # normal perpendicular to the viewing ray through the centre (Sec. 3.1 normal)
    cam = ident_cam()
    q = Rotation.from_euler("y", 90, degrees=True).as_quat()  # x,y,z,w
    sc = make_scene([[0.0, 0.0, 3.0]], [[0.2, 0.2]], [[q[3], q[0], q[1], q[2]]], [0.9])
    T, z, ca, ok = O.geometry(sc, cam, O.make_params())
    assert abs(ca[0]) < 1e-6 and ok[0] == 0
    rec, reci, cnt = O.mirror_project(sc, cam, O.make_params())
    assert reci[0, 1] == 1 and cnt[0] == 0
    r = O.render(sc, cam, O.make_params(K=2, C=4), brute=True)
    assert np.all(r["T"] == 1.0) and np.all(r["F"] == 0.0)

"""Seeded synthetic scenes and pinhole cameras for the 2DGS feature rasterizer.

This module only draws inputs: surfel parameters, per-surfel features and
cameras.  It holds none of the renderer's arithmetic (no projection, no
blending, no selection), so the CUDA library and the FP64 checker can both
consume what it produces without sharing any of the method.

The paper measures on ScanNet-V2 / ScanNet++ rooms reconstructed with a
surfel model (Sec. 4.1, its dataset and implementation paragraphs).  Those
scenes are not available here; the room generator below stands in for them
with the same structure: thin surfels lying on the surfaces of a closed
indoor room plus compact objects, Kinect-like 640x480 intrinsics, and
clustered semantic features (Sec. 3.4 feature dimensions 16/32, generalised
to C = 16..128).

Conventions (shared by every consumer of these arrays):
  * camera: OpenCV pinhole, x right, y down, z forward; ``viewmat`` is the
    3x4 row-major world->camera [R | t];
  * quaternions are (w, x, y, z), not necessarily unit length;
  * ``scales`` = exp(``log_scales``) and ``opacities`` = sigmoid(logits) are
    provided pre-activated in float32 for the C-ABI, which takes activated
    parameters; the autograd wrapper activates the raw ones itself.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "Camera",
    "Scene",
    "tiny_scene",
    "room_scene",
    "circle_poses",
    "fd_subscene",
    "batched_cameras",
    "look_at",
    "save_scene",
    "load_scene",
]


@dataclasses.dataclass
class Camera:
    """Pinhole camera; pixel (px, py) has its centre at (px + 0.5, py + 0.5)."""

    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    viewmat: np.ndarray  # (3, 4) float32, world -> camera
    near: float = 0.2

    def __post_init__(self):
        self.viewmat = np.ascontiguousarray(np.asarray(self.viewmat, dtype=np.float32).reshape(3, 4))


@dataclasses.dataclass
class Scene:
    means: np.ndarray          # (N, 3) f32
    log_scales: np.ndarray     # (N, 2) f32
    quats: np.ndarray          # (N, 4) f32, (w, x, y, z)
    opacity_logits: np.ndarray # (N,)  f32
    rgb: np.ndarray            # (N, 3) f32 in [0, 1]
    feats: np.ndarray          # (N, C) f32
    scales: np.ndarray = None  # (N, 2) f32 = exp(log_scales)
    opacities: np.ndarray = None  # (N,) f32 = sigmoid(opacity_logits)

    def __post_init__(self):
        f32 = np.float32
        self.means = np.ascontiguousarray(self.means, dtype=f32)
        self.log_scales = np.ascontiguousarray(self.log_scales, dtype=f32)
        self.quats = np.ascontiguousarray(self.quats, dtype=f32)
        self.opacity_logits = np.ascontiguousarray(self.opacity_logits, dtype=f32)
        self.rgb = np.ascontiguousarray(self.rgb, dtype=f32)
        self.feats = np.ascontiguousarray(self.feats, dtype=f32)
        if self.scales is None:
            self.scales = np.exp(self.log_scales).astype(f32)
        if self.opacities is None:
            self.opacities = (f32(1.0) / (f32(1.0) + np.exp(-self.opacity_logits))).astype(f32)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def C(self) -> int:
        return int(self.feats.shape[1])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx], self.log_scales[idx], self.quats[idx],
                     self.opacity_logits[idx], self.rgb[idx], self.feats[idx],
                     self.scales[idx], self.opacities[idx])


# --------------------------------------------------------------------------
# small quaternion / pose helpers used only to *place* inputs
# --------------------------------------------------------------------------

def _random_unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (Shoemake's subgroup algorithm)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=1)
    return q


def _quat_mul(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Hamilton product of (w, x, y, z) quaternions, row-wise."""
    pw, px, py, pz = p.T
    qw, qx, qy, qz = q.T
    return np.stack([pw * qw - px * qx - py * qy - pz * qz,
                     pw * qx + px * qw + py * qz - pz * qy,
                     pw * qy - px * qz + py * qw + pz * qx,
                     pw * qz + px * qy - py * qx + pz * qw], axis=1)


def _quats_with_normal(rng: np.random.Generator, normals: np.ndarray) -> np.ndarray:
    """Quaternions whose rotation takes local +z to ``normals`` (unit rows),
    followed by a uniformly random spin about that normal, so the surfel's
    tangent plane lies in the surface."""
    n = normals / np.linalg.norm(normals, axis=1, keepdims=True)
    # shortest-arc rotation e_z -> n : (1 + n_z, e_z x n) normalised
    q_align = np.stack([1.0 + n[:, 2], -n[:, 1], n[:, 0], np.zeros(len(n))], axis=1)
    flip = q_align[:, 0] < 1e-9          # n == -e_z: half turn about x
    q_align[flip] = np.array([0.0, 1.0, 0.0, 0.0])
    q_align /= np.linalg.norm(q_align, axis=1, keepdims=True)
    phi = rng.uniform(0.0, 2.0 * np.pi, len(n))
    q_spin = np.stack([np.cos(phi / 2), np.zeros(len(n)), np.zeros(len(n)), np.sin(phi / 2)], axis=1)
    return _quat_mul(q_align, q_spin)


def look_at(position, forward, width, height, fx, fy=None, cx=None, cy=None, near=0.2) -> Camera:
    """OpenCV-convention camera at ``position`` looking along ``forward``
    with world +y as the image's down direction."""
    c = np.asarray(position, dtype=np.float64)
    f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    r = np.cross(down, f)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], axis=0)
    t = -R @ c
    vm = np.concatenate([R, t[:, None]], axis=1)
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    return Camera(float(fx), float(fy), float(cx), float(cy), int(width), int(height), vm, near)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------

def tiny_scene(seed: int = 0, n: int = 2000, C: int = 16):
    """2,000 surfels, means U[-1,1]^3, log-scales N(-3, 0.5), uniform random
    rotations, opacity sigmoid(N(0,1)), features N(0,1), RGB U[0,1]; one
    128x128 camera (fx=fy=128, c=64) at (0,0,-3) looking +z."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    log_scales = rng.normal(-3.0, 0.5, (n, 2))
    quats = _random_unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n)
    feats = rng.normal(0.0, 1.0, (n, C))
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    scene = Scene(means, log_scales, quats, logits, rgb, feats)
    vm = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3.0]], dtype=np.float32)
    cam = Camera(128.0, 128.0, 64.0, 64.0, 128, 128, vm)
    return scene, cam


ROOM_HALF = np.array([3.0, 1.5, 2.5])   # room box x in [-3,3], y in [-1.5,1.5] (y down), z in [-2.5,2.5]
CAM_CIRCLE_R = 1.0


def _room_walls():
    """(axis, sign, span axes, area) for the 6 inner faces of the room box."""
    walls = []
    for axis in range(3):
        others = [a for a in range(3) if a != axis]
        area = (2 * ROOM_HALF[others[0]]) * (2 * ROOM_HALF[others[1]])
        for sign in (-1.0, 1.0):
            walls.append((axis, sign, others, area))
    return walls


def room_scene(n: int = 500_000, C: int = 64, seed: int = 1, n_blobs: int = 40,
               wall_fraction: float = 0.85):
    """Indoor room stand-in: 85% of surfels on the 6 inner walls of a
    6 x 3 x 5 m box (in proportion to area, normals along the wall normal,
    2 mm normal jitter), 15% on ``n_blobs`` sphere/ellipsoid objects with
    surface-aligned normals; log-scales N(-4.5, 0.6), opacity
    sigmoid(N(1, 1.5)); features = one of 40 cluster centres ~N(0,1)^C plus
    N(0, 0.1) noise (walls -> clusters 0..5, blob b -> b mod 40); RGB a
    per-cluster base U[0,1]^3 plus N(0, 0.05), clipped."""
    rng = np.random.default_rng(seed)
    n_wall = int(round(wall_fraction * n))
    n_blob = n - n_wall
    walls = _room_walls()
    areas = np.array([w[3] for w in walls])
    per_wall = rng.multinomial(n_wall, areas / areas.sum())

    means, normals, cluster = [], [], []
    for wi, ((axis, sign, others, _), k) in enumerate(zip(walls, per_wall)):
        p = np.zeros((k, 3))
        p[:, axis] = sign * ROOM_HALF[axis] + rng.normal(0.0, 0.002, k)
        for a in others:
            p[:, a] = rng.uniform(-ROOM_HALF[a], ROOM_HALF[a], k)
        nrm = np.zeros((k, 3))
        nrm[:, axis] = -sign                    # inward normal
        means.append(p); normals.append(nrm); cluster.append(np.full(k, wi))

    # object blobs: centres kept away from walls and from the camera circle
    per_blob = rng.multinomial(n_blob, np.full(n_blobs, 1.0 / n_blobs))
    for b in range(n_blobs):
        if rng.random() < 0.5:
            radii = np.full(3, rng.uniform(0.15, 0.5))
        else:
            radii = rng.uniform(0.15, 0.5, 3)
        margin = 0.5 + radii.max()
        for _ in range(10_000):
            c = rng.uniform(-ROOM_HALF + margin, ROOM_HALF - margin) if np.all(ROOM_HALF > margin) else np.zeros(3)
            ring = math.hypot(math.hypot(c[0], c[2]) - CAM_CIRCLE_R, c[1])
            if ring >= margin:
                break
        k = per_blob[b]
        d = rng.normal(size=(k, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        means.append(c + d * radii)
        normals.append(d / radii)
        cluster.append(np.full(k, b % 40))

    means = np.concatenate(means)
    normals = np.concatenate(normals)
    cluster = np.concatenate(cluster).astype(np.int64)
    quats = _quats_with_normal(rng, normals)
    log_scales = rng.normal(-4.5, 0.6, (n, 2))
    logits = rng.normal(1.0, 1.5, n)
    centres = rng.normal(0.0, 1.0, (40, C))
    feats = centres[cluster] + rng.normal(0.0, 0.1, (n, C))
    base_rgb = rng.uniform(0.0, 1.0, (40, 3))
    rgb = np.clip(base_rgb[cluster] + rng.normal(0.0, 0.05, (n, 3)), 0.0, 1.0)
    perm = rng.permutation(n)            # no spatial order in the input
    return Scene(means[perm], log_scales[perm], quats[perm], logits[perm], rgb[perm], feats[perm])


def room_queries(means: np.ndarray, n_queries: int = 32, dim: int = 32, seed: int = 0):
    """Inputs of the query-guided instance labels (Sec. 3.3) for Gaussians at
    ``means``: ``n_queries`` instance queries with centres uniform in the
    room (0.5 m from the walls), Gaussian extents with per-axis standard
    deviations U[0.4, 1.2] m under a uniform random rotation (given as the
    precision matrix entries xx, yy, zz, xy, xz, yz), and ``dim``-d query
    features 3 c_q with c_q ~ N(0, 1/dim); each scene Gaussian takes the
    nearest query centre as its instance, and its instance feature is that
    query's feature plus N(0, 0.3^2 / dim) noise.  Returns float32 arrays
    (f_ins [N, dim], f_q [nq, dim], p_q [nq, 3], prec [nq, 6])."""
    rng = np.random.default_rng(seed)
    p_q = rng.uniform(-ROOM_HALF + 0.5, ROOM_HALF - 0.5, (n_queries, 3))
    sig = rng.uniform(0.4, 1.2, (n_queries, 3))
    q = _random_unit_quats(rng, n_queries)
    w, x, y, z = q.T
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                  np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                  np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    Pm = np.einsum("qab,qb,qcb->qac", R, 1.0 / sig ** 2, R)
    prec = np.stack([Pm[:, 0, 0], Pm[:, 1, 1], Pm[:, 2, 2], Pm[:, 0, 1], Pm[:, 0, 2], Pm[:, 1, 2]], -1)
    f_q = 3.0 * rng.normal(0.0, 1.0 / math.sqrt(dim), (n_queries, dim))
    m = np.asarray(means, np.float64)
    inst = np.empty(m.shape[0], np.int64)
    for a in range(0, m.shape[0], 65536):
        d2 = ((m[a:a + 65536, None, :] - p_q[None]) ** 2).sum(-1)
        inst[a:a + 65536] = d2.argmin(1)
    f_ins = f_q[inst] + rng.normal(0.0, 0.3 / math.sqrt(dim), (m.shape[0], dim))
    return (f_ins.astype(np.float32), f_q.astype(np.float32), p_q.astype(np.float32), prec.astype(np.float32))


def circle_poses(n_poses: int = 16, width: int = 640, height: int = 480, f: float = 525.0,
                 radius: float = CAM_CIRCLE_R, yaw_offset_deg: float = 30.0,
                 pitch_deg: float = 10.0) -> List[Camera]:
    """Cameras on a horizontal circle of ``radius`` at mid-height (y = 0),
    yaw 2*pi*k/n, looking outward with a 30 deg tangential turn and a 10 deg
    downward pitch."""
    cams = []
    for k in range(n_poses):
        th = 2.0 * np.pi * k / n_poses
        pos = np.array([radius * np.cos(th), 0.0, radius * np.sin(th)])
        yaw = th + np.deg2rad(yaw_offset_deg)
        pitch = np.deg2rad(pitch_deg)
        fwd = np.array([np.cos(pitch) * np.cos(yaw), np.sin(pitch), np.cos(pitch) * np.sin(yaw)])
        cams.append(look_at(pos, fwd, width, height, f))
    return cams


def fd_subscene(seed: int = 5, n: int = 200, C: int = 8):
    """200 surfels drawn like the tiny scene in a [-0.5, 0.5]^3 box centred
    3 m in front of a 32x32 camera (fx=fy=32, c=16) at the origin."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.5, 0.5, (n, 3)) + np.array([0.0, 0.0, 3.0])
    log_scales = rng.normal(-3.0, 0.5, (n, 2))
    quats = _random_unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n)
    feats = rng.normal(0.0, 1.0, (n, C))
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    scene = Scene(means, log_scales, quats, logits, rgb, feats)
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    cam = Camera(32.0, 32.0, 16.0, 16.0, 32, 32, vm)
    return scene, cam


def batched_cameras(sizes=((320, 240, 262.5), (640, 480, 525.0), (1280, 720, 900.0)),
                    per_size: int = 4) -> List[Camera]:
    """Mixed-resolution views spread over the camera circle: ``per_size``
    views of each (width, height, focal) triple, interleaved."""
    n = per_size * len(sizes)
    out = []
    for k in range(n):
        w, h, f = sizes[k % len(sizes)]
        th = 2.0 * np.pi * k / n
        pos = np.array([CAM_CIRCLE_R * np.cos(th), 0.0, CAM_CIRCLE_R * np.sin(th)])
        yaw = th + np.deg2rad(30.0)
        pitch = np.deg2rad(10.0)
        fwd = np.array([np.cos(pitch) * np.cos(yaw), np.sin(pitch), np.cos(pitch) * np.sin(yaw)])
        out.append(look_at(pos, fwd, w, h, f))
    return out


def targets(seed: int, n_pixels: int, C: int):
    """Per-pixel random targets for the L2-feature + L1-RGB loss:
    F_tgt ~ N(0, 1), rgb_tgt ~ U[0, 1]."""
    rng = np.random.default_rng(seed)
    return (rng.normal(0.0, 1.0, (n_pixels, C)).astype(np.float32),
            rng.uniform(0.0, 1.0, (n_pixels, 3)).astype(np.float32))


def save_scene(path: str, scene: Scene, cams: Optional[List[Camera]] = None) -> None:
    """Write a scene (and optionally cameras) to an ``.npz`` file."""
    d = {f.name: getattr(scene, f.name) for f in dataclasses.fields(scene)}
    if cams:
        d["cam_intr"] = np.array([[c.fx, c.fy, c.cx, c.cy, c.width, c.height, c.near] for c in cams])
        d["cam_view"] = np.stack([c.viewmat for c in cams])
    np.savez(path, **d)


def load_scene(path: str):
    """Inverse of :func:`save_scene`; returns (scene, cameras or None)."""
    z = np.load(path)
    scene = Scene(*(z[f.name] for f in dataclasses.fields(Scene)))
    cams = None
    if "cam_intr" in z:
        cams = [Camera(i[0], i[1], i[2], i[3], int(i[4]), int(i[5]), v, float(i[6]))
                for i, v in zip(z["cam_intr"], z["cam_view"])]
    return scene, cams

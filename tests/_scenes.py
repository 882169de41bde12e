"""Small hand-built scenes for closed-form checks (test helper)."""
import numpy as np

from paper_2604_10951_gb300.scenes import Camera, Scene


def ident_cam(W=32, H=32, f=32.0, cx=None, cy=None, near=0.2):
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    return Camera(f, f, W / 2 if cx is None else cx, H / 2 if cy is None else cy, W, H, vm, near)


def make_scene(means, scales, quats, opac, rgb=None, feats=None, C=4, seed=0):
    rng = np.random.default_rng(seed)
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    scales = np.asarray(scales, np.float32).reshape(n, 2)
    quats = np.asarray(quats, np.float32).reshape(n, 4)
    opac = np.asarray(opac, np.float32).reshape(n)
    rgb = rng.uniform(0, 1, (n, 3)).astype(np.float32) if rgb is None else np.asarray(rgb, np.float32)
    feats = rng.normal(0, 1, (n, C)).astype(np.float32) if feats is None else np.asarray(feats, np.float32)
    with np.errstate(divide="ignore"):
        return Scene(means, np.log(scales), quats, np.log(opac) - np.log1p(-opac), rgb, feats,
                     scales=scales, opacities=opac)

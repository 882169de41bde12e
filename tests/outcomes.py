"""Two-outcome parity at borderline pixels (test helper).

Where a discrete decision of Eq. 2 or Eq. 7 (skip below alpha_min, the near
plane, the T_min stop, the exact Top-K stop, the K-th place of the Top-K
set) is taken within rounding distance of its threshold, a binary32
evaluation may take it either way and both results are correct.  Instead of
leaving such pixels out, the comparison asks the oracle for the other
outcomes (its per-pixel flip masks) and requires the GPU's result to equal
one of them at the same tolerances as every other pixel.  Pixels that match
no outcome are counted; their share is capped at 0.1 %.

The matched outcome of each pixel is returned as a flip mask, so that the
oracle's backward can differentiate the function the GPU evaluated.
"""
import numpy as np

import oracle as O

MAX_UNMATCHED = 1e-3  # share of pixels that may match none of the outcomes
MAX_FLIP = 15         # flip masks tried: every combination of the first four borderline decisions


def scale_of(scene, cam, params, binned, feats=None, sh=None, flip=None, only=None):
    """S(x, ch) = sum over the accumulated set of w_i |c_i,ch| + 1e-6."""
    f = scene.feats if feats is None else feats
    out = O.render(scene, cam, params, feats=np.abs(np.asarray(f, np.float64)), binned=binned, sh=sh,
                   flip=flip, only=only)
    return out["F"] + 1e-6


def pixel_match(g, ref, S, tol, K, rgb_atol=2e-5, T_atol=2e-5, T_rtol=1e-4):
    """Per pixel: True where the GPU outputs equal the reference at the
    tolerances of the parity tests (features within tol * S, colour and T
    absolute, ids, list positions and traversal lengths exactly)."""
    ok = (np.abs(g["F"] - ref["F"]) <= tol * S).all(axis=-1)
    ok &= (np.abs(g["rgb"] - ref["rgb"]) <= rgb_atol).all(axis=-1)
    ok &= np.abs(g["T"] - ref["T"]) <= T_atol + T_rtol * np.abs(ref["T"])
    if K:
        if "ids" in g:
            ok &= (g["ids"] == ref["ids"]).all(axis=-1)
        if "pos" in g:
            ok &= (g["pos"] == ref["pos"]).all(axis=-1)
        if "nstop" in g:
            ok &= g["nstop"] == ref["nstop"]
    return ok


MERGED = ("F", "rgb", "T", "ids", "pos", "w", "nstop", "ncontrib", "depth", "depth_med", "normal")


def resolve(g, scene, cam, params, binned, tol, K, feats=None, sh=None, ref=None, S=None, match=pixel_match):
    """Reference outputs with, at each borderline pixel, the outcome the GPU
    took.  Returns (ref, S, flip, unmatched, stats): ``ref`` the oracle's
    outputs merged over the matched outcomes, ``S`` the tolerance scale of
    those outcomes, ``flip`` the per-pixel flip mask of the matched outcome
    (0 at ordinary pixels), ``unmatched`` the borderline pixels equal to no
    outcome, and ``stats`` the counts.  Ordinary pixels have one outcome
    only; the caller checks them like every other pixel outside
    ``unmatched``."""
    if ref is None:
        ref = O.render(scene, cam, params, feats=feats, binned=binned, sh=sh)
    if S is None:
        S = scale_of(scene, cam, params, binned, feats=feats, sh=sh)
    ref = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in ref.items()}
    S = S.copy()
    border = ref["nborder"] > 0
    ok = match(g, ref, S, tol, K)
    flip = np.zeros(ref["T"].shape, np.uint32)
    todo = border & ~ok
    plain_border_ok = int((border & ok).sum())
    for m in range(1, MAX_FLIP + 1):
        if not todo.any():
            break
        fl = np.where(todo, np.uint32(m), np.uint32(0))
        alt = O.render(scene, cam, params, feats=feats, binned=binned, sh=sh, flip=fl, only=todo)
        S_alt = scale_of(scene, cam, params, binned, feats=feats, sh=sh, flip=fl, only=todo)
        hit = todo & match(g, alt, S_alt, tol, K)
        for k in MERGED:
            if k in ref and k in alt:
                ref[k][hit] = alt[k][hit]
        S[hit] = S_alt[hit]
        flip[hit] = m
        todo &= ~hit
    unmatched = todo
    stats = dict(pixels=int(ok.size), border=int(border.sum()), plain=plain_border_ok,
                 flipped=int((flip > 0).sum()), unmatched=int(unmatched.sum()))
    return ref, S, flip, unmatched, stats


def oracle_ref(scene, cam, params, binned=None, feats=None, sh=None):
    """The oracle's plain outputs and tolerance scale, carrying what
    :func:`settle` needs to render the other outcomes."""
    if binned is None:
        binned = O.binning(scene, cam, params)
    ref = O.render(scene, cam, params, feats=feats, binned=binned, sh=sh)
    S = scale_of(scene, cam, params, binned, feats=feats, sh=sh)
    ref["_ctx"] = dict(scene=scene, cam=cam, params=params, binned=binned, feats=feats, sh=sh)
    return ref, S


def settle(g, ref, S, tol, K, match=pixel_match):
    """Resolve the borderline pixels of ``g`` against the outcomes of an
    :func:`oracle_ref` result, in place: ``ref`` and ``S`` then hold the
    outcome the GPU took at every matched pixel, ``ref["flip"]`` its flip
    mask (for the oracle's backward), ``ref["unmatched"]`` the borderline
    pixels equal to no outcome (at most 0.1 % of the pixels, asserted) and
    ``ref["outcomes"]`` the counts.  Returns the pixels to compare: all but
    the unmatched ones."""
    c = ref["_ctx"]
    merged, S2, flip, unmatched, stats = resolve(g, c["scene"], c["cam"], c["params"], c["binned"], tol, K,
                                                 feats=c["feats"], sh=c["sh"], ref=ref, S=S, match=match)
    for k in MERGED:
        if k in ref:
            ref[k][...] = merged[k]
    S[...] = S2
    ref["flip"], ref["unmatched"], ref["outcomes"] = flip, unmatched, stats
    assert unmatched.mean() <= MAX_UNMATCHED, stats
    return ~unmatched


def upstream_mask(ref, extra_flags=0):
    """Pixels whose upstream gradient the gradient tests zero: the unmatched
    borderline pixels, and pixels with a decision that leaves the forward
    values continuous but switches the derivative (alpha within rounding
    distance of the alpha_max clamp, and ``extra_flags``), where the
    forward cannot tell which side the GPU took."""
    return ref["unmatched"] | ((ref["flags"] & (O.FLAG_CLAMP | extra_flags)) != 0)

"""Tolerances of the image comparisons against the FP64 oracle (shared by the GPU tests).

Exact mode: |GPU - oracle| <= 2e-4 per channel on every pixel. The only extra
allowance is the colour jump of a skip (alpha < 1/255) or stop (T < 1e-4)
decision that lies within single-precision rounding of its threshold, where
FP32 and FP64 may rightly decide differently (diag[1] + diag[2] of the
oracle); the share of pixels that carry such a flag is reported and bounded.

RoofGS mode: within eps_max = 0.0312 (the measured bound of Eq. (24)) + 2e-4 +
FP16 colour rounding of the oracle with exact exp, with the same flip
allowance. The tighter supplementary check against the oracle that evaluates
Eq. (24) itself in FP32 also allows the oracle's first-order FP32 estimate of
the exponent's rounding (diag[0]): RoofGS evaluates the folded polynomial of
Eqs. (13)-(16) from a single-precision projected mean, as the paper does.
"""
from __future__ import annotations

import numpy as np

import oracle

TOL = 2e-4
HALF_COLOUR = 2.0 ** -12  # FP16 rounding of a colour in [0, 1] (RoofGS raster record)
# RoofGS mode's flip windows are wider (its exponent carries the FP32 rounding of the
# projected mean): a larger share of pixels may carry a flag
ROOFGS_FLAGGED = 0.1


def flips(diag):
    return diag[..., 1] + diag[..., 2]


def fp32_estimate(diag):
    return 4.0 * diag[..., 0]


def allowance(diag, fp32=False):
    return flips(diag) + (fp32_estimate(diag) if fp32 else 0.0)


def check(img, ref, diag, base, fp32=False, mask=None, max_flagged=0.01, label=""):
    """Every value within base + allowance; the share of pixels that carry a threshold
    flag at most max_flagged. mask selects the compared pixels ([H, W] bool)."""
    if mask is None:
        mask = ~np.isnan(ref[0])
    allow = allowance(diag, fp32)[mask]
    flag = flips(diag)[mask] > 0
    err = np.abs(img - ref)[:, mask]
    tol = base + allow
    bad = err > tol[None]
    flagged = float(np.mean(flag)) if flag.size else 0.0
    over = float(np.mean((err > base).any(axis=0))) if err.size else 0.0
    unflagged = err[:, ~flag]
    print("%s: max |err| %.3g, unflagged max %.3g, pixels over %.3g: %.5f, flagged %.5f" % (
        label, float(err.max()) if err.size else 0.0, float(unflagged.max()) if unflagged.size else 0.0, base, over,
        flagged))
    assert not bad.any(), "%s: %d values over tolerance, worst excess %.3g" % (
        label, int(bad.sum()), float((err - tol[None]).max()))
    assert flagged <= max_flagged, "%s: %.4f of the pixels carry a threshold flag" % (label, flagged)
    return float(err.max()) if err.size else 0.0, flagged


def tile_mask(cam, tiles, tile=(16, 16)):
    lay = oracle.layout(cam, tile)
    m = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        tx, ty = t % lay["tiles_x"], t // lay["tiles_x"]
        m[ty * tile[1]:(ty + 1) * tile[1], tx * tile[0]:(tx + 1) * tile[0]] = True
    return m


def sample_tiles(cam, k, seed, tile=(16, 16)):
    lay = oracle.layout(cam, tile)
    nt = lay["tiles_x"] * lay["tiles_y"]
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(nt, size=min(k, nt), replace=False)).astype(np.int32)


def check_view(img, scene, cam, mode, tile=(16, 16), tiles=None, comp=None, max_flagged=0.02, label=""):
    """One rendered view (float64 [3, H, W]) against the oracle on the listed tiles (all if None):
    exact mode at 2e-4; RoofGS mode within the fast-exp bound of the exact-exp oracle and
    within 2e-4 + FP16 colour (+ FP32 estimate) of the FP32 fast-exp oracle."""
    mask = None if tiles is None else tile_mask(cam, tiles, tile)
    if mode == "exact":
        ref, diag, _ = oracle.render(scene, cam, oracle.EXACT, tile=tile, tiles=tiles)
        return check(img, ref, diag, TOL, mask=mask, max_flagged=max_flagged, label=label + " exact")
    comp = comp if comp is not None else oracle.compact(scene)
    ref, diag, _ = oracle.render(scene, cam, oracle.ROOFGS, comp=comp, tile=tile, tiles=tiles)
    check(img, ref, diag, oracle.EPS_MAX + TOL + HALF_COLOUR, mask=mask, max_flagged=ROOFGS_FLAGGED,
          label=label + " roofgs vs exact exp")
    ref, diag, _ = oracle.render(scene, cam, oracle.ROOFGS, comp=comp, tile=tile, tiles=tiles,
                                 exp_kind=oracle.EXP_FAST32)
    return check(img, ref, diag, TOL + HALF_COLOUR, fp32=True, mask=mask, max_flagged=ROOFGS_FLAGGED,
                 label=label + " roofgs vs fp32 fast exp")

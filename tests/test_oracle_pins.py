"""Pins of the CPU oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: the paper's worked example and constants (tests/golden/), library
routines (scipy's spherical harmonics and rotations), closed forms, finite
differences, Monte-Carlo moments, brute force on tiny scenes and invariants.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2608_15785_gb300 import synth
from tests._helpers import read_golden, single_scene, small_random_scene

LN255 = math.log(255.0)


# --------------------------------------------------------------------------
# Sort-key layout (Sec. IV-A.2)
# --------------------------------------------------------------------------

def test_layout_worked_example():
    g = read_golden("key_layout_1080p.txt")
    cam = synth.look_at_camera((0, 0, -4), g["width"], g["height"])
    lay = oracle.layout(cam, (g["tile_w"], g["tile_h"]))
    assert lay["tiles_x"] == g["tiles_x"] and lay["tiles_y"] == g["tiles_y"]
    assert lay["tiles_x"] * lay["tiles_y"] == g["tiles"]
    assert lay["b_t"] == g["b_t"] and lay["b_d"] == g["b_d"]
    assert lay["qmax"] + 1 == g["levels"]


@pytest.mark.parametrize("w,h,tiles", [(16, 16, 1), (17, 16, 2), (32, 32, 4), (48, 16, 3), (3840, 2160, 32400),
                                       (7680, 4320, 129600)])
def test_layout_bit_split_is_ceil_log2(w, h, tiles):
    cam = synth.look_at_camera((0, 0, -4), w, h)
    lay = oracle.layout(cam)
    assert lay["tiles_x"] * lay["tiles_y"] == tiles
    # smallest b with 2^b >= tiles, by enumeration
    b = next(b for b in range(33) if 2 ** b >= tiles)
    assert lay["b_t"] == b and lay["b_d"] == 32 - b
    assert lay["qmax"] == 2 ** (32 - b) - 1


# --------------------------------------------------------------------------
# Spherical harmonics, rotations, projection
# --------------------------------------------------------------------------

def _real_sh_scipy(l, m, theta, phi):
    from scipy.special import sph_harm_y
    c = sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return math.sqrt(2) * (-1) ** m * c.real
    if m < 0:
        return math.sqrt(2) * (-1) ** m * c.imag
    return c.real


def test_sh_basis_matches_scipy_real_harmonics():
    rng = np.random.default_rng(3)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle.sh_basis(d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(_real_sh_scipy(l, m, theta, phi), abs=1e-12)


def test_sh_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform azimuth: exact for polynomials of degree <= 6
    mu, w = np.polynomial.legendre.leggauss(8)
    phis = np.arange(16) * (2 * math.pi / 16)
    G = np.zeros((16, 16))
    for m_, wm in zip(mu, w):
        st = math.sqrt(1 - m_ * m_)
        for ph in phis:
            Y = oracle.sh_basis((st * math.cos(ph), st * math.sin(ph), m_))
            G += wm * (2 * math.pi / 16) * np.outer(Y, Y)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_cov3d_matches_scipy_rotation():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(4)
    for _ in range(20):
        q = rng.normal(size=4)
        s = np.exp(rng.normal(-3, 1, size=3))
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is scalar-last
        ref = Rm @ np.diag(s ** 2) @ Rm.T
        got = oracle.cov3d(q, s)
        assert np.abs(got - ref).max() < 1e-14 * max(1.0, np.abs(ref).max()) * 10


def _pix(cam, p):
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


def test_projection_is_first_order_propagation():
    """Sigma' - 0.3 I = J W Sigma W^T J^T with J the finite-difference Jacobian of the pixel map."""
    cam = synth.look_at_camera((0.7, -0.4, -3.2), 320, 240)
    R = np.asarray(cam.R, dtype=np.float64).reshape(3, 3)
    t = np.asarray(cam.t, dtype=np.float64)
    rng = np.random.default_rng(5)
    for _ in range(10):
        m = rng.uniform(-0.5, 0.5, size=3).astype(np.float32)
        q = rng.normal(size=4).astype(np.float32)
        s = np.exp(rng.normal(-3, 0.5, size=3)).astype(np.float32)
        pr = oracle.project64(m, q, s, cam)
        p = R @ m.astype(np.float64) + t
        h = 1e-6
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            J[:, k] = (_pix(cam, p + e) - _pix(cam, p - e)) / (2 * h)
        Sig = oracle.cov3d(q.astype(np.float64), s.astype(np.float64))
        ref = J @ R @ Sig @ R.T @ J.T + 0.3 * np.eye(2)
        assert np.allclose(pr["cov2d"], ref, rtol=1e-6, atol=1e-9)
        uv = _pix(cam, p)
        assert pr["u"] == pytest.approx(uv[0], abs=1e-9) and pr["v"] == pytest.approx(uv[1], abs=1e-9)
        assert pr["z"] == pytest.approx(p[2], abs=1e-12)
        inv = np.linalg.inv(pr["cov2d"])
        assert pr["a"] == pytest.approx(inv[0, 0], rel=1e-12)
        assert pr["b"] == pytest.approx(2 * inv[0, 1], rel=1e-12)  # b multiplies dx*dy in Eq. (10)
        assert pr["c"] == pytest.approx(inv[1, 1], rel=1e-12)


def test_projection_matches_monte_carlo_moments():
    cam = synth.tiny_camera()
    rng = np.random.default_rng(6)
    m = np.array([0.2, -0.1, 0.1], dtype=np.float32)
    q = np.array([0.9, 0.2, -0.3, 0.1], dtype=np.float32)
    s = np.array([0.02, 0.006, 0.012], dtype=np.float32)
    Sig = oracle.cov3d(q.astype(np.float64), s.astype(np.float64))
    X = rng.multivariate_normal(m.astype(np.float64), Sig, size=400_000)
    R = np.asarray(cam.R, dtype=np.float64).reshape(3, 3)
    P = X @ R.T + np.asarray(cam.t, dtype=np.float64)
    uv = np.stack([cam.fx * P[:, 0] / P[:, 2] + cam.cx, cam.fy * P[:, 1] / P[:, 2] + cam.cy], axis=1)
    emp = np.cov(uv.T)
    pr = oracle.project64(m, q, s, cam)
    ref = pr["cov2d"] - 0.3 * np.eye(2)
    assert np.abs(emp - ref).max() < 0.01 * np.abs(ref).max()


def test_sh_colour_clamps_and_offsets():
    cam = synth.tiny_camera()
    sh = np.zeros((16, 3))
    sh[0] = [0.3, -5.0, 5.0]
    col = oracle.sh_colour(np.zeros(3, np.float32), sh, 0, cam)
    y00 = _real_sh_scipy(0, 0, 0.3, 0.2)
    assert col[0] == pytest.approx(0.3 * y00 + 0.5, abs=1e-15)
    assert col[1] == 0.0 and col[2] == 1.0


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def _isotropic_expected(cam, u, v, sig2, colour, alpha_of_q):
    H, W = cam.height, cam.width
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    r2 = (xs - u) ** 2 + (ys - v) ** 2
    a = alpha_of_q(r2 / sig2)
    return np.stack([colour[c] * a for c in range(3)])


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.ROOFGS])
def test_single_isotropic_gaussian_closed_form(mode):
    cam = synth.tiny_camera(255, 255)  # cx = cy = 127 lands on a pixel
    s, o, z = float(np.float32(0.03)), float(np.float32(0.3)), 3.0  # inputs are FP32
    dc = np.array([0.6, 0.1, -0.4], dtype=np.float32).astype(np.float64)
    sc = single_scene([0, 0, 0], [s, s, s], [1, 0, 0, 0], [o], dc)
    comp = oracle.compact(sc) if mode == oracle.ROOFGS else None
    img, diag, _ = oracle.render(sc, cam, mode, comp=comp, sh_degree=0)
    if mode == oracle.ROOFGS:
        s = float(comp.scales[0, 0])
        logo = float(comp.log_opac[0])
        col = np.clip(comp.sh[0, 0] * (0.5 / math.sqrt(math.pi)) + 0.5, 0, 1)

        def alpha(qq):
            P = -0.5 * qq + logo
            return np.where(P < -LN255, 0.0, np.minimum(0.99, np.exp(P)))
    else:
        col = np.clip(dc * (0.5 / math.sqrt(math.pi)) + 0.5, 0, 1)

        def alpha(qq):
            a = np.minimum(0.99, o * np.exp(-0.5 * qq))
            return np.where(a < 1 / 255, 0.0, a)
    sig2 = (cam.fx * s / z) ** 2 + 0.3
    ref = _isotropic_expected(cam, 127.0, 127.0, sig2, col, alpha)
    ok = diag[..., 1] == 0  # pixels whose skip decision is not within rounding of 1/255
    assert ok.mean() > 0.99
    assert np.abs(img - ref)[:, ok].max() < 1e-12


def test_two_gaussian_closed_form():
    cam = synth.tiny_camera(255, 255)
    dc = np.array([[0.9, -0.2, 0.1], [-0.5, 0.8, 0.3]], dtype=np.float32).astype(np.float64)
    sc = single_scene([[0, 0, 0], [0, 0, 0.5]], [[0.03] * 3, [0.05] * 3], [[1, 0, 0, 0]] * 2, [0.7, 0.6], dc)
    img, _, _ = oracle.render(sc, cam, oracle.EXACT, sh_degree=0)
    c = np.clip(dc * (0.5 / math.sqrt(math.pi)) + 0.5, 0, 1)
    a1, a2 = float(np.float32(0.7)), float(np.float32(0.6))  # at the shared centre pixel the power is 0
    expect = c[0] * a1 + c[1] * a2 * (1 - a1)
    assert np.abs(img[:, 127, 127] - expect).max() < 1e-12
    # swapping the input order must not change the front-to-back result
    sc2 = single_scene([[0, 0, 0.5], [0, 0, 0]], [[0.05] * 3, [0.03] * 3], [[1, 0, 0, 0]] * 2, [0.6, 0.7], dc[::-1])
    img2, _, _ = oracle.render(sc2, cam, oracle.EXACT, sh_degree=0)
    assert np.abs(img2 - img).max() < 1e-15


def test_transmittance_stop_without_adding():
    """Three opaque (0.99) Gaussians on a pixel: T goes 1 -> 0.01 -> 1e-4 (not < 1e-4) -> stop at the third."""
    cam = synth.tiny_camera(255, 255)
    dc = np.array([[0.9, 0.9, 0.9], [-0.9, -0.9, -0.9], [0.5, 0.0, -0.5]], dtype=np.float32).astype(np.float64)
    sc = single_scene([[0, 0, 0], [0, 0, 0.3], [0, 0, 0.6]], [[0.05] * 3] * 3, [[1, 0, 0, 0]] * 3,
                      [1.0, 1.0, 1.0], dc)
    img, _, _ = oracle.render(sc, cam, oracle.EXACT, sh_degree=0)
    c = np.clip(dc * (0.5 / math.sqrt(math.pi)) + 0.5, 0, 1)
    # 1 * 0.01 = 0.01; 0.01 * 0.01 = 1e-4 which is not < 1e-4, so the second adds;
    # the third would give 1e-6 < 1e-4 and is not added.
    expect = c[0] * 0.99 + c[1] * 0.99 * 0.01
    assert np.abs(img[:, 127, 127] - expect).max() < 1e-12


# --------------------------------------------------------------------------
# Brute force against the tiled oracle
# --------------------------------------------------------------------------

def _brute_force(scene, cam, mode, comp=None, sh_degree=3):
    """Per pixel over ALL Gaussians, ordered by FP64 depth, with the paper's skip/clamp/stop rules."""
    H, W = cam.height, cam.width
    src = comp if comp is not None else scene
    op = comp.log_opac if comp is not None else scene.opacities
    sh = comp.sh if comp is not None else scene.sh.astype(np.float64)
    G = []
    for i in range(scene.n):
        pr = oracle.project64(src.means[i], src.quats[i], src.scales[i], cam)
        if not (cam.znear < pr["z"] <= cam.zfar):
            continue
        if mode == oracle.ROOFGS and not (op[i] >= -LN255):
            continue
        col = oracle.sh_colour(src.means[i], sh[i], sh_degree, cam)
        G.append((pr["z"], i, pr, col))
    G.sort(key=lambda g: (g[0], g[1]))
    img = np.zeros((3, H, W))
    pmax = -np.inf
    for y in range(H):
        for x in range(W):
            T, Cc = 1.0, np.zeros(3)
            for _, i, pr, col in G:
                dx, dy = x - pr["u"], y - pr["v"]
                p = -0.5 * (pr["a"] * dx * dx + pr["b"] * dx * dy + pr["c"] * dy * dy)
                if mode == oracle.EXACT:
                    a = min(0.99, float(op[i]) * math.exp(p))
                    if a < 1 / 255:
                        continue
                else:
                    P = p + float(op[i])
                    if P < -LN255:
                        continue
                    pmax = max(pmax, P)
                    a = min(0.99, math.exp(P))
                Tn = T * (1 - a)
                if Tn < 1e-4:
                    break
                Cc += col * a * T
                T = Tn
            img[:, y, x] = Cc + T * np.asarray(cam.bg, dtype=np.float64)
    return img, pmax


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.ROOFGS])
@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 4)])
def test_brute_force_matches_tiled(mode, tile):
    # Exact mode truncates at the 3-sigma box; with o <= 0.35 every alpha >= 1/255 lies inside it,
    # so membership equals "alpha >= 1/255" and brute force over all Gaussians is the same image.
    sc = small_random_scene(48, seed=11, max_opacity=0.35 if mode == oracle.EXACT else 1.0)
    cam = synth.tiny_camera(32, 32, bg=(0.2, 0.5, 0.9))
    cam.fx = cam.fy = float(np.float32(16 / math.tan(math.radians(30))))
    comp = oracle.compact(sc) if mode == oracle.ROOFGS else None
    img, diag, _ = oracle.render(sc, cam, mode, tile=tile, comp=comp)
    ref, pmax = _brute_force(sc, cam, mode, comp)
    ok = (diag[..., 1] == 0) & (diag[..., 2] == 0)
    assert ok.mean() > 0.95
    assert np.abs(img - ref)[:, ok].max() < 1e-12
    assert np.abs(img - ref).max() <= (diag[..., 1] + diag[..., 2]).max() + 1e-12
    if mode == oracle.ROOFGS:
        assert pmax <= 0.0  # Eq. (23): surviving exponents are non-positive


# --------------------------------------------------------------------------
# Invariants on the tiny workload
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny():
    sc, cams = synth.workload("tiny_256")
    return sc.subset(np.arange(3000)), cams[0]


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.ROOFGS])
def test_pixels_in_unit_range_and_transmittance_bounds(tiny, mode):
    sc, cam = tiny
    comp = oracle.compact(sc) if mode == oracle.ROOFGS else None
    img0, _, _ = oracle.render(sc, cam, mode, comp=comp, with_diag=False)
    cam1 = synth.tiny_camera(bg=(1.0, 1.0, 1.0))
    img1, _, _ = oracle.render(sc, cam1, mode, comp=comp, with_diag=False)
    assert img0.min() >= 0.0 and img1.max() <= 1.0 + 1e-12
    T = img1 - img0  # final transmittance, identical in every channel
    assert np.abs(T - T[0:1]).max() < 1e-12
    assert T.min() >= 1e-4 - 1e-15 and T.max() <= 1.0


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.ROOFGS])
def test_permutation_invariance(tiny, mode):
    sc, cam = tiny
    perm = np.random.default_rng(7).permutation(sc.n)
    scp = sc.subset(perm)
    if mode == oracle.ROOFGS:
        ca, cb = oracle.compact(sc), oracle.compact(scp)
    else:
        ca = cb = None
    a, _, _ = oracle.render(sc, cam, mode, comp=ca, with_diag=False)
    b, _, _ = oracle.render(scp, cam, mode, comp=cb, with_diag=False)
    assert np.abs(a - b).max() < 1e-12


def test_snug_box_image_independent_of_tile_shape(tiny):
    sc, cam = tiny
    comp = oracle.compact(sc)
    a, da, _ = oracle.render(sc, cam, oracle.ROOFGS, tile=(16, 16), comp=comp)
    for tile in [(8, 8), (32, 8), (4, 64)]:
        b, _, _ = oracle.render(sc, cam, oracle.ROOFGS, tile=tile, comp=comp)
        ok = da[..., 1] == 0
        assert np.abs(a - b)[:, ok].max() < 1e-12


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.ROOFGS])
def test_box_contains_every_pixel_it_must(tiny, mode):
    """RoofGS box holds every pixel with alpha~ >= 1/255; exact box holds the 3-sigma ellipse."""
    sc, cam = tiny
    comp = oracle.compact(sc) if mode == oracle.ROOFGS else None
    src = comp if comp is not None else sc
    keys_, vals_, _, bins = oracle.keys(sc, cam, mode, comp=comp)
    lay = oracle.layout(cam)
    shift = np.uint64(32 if mode == oracle.EXACT else lay["b_d"])
    tiles_of = {}
    for kk, vv in zip((keys_ >> shift).astype(np.int64), vals_):
        tiles_of.setdefault(int(vv), set()).add(int(kk))
    checked = 0
    for i in range(0, sc.n, 7):
        pr = oracle.project64(src.means[i], src.quats[i], src.scales[i], cam)
        if not (cam.znear < pr["z"] <= cam.zfar):
            continue
        x0, x1 = int(pr["u"]) - 40, int(pr["u"]) + 40
        y0, y1 = int(pr["v"]) - 40, int(pr["v"]) + 40
        ys, xs = np.mgrid[max(0, y0):min(cam.height, y1), max(0, x0):min(cam.width, x1)]
        dx, dy = xs - pr["u"], ys - pr["v"]
        qq = pr["a"] * dx * dx + pr["b"] * dx * dy + pr["c"] * dy * dy
        if mode == oracle.ROOFGS:
            must = -0.5 * qq + float(comp.log_opac[i]) > -LN255 + 1e-5
        else:
            must = qq < 9.0 * (1 - 1e-5)
        if not must.any():
            continue
        vis, tx0, ty0, tx1, ty1, _, _ = bins[i]
        assert vis == 1
        tx, ty = xs[must] // 16, ys[must] // 16
        assert tx.min() >= tx0 and tx.max() <= tx1 and ty.min() >= ty0 and ty.max() <= ty1
        # every such pixel's tile is one of the Gaussian's entries (RoofGS: per-row test)
        assert set((ty * lay["tiles_x"] + tx).tolist()) <= tiles_of[i]
        checked += 1
    assert checked > 50


@pytest.mark.parametrize("ties", [False, True])
def test_exact_key_low_word_is_depth_ascending_within_tiles(ties):
    """Exact mode's 64-bit key (the baseline key of Sec. IV-A.2): its low word, read as an
    IEEE single, is the camera depth of the entry's Gaussian (the FP64 depth within FP32
    rounding); inside every tile the entries ascend by that depth, equal depths by
    ascending Gaussian index, and the order agrees with the FP64 depths up to rounding."""
    if ties:  # 60 Gaussians share the mean (hence the depth) of another one
        sc = small_random_scene(300, seed=4)
        sc.means[200:260] = sc.means[0:60]
        cam = synth.tiny_camera(64, 64)
    else:
        sc, cams = synth.workload("tiny_256")
        cam = cams[0]
    k, v, ranges, bins = oracle.keys(sc, cam, oracle.EXACT)
    assert k.size > 100
    R = np.asarray(cam.R, dtype=np.float64).reshape(3, 3)
    z = (sc.means.astype(np.float64) @ R.T + np.asarray(cam.t, np.float64))[:, 2]
    low = (k & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    zv = z[v.astype(np.int64)]
    assert np.all(np.abs(low - zv) <= 4.0 * 2.0 ** -24 * np.abs(zv))
    tile = (k >> np.uint64(32)).astype(np.int64)
    assert np.all(np.diff(tile) >= 0)
    same = tile[1:] == tile[:-1]
    assert np.all(low[1:][same] >= low[:-1][same])
    eq = same & (low[1:] == low[:-1])
    assert np.all(v[1:][eq] > v[:-1][eq])
    assert np.all(zv[1:][same] >= zv[:-1][same] - 8.0 * 2.0 ** -24 * np.abs(zv[1:][same]))
    if ties:
        assert eq.sum() >= 20  # tied depths were met and ordered by index
    # the tile word and the ranges agree
    for t in np.unique(tile):
        s, e = ranges[t]
        assert np.all(tile[s:e] == t) and e - s == np.count_nonzero(tile == t)


# --------------------------------------------------------------------------
# Quantized depth key (Eq. (9))
# --------------------------------------------------------------------------

def test_quantized_depth_is_monotone_with_bounded_bins():
    sc, cams = synth.workload("tiny_256")
    cam = cams[0]
    comp = oracle.compact(sc)
    k, v, ranges, bins = oracle.keys(sc, cam, oracle.ROOFGS, comp=comp)
    lay = oracle.layout(cam)
    R = np.asarray(cam.R, dtype=np.float64).reshape(3, 3)
    z = (sc.means.astype(np.float64) @ R.T + np.asarray(cam.t, np.float64))[:, 2]
    vis = bins[:, 0] == 1
    qd = bins[vis, 5].astype(np.uint32).astype(np.int64)
    zv = z[vis]
    order = np.argsort(zv, kind="stable")
    assert np.all(np.diff(qd[order]) >= 0)  # non-decreasing in depth
    delta = (cam.zfar - cam.znear) / lay["qmax"]
    exact = np.floor((zv - cam.znear) / (cam.zfar - cam.znear) * lay["qmax"])
    assert np.abs(qd - exact).max() <= 1
    for q in np.unique(qd)[:2000]:
        zs = zv[qd == q]
        assert zs.max() - zs.min() < delta * 1.0001 + 4e-7
    # tile bits on top, depth bits below; entries ascending
    assert np.all(np.diff(k.astype(np.uint64).astype(np.float64)) >= 0)
    tiles = (k >> np.uint64(lay["b_d"])).astype(np.int64)
    for t in np.unique(tiles)[:50]:
        s, e = ranges[t]
        assert np.all(tiles[s:e] == t) and e - s == np.count_nonzero(tiles == t)


# --------------------------------------------------------------------------
# Fast exponential (Eq. (23)-(24)) and the colour error bound
# --------------------------------------------------------------------------

def _all_fp32_between(lo, hi):
    """Every float32 value in [lo, hi] for lo < hi < 0."""
    a = np.uint32(np.float32(hi).view(np.uint32))
    b = np.uint32(np.float32(lo).view(np.uint32))
    return np.arange(a, b + 1, dtype=np.uint32).view(np.float32).astype(np.float64)


def test_fast_exp_error_within_stated_bound():
    g = read_golden("fast_exp.txt")
    assert g["sigma"] == oracle.SIGMA
    lo = -LN255
    assert lo == pytest.approx(g["range_lo"], abs=1e-3)
    # every float32 in [-1.5, -0.5] (more than one period ln 2 of the error), a fine sweep of
    # the whole range [-ln 255, 0], and its end points
    P = np.concatenate([_all_fp32_between(-1.5, -0.5), np.linspace(lo, 0.0, 2_000_001),
                        [np.float64(np.float32(lo)), -0.0]])
    P = P[P >= lo]
    for kind in (oracle.EXP_FAST64, oracle.EXP_FAST32):
        rel = oracle.fast_exp_many(P, kind) / np.exp(P) - 1.0
        assert rel.max() <= 0.02841 and rel.min() >= -0.03118
        # the bound is attained: pins sigma (sigma = 0 would give errors up to -6 %)
        assert abs(rel.min()) > 0.0311
        assert max(abs(rel.min()), rel.max()) <= oracle.EPS_MAX
        assert oracle.EPS_MAX == pytest.approx(g["eps_max_stated"], abs=0.0015)
    d = oracle.fast_exp_many(P, oracle.EXP_FAST32) / oracle.fast_exp_many(P, oracle.EXP_FAST64) - 1
    assert np.abs(d).max() <= 2.0 ** -16  # FP32 evaluation moves I(P) by less than 64 units


def test_fast_exp_bit_pattern_at_zero():
    # I(0) = floor(2^23 (127 - sigma)) = 1064970049; as float bits that is 0x3F7A4441
    i0 = math.floor(2 ** 23 * (127 - 0.045677))
    assert i0 == 1064970049
    f = np.array([i0], dtype=np.uint32).view(np.float32)[0]
    assert oracle.fast_exp64(0.0) == float(f)
    assert 1 - 0.0312 < f < 1.0


@pytest.mark.parametrize("kind", [oracle.EXP_FAST64, oracle.EXP_FAST32])
def test_colour_error_bound_of_fast_exp(tiny, kind):
    """|C_fast - C_exact|_inf <= eps_max per pixel, independent of the Gaussian count."""
    sc, cam = tiny
    comp = oracle.compact(sc)
    a, _, _ = oracle.render(sc, cam, oracle.ROOFGS, comp=comp, with_diag=False)
    b, _, _ = oracle.render(sc, cam, oracle.ROOFGS, comp=comp, exp_kind=kind, with_diag=False)
    assert np.abs(a - b).max() <= oracle.EPS_MAX


# --------------------------------------------------------------------------
# INT8 SH codec (Eq. (8))
# --------------------------------------------------------------------------

@pytest.mark.parametrize("per_gaussian", [False, True])
def test_sh_codec_error_and_extremes(per_gaussian):
    sc = synth.tiny_scene(2000, seed=9)
    codes, bs, g, deq = oracle.sh_encode(sc.sh, per_gaussian)
    assert codes.dtype == np.int8 and np.abs(codes.astype(np.int32)).max() <= 127
    s_k = bs[oracle.SH_BAND]
    den = (g[:, None, None] * s_k[None]) if per_gaussian else np.broadcast_to(s_k, sc.sh.shape)
    den = den.astype(np.float64)
    err = np.abs(deq - sc.sh.astype(np.float64))
    # half a step, plus the FP32 rounding of SH / s (|code| <= 127 -> at most 127 * 2^-24 of a step)
    assert np.all(err <= den * (0.5 + 127 * 2.0 ** -24) + 1e-12)
    for d in range(4):
        ks = np.nonzero(oracle.SH_BAND == d)[0]
        for c in range(3):
            # the largest |SH| of degree d, channel c maps to +-127 under the global scale
            a = np.abs(sc.sh[:, ks, c])
            assert bs[d, c] == np.float32(a.max()) / np.float32(127)
            if not per_gaussian:
                i, j = np.unravel_index(np.argmax(a), a.shape)
                assert abs(int(codes[i, ks[j], c])) == 127
    if per_gaussian:
        # every Gaussian uses its own range: its largest normalised coefficient maps to ~127
        top = np.abs(codes.astype(np.int32)).reshape(len(g), -1).max(axis=1)
        assert np.all(top >= 126)


# --------------------------------------------------------------------------
# FP64 gradient of the exact-mode render
# --------------------------------------------------------------------------

def test_fp64_gradient_matches_central_differences():
    """oracle.backward (back-to-front adjoint of Eq. (7), complex-step Jacobian of the
    per-Gaussian projection and colour) against central differences of the FP64 forward,
    for every attribute kind of several Gaussians. The forward has steps (the 1/255 skip,
    the 1e-4 stop, the 0.99 clamp): a sample whose two step sizes disagree sits on one
    and is set aside; the rest agree to 1e-5."""
    sc = small_random_scene(40, seed=3)
    cam = synth.tiny_camera(48, 40, bg=(0.1, 0.2, 0.3))
    w = np.random.default_rng(0).normal(size=(3, 40, 48))
    g = oracle.backward(sc, cam, w)

    def loss(s):
        return float(np.sum(w * oracle.render(s, cam, oracle.EXACT, with_diag=False)[0]))

    def fd(field, i, k, rel):
        x0 = float(getattr(sc, field)[i].reshape(-1)[k])
        h = rel * max(abs(x0), 0.05)
        val = []
        for sgn in (1, -1):
            s2 = sc.subset(np.arange(sc.n))
            arr = getattr(s2, field)
            xv = np.float32(x0 + sgn * h)
            if arr.ndim == 1:
                arr[i] = xv
            else:
                arr[i].reshape(-1)[k] = xv
            val.append((loss(s2), float(xv)))
        return (val[0][0] - val[1][0]) / (val[0][1] - val[1][1])

    checked = skipped = 0
    for field, dim in (("means", 3), ("scales", 3), ("quats", 4), ("opacities", 1), ("sh", 48)):
        for i in range(1, 40, 6):
            for k in ((0, 1, 2) if dim == 3 else (0, 2, 3) if dim == 4 else (0,) if dim == 1 else (0, 4, 47)):
                a, b = fd(field, i, k, 1e-4), fd(field, i, k, 3e-5)
                if abs(a - b) > 1e-4 * (abs(a) + 1e-3):
                    skipped += 1
                    continue
                gv = float(g[field][i].reshape(-1)[k])
                assert abs(gv - b) <= 1e-5 * abs(b) + 1e-7, (field, i, k, gv, b)
                checked += 1
    assert checked >= 80 and skipped <= checked // 10, (checked, skipped)


def test_fp64_gradient_of_clamped_and_absent_gaussians_is_zero():
    """A Gaussian behind the camera, and one whose colour is clamped above 1 in every channel,
    receive no gradient through the clamped colour; the first receives none at all."""
    sc = small_random_scene(30, seed=5)
    sc.means[3] = [0.0, 0.0, -10.0]           # behind the camera
    sc.sh[4, 0, :] = 10.0                      # raw colour far above 1: clamped
    cam = synth.tiny_camera(40, 40)
    g = oracle.backward(sc, cam, np.ones((3, 40, 40)))
    for f in ("means", "scales", "quats", "opacities", "sh"):
        assert np.all(g[f][3] == 0.0)
    assert np.all(g["sh"][4] == 0.0)

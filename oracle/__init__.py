"""CPU oracle of the RoofGS forward render -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The renderer (``paper_2608_15785_gb300``)
never imports it and shares no code with it.

The heavy part is plain C (``rg_oracle.c``, FP64 blending plus the FP32
pinned-order binning path); this module compiles it with gcc, wraps it with
ctypes, and implements in numpy the compact-attribute conversion of RoofGS mode
(Sec. IV-A.1): FP16 rotation and scale, log-opacity, and the INT8 spherical
harmonics quantiser of Eq. (8) with one symmetric scale per SH degree d and
colour channel c (optionally times one FP16 scale per Gaussian).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "librg_oracle.so")
_lib = None

EXACT = 0
ROOFGS = 1
EXP_EXACT = 0
EXP_FAST64 = 1
EXP_FAST32 = 2

LN255 = float(np.log(255.0))
SIGMA = 0.045677  # calibration constant of Eq. (24)
EPS_MAX = 0.0312  # measured sup |relative error| of Eq. (24) on [-ln 255, 0]

# SH degree of each of the 16 coefficients (k = l^2 + l + m)
SH_BAND = np.array([0, 1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3], dtype=np.int64)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FP contraction, IEEE semantics)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cam(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("zfar", C.c_float), ("bg", C.c_float * 3)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        lib.orc_render.restype = C.c_int64
        lib.orc_render.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, P, C.c_int, C.c_int32, C.c_int32,
                                   C.c_int, P, C.c_int64, P, P]
        lib.orc_keys.restype = C.c_int64
        lib.orc_keys.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, C.c_int32, C.c_int32, P, P,
                                 C.c_int64, P, P]
        lib.orc_layout_query.restype = C.c_int
        lib.orc_layout_query.argtypes = [P, C.c_int32, C.c_int32, P]
        lib.orc_sh_basis.restype = None
        lib.orc_sh_basis.argtypes = [C.c_double, C.c_double, C.c_double, P]
        lib.orc_cov3d.restype = None
        lib.orc_cov3d.argtypes = [P, P, P]
        lib.orc_project64.restype = None
        lib.orc_project64.argtypes = [P, P, P, P, P]
        lib.orc_sh_colour.restype = None
        lib.orc_sh_colour.argtypes = [P, P, C.c_int, P, P]
        lib.orc_fast_exp64.restype = C.c_double
        lib.orc_fast_exp64.argtypes = [C.c_double]
        lib.orc_fast_exp32.restype = C.c_double
        lib.orc_fast_exp32.argtypes = [C.c_float]
        lib.orc_fast_exp_many.restype = None
        lib.orc_fast_exp_many.argtypes = [C.c_int64, P, P, C.c_int]
        lib.orc_log_opacity.restype = None
        lib.orc_log_opacity.argtypes = [C.c_int64, P, P]
        lib.orc_backward.restype = C.c_int
        lib.orc_backward.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, P, C.c_int32, C.c_int32, P, P, P, P, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def cam_struct(cam) -> _Cam:
    """Camera object with fields R(9), t(3), fx, fy, cx, cy, width, height, znear, zfar, bg(3)."""
    c = _Cam()
    for i, x in enumerate(np.asarray(cam.R, dtype=np.float32).reshape(9)):
        c.R[i] = float(x)
    for i, x in enumerate(np.asarray(cam.t, dtype=np.float32).reshape(3)):
        c.t[i] = float(x)
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear, c.zfar = float(np.float32(cam.znear)), float(np.float32(cam.zfar))
    for i, x in enumerate(np.asarray(cam.bg, dtype=np.float32).reshape(3)):
        c.bg[i] = float(x)
    return c


# --------------------------------------------------------------------------
# Compact attributes of RoofGS mode (Sec. IV-A.1)
# --------------------------------------------------------------------------

@dataclass
class Compact:
    means: np.ndarray      # [N,3] f32 (kept in FP32)
    quats: np.ndarray      # [N,4] f32 holding FP16-rounded values
    scales: np.ndarray     # [N,3] f32 holding FP16-rounded values
    log_opac: np.ndarray   # [N] f32, log o rounded to FP32
    codes: np.ndarray      # [N,16,3] int8
    band_scale: np.ndarray  # [4,3] f32, s_{d,c}
    gauss_scale: np.ndarray  # [N] f32 holding FP16-rounded per-Gaussian factors (ones if unused)
    sh: np.ndarray         # [N,16,3] f64 dequantised coefficients


def log_opacity(o: np.ndarray) -> np.ndarray:
    """log o computed in FP64 by the C library and rounded to FP32."""
    lib = _load()
    o = _f32(o)
    out = np.empty_like(o)
    lib.orc_log_opacity(o.size, _ptr(o), _ptr(out))
    return out


def sh_encode(sh: np.ndarray, per_gaussian: bool = False):
    """INT8 quantiser of Eq. (8), in FP32.

    s_{d,c} = max_i |SH_{i,d,c}| / 127 over every Gaussian i and every
    coefficient of degree d; code = round(SH / s) with ties to even.
    With per_gaussian, every Gaussian i also carries
    g_i = max_k |SH_{i,k,c}| / (127 s_{d(k),c}) rounded to FP16, and its codes
    are round(SH / fl32(g_i s_{d,c})). Codes are clamped to [-127, 127].
    Returns (codes int8 [N,16,3], band_scale f32 [4,3], g f32 [N], dequantised f64 [N,16,3]).
    """
    sh = _f32(sh)
    n = sh.shape[0]
    a = np.abs(sh)
    band_scale = np.zeros((4, 3), dtype=np.float32)
    for d in range(4):
        ks = np.nonzero(SH_BAND == d)[0]
        if n:
            band_scale[d] = a[:, ks, :].max(axis=(0, 1))
    band_scale = (band_scale / np.float32(127.0)).astype(np.float32)
    s_k = band_scale[SH_BAND]  # [16,3]
    if per_gaussian:
        den127 = (np.float32(127.0) * s_k).astype(np.float32)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(den127 > 0, a / den127, np.float32(0)).astype(np.float32)
        g = r.reshape(n, -1).max(axis=1) if n else np.zeros(0, np.float32)
        g = g.astype(np.float16).astype(np.float32)
        den = (g[:, None, None] * s_k[None]).astype(np.float32)
    else:
        g = np.ones(n, dtype=np.float32)
        den = np.broadcast_to(s_k[None], sh.shape).astype(np.float32)
    with np.errstate(divide="ignore", invalid="ignore"):
        qf = np.where(den > 0, sh / den, np.float32(0)).astype(np.float32)
    codes = np.clip(np.rint(qf), -127, 127).astype(np.int8)
    deq = den.astype(np.float64) * codes.astype(np.float64)
    return codes, band_scale, g, deq


def compact(scene, per_gaussian_sh_scale: bool = False) -> Compact:
    codes, bs, g, deq = sh_encode(scene.sh, per_gaussian_sh_scale)
    return Compact(
        means=_f32(scene.means),
        quats=_f32(scene.quats).astype(np.float16).astype(np.float32),
        scales=_f32(scene.scales).astype(np.float16).astype(np.float32),
        log_opac=log_opacity(scene.opacities),
        codes=codes, band_scale=bs, gauss_scale=g, sh=deq)


# --------------------------------------------------------------------------
# Rendering and keys
# --------------------------------------------------------------------------

def _inputs(scene, mode, comp: Compact | None):
    if mode == EXACT:
        return (_f32(scene.means), _f32(scene.quats), _f32(scene.scales), _f32(scene.opacities),
                np.ascontiguousarray(scene.sh, dtype=np.float64))
    if comp is None:
        raise ValueError("RoofGS mode needs the compact attributes")
    return comp.means, comp.quats, comp.scales, comp.log_opac, np.ascontiguousarray(comp.sh)


def render(scene, cam, mode=EXACT, tile=(16, 16), exp_kind=EXP_EXACT, comp: Compact | None = None,
           tiles=None, sh_degree=3, with_diag=True):
    """FP64 tiled render. Returns (img [3,H,W] f64, diag [H,W,4] f64 or None, n_entries).

    Pixels of tiles not listed in ``tiles`` are NaN.
    """
    lib = _load()
    m, q, s, op, sh = _inputs(scene, mode, comp)
    n = m.shape[0]
    H, W = int(cam.height), int(cam.width)
    img = np.full((3, H, W), np.nan, dtype=np.float64)
    diag = np.zeros((H, W, 4), dtype=np.float64) if with_diag else None
    c = cam_struct(cam)
    if tiles is None:
        tptr, nt = None, 0
    else:
        tarr = np.ascontiguousarray(tiles, dtype=np.int32)
        tptr, nt = _ptr(tarr), tarr.size
    total = lib.orc_render(n, _ptr(m), _ptr(q), _ptr(s), _ptr(op), _ptr(sh), int(sh_degree), C.byref(c),
                           int(mode), int(tile[0]), int(tile[1]), int(exp_kind), tptr, nt, _ptr(img),
                           _ptr(diag) if diag is not None else None)
    if total < 0:
        raise RuntimeError("oracle render failed")
    return img, diag, int(total)


def backward(scene, cam, dL_dimg, tile=(16, 16), sh_degree=3) -> dict:
    """FP64 gradient of L = sum(dL_dimg * img) for the exact-mode image of ``render``, with
    respect to the scene's FP32 attributes: dict of means [N,3], scales [N,3], quats [N,4],
    opacities [N], sh [N,16,3] (float64)."""
    lib = _load()
    m, q, s, op, sh = _inputs(scene, EXACT, None)
    n = m.shape[0]
    H, W = int(cam.height), int(cam.width)
    g = np.ascontiguousarray(dL_dimg, dtype=np.float64).reshape(3, H, W)
    nn = max(n, 1)
    out = {"means": np.zeros((nn, 3)), "scales": np.zeros((nn, 3)), "quats": np.zeros((nn, 4)),
           "opacities": np.zeros(nn), "sh": np.zeros((nn, 16, 3))}
    c = cam_struct(cam)
    rc = lib.orc_backward(n, _ptr(m), _ptr(q), _ptr(s), _ptr(op), _ptr(sh), int(sh_degree), C.byref(c),
                          int(tile[0]), int(tile[1]), _ptr(g), _ptr(out["means"]), _ptr(out["scales"]),
                          _ptr(out["quats"]), _ptr(out["opacities"]), _ptr(out["sh"]))
    if rc != 0:
        raise RuntimeError("oracle backward failed")
    return {k: v[:n] for k, v in out.items()}


def keys(scene, cam, mode=EXACT, tile=(16, 16), comp: Compact | None = None):
    """Sorted entries of the frame: (keys u64, vals u32, ranges u32 [NT,2], bins i32 [N,7]).

    bins[i] = (visible, tx0, ty0, tx1, ty1, q_d, entries of Gaussian i)."""
    lib = _load()
    m, q, s, op, _ = _inputs(scene, mode, comp)
    n = m.shape[0]
    c = cam_struct(cam)
    lay = layout(cam, tile)
    nt = lay["tiles_x"] * lay["tiles_y"]
    bins = np.zeros((n, 7), dtype=np.int32)
    total = lib.orc_keys(n, _ptr(m), _ptr(q), _ptr(s), _ptr(op), C.byref(c), int(mode), int(tile[0]),
                         int(tile[1]), None, None, 0, None, _ptr(bins))
    if total < 0:
        raise RuntimeError("oracle keys failed")
    k = np.zeros(max(total, 1), dtype=np.uint64)
    v = np.zeros(max(total, 1), dtype=np.uint32)
    ranges = np.zeros((nt, 2), dtype=np.uint32)
    lib.orc_keys(n, _ptr(m), _ptr(q), _ptr(s), _ptr(op), C.byref(c), int(mode), int(tile[0]), int(tile[1]),
                 _ptr(k), _ptr(v), total, _ptr(ranges), None)
    return k[:total], v[:total], ranges, bins


def layout(cam, tile=(16, 16)) -> dict:
    lib = _load()
    out = np.zeros(6, dtype=np.int64)
    c = cam_struct(cam)
    if lib.orc_layout_query(C.byref(c), int(tile[0]), int(tile[1]), _ptr(out)) != 0:
        raise ValueError("bad layout")
    return {"tiles_x": int(out[0]), "tiles_y": int(out[1]), "b_t": int(out[2]), "b_d": int(out[3]),
            "qmax": int(out[4]),
            "depth_scale": float(np.array([out[5]], dtype=np.uint32).view(np.float32)[0])}


def sh_basis(d) -> np.ndarray:
    lib = _load()
    out = np.zeros(16, dtype=np.float64)
    lib.orc_sh_basis(float(d[0]), float(d[1]), float(d[2]), _ptr(out))
    return out


def cov3d(q, s) -> np.ndarray:
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros(9, dtype=np.float64)
    lib.orc_cov3d(_ptr(q), _ptr(s), _ptr(out))
    return out.reshape(3, 3)


def project64(mean, quat, scale, cam) -> dict:
    lib = _load()
    m, q, s = _f32(mean), _f32(quat), _f32(scale)
    out = np.zeros(10, dtype=np.float64)
    c = cam_struct(cam)
    lib.orc_project64(_ptr(m), _ptr(q), _ptr(s), C.byref(c), _ptr(out))
    return {"u": out[0], "v": out[1], "z": out[2], "cov2d": np.array([[out[3], out[4]], [out[4], out[5]]]),
            "a": out[6], "b": out[7], "c": out[8], "det": out[9]}


def sh_colour(mean, sh16x3, deg, cam) -> np.ndarray:
    lib = _load()
    m = _f32(mean)
    sh = np.ascontiguousarray(sh16x3, dtype=np.float64)
    out = np.zeros(3, dtype=np.float64)
    c = cam_struct(cam)
    lib.orc_sh_colour(_ptr(m), _ptr(sh), int(deg), C.byref(c), _ptr(out))
    return out


def fast_exp64(P: float) -> float:
    return _load().orc_fast_exp64(float(P))


def fast_exp32(P: float) -> float:
    return _load().orc_fast_exp32(float(np.float32(P)))


def fast_exp_many(P, kind=EXP_FAST64) -> np.ndarray:
    """Eq. (24) over an array of exponents (kind EXP_FAST64 or EXP_FAST32)."""
    lib = _load()
    P = np.ascontiguousarray(P, dtype=np.float64)
    out = np.empty_like(P)
    lib.orc_fast_exp_many(P.size, _ptr(P), _ptr(out), int(kind))
    return out

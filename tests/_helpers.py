"""Shared test helpers: golden-file reader and small scene builders."""
from __future__ import annotations

import math
import os

import numpy as np

from paper_2608_15785_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(None, 1)
            out[k] = float(v) if any(ch in v for ch in ".e") else int(v)
    return out


def single_scene(means, scales, quats, opac, dc, sh_rest=None) -> synth.Scene:
    means = np.asarray(means, dtype=np.float32).reshape(-1, 3)
    n = means.shape[0]
    sh = np.zeros((n, 16, 3), dtype=np.float32)
    sh[:, 0, :] = np.asarray(dc, dtype=np.float32).reshape(n, 3)
    if sh_rest is not None:
        sh[:, 1:, :] = sh_rest
    return synth.Scene(means, np.asarray(scales, dtype=np.float32).reshape(n, 3),
                       np.asarray(quats, dtype=np.float32).reshape(n, 4),
                       np.asarray(opac, dtype=np.float32).reshape(n), sh)


def small_random_scene(n: int, seed: int, max_opacity: float = 1.0, spread: float = 0.6,
                       log_scale=(-2.8, 0.4)) -> synth.Scene:
    """Few, larger Gaussians in front of the tiny camera (for 32x32-ish images)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-spread, spread, size=(n, 3)).astype(np.float32)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], size=(n, 3))).astype(np.float32)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = (max_opacity / (1.0 + np.exp(-rng.normal(0, 1.5, size=n)))).astype(np.float32)
    sh = np.empty((n, 16, 3), dtype=np.float32)
    sh[:, 0, :] = rng.normal(0.5, 0.2, size=(n, 3))
    sh[:, 1:, :] = rng.normal(0.0, 0.3, size=(n, 15, 3))
    return synth.Scene(means, scales, q.astype(np.float32), opac, sh)


def hfov_fx(width: int, hfov_deg: float = 60.0) -> float:
    return (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)

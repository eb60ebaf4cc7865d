"""Seeded synthetic scenes and cameras.

This module only draws inputs; it holds none of the renderer's arithmetic.
Both the GPU renderer's tests and the CPU oracle take their inputs from here.

The trained scenes of the paper's evaluation (Mip-NeRF 360, Tanks & Temples,
Deep Blending, Sec. I) are not available, so these seeded scenes stand in for
them with the same attribute layout: 3D mean, activated per-axis scale, unit
quaternion (w, x, y, z), activated opacity and degree-3 spherical harmonics
(16 coefficients x 3 channels, coefficient index k = l^2 + l + m).

Recipes (numpy PCG64(seed), draws in the order listed):
  tiny      N means ~ U[-1,1]^3; log-scale ~ N(-4, 0.5) per axis.
  clustered 90 % of N in 20 Gaussian clusters (centres ~ U[-1.5,1.5]^3,
            isotropic std ~ U(0.05, 0.4), weights ~ Dirichlet(1)), 10 % on a
            shell of radius 50 (1 + N(0, 0.01)) with uniform directions;
            log-scale ~ N(-4.5, 0.8) per axis.
  all       quaternion = normalise(N(0,1)^4); opacity = sigmoid(N(0, 1.5));
            SH DC ~ N(0.5, 0.2) per channel, the other 45 ~ N(0, 0.3).
Cameras look along +z with x right and y down (world -> camera R, t).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    means: np.ndarray      # [N,3] float32
    scales: np.ndarray     # [N,3] float32, activated (exp of log-scale)
    quats: np.ndarray      # [N,4] float32, (w, x, y, z), unit length
    opacities: np.ndarray  # [N]   float32, in (0, 1)
    sh: np.ndarray         # [N,16,3] float32
    sh_degree: int = 3

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.opacities[idx].copy(), self.sh[idx].copy(), self.sh_degree)


@dataclass
class Camera:
    R: np.ndarray          # [9] float32 world->camera rotation, row-major
    t: np.ndarray          # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float
    zfar: float
    bg: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=np.float32))


def _attributes(rng: np.random.Generator, n: int, log_mu: float, log_sigma: float):
    scales = np.exp(rng.normal(log_mu, log_sigma, size=(n, 3))).astype(np.float32)
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    quats = q.astype(np.float32)
    opac = (1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.5, size=n)))).astype(np.float32)
    sh = np.empty((n, 16, 3), dtype=np.float32)
    sh[:, 0, :] = rng.normal(0.5, 0.2, size=(n, 3))
    sh[:, 1:, :] = rng.normal(0.0, 0.3, size=(n, 15, 3))
    return scales, quats, opac, sh


def tiny_scene(n: int = 10_000, seed: int = 0) -> Scene:
    """Uniform cube scene (10k Gaussians at 256x256 in the tiny configuration)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    scales, quats, opac, sh = _attributes(rng, n, -4.0, 0.5)
    return Scene(means, scales, quats, opac, sh)


def clustered_scene(n: int, seed: int) -> Scene:
    """20 Gaussian clusters plus a far background shell of radius 50."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_shell = n // 10
    n_cl = n - n_shell
    centres = rng.uniform(-1.5, 1.5, size=(20, 3))
    stds = rng.uniform(0.05, 0.4, size=20)
    weights = rng.dirichlet(np.ones(20))
    which = rng.choice(20, size=n_cl, p=weights)
    pts = centres[which] + rng.normal(0.0, 1.0, size=(n_cl, 3)) * stds[which, None]
    d = rng.normal(0.0, 1.0, size=(n_shell, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    radius = 50.0 * (1.0 + rng.normal(0.0, 0.01, size=n_shell))
    shell = d * radius[:, None]
    means = np.concatenate([pts, shell], axis=0).astype(np.float32)
    scales, quats, opac, sh = _attributes(rng, n, -4.5, 0.8)
    return Scene(means, scales, quats, opac, sh)


def look_at_camera(position, width: int, height: int, hfov_deg: float = 60.0,
                   znear: float = 0.2, zfar: float = 100.0, target=(0.0, 0.0, 0.0), bg=(0.0, 0.0, 0.0)) -> Camera:
    """Pinhole camera at `position` looking at `target`, world y pointing down in the image."""
    c = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ c
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return Camera(R=R.reshape(9).astype(np.float32), t=t.astype(np.float32), fx=float(np.float32(fx)),
                  fy=float(np.float32(fx)), cx=(width - 1) / 2.0, cy=(height - 1) / 2.0, width=int(width),
                  height=int(height), znear=float(np.float32(znear)), zfar=float(np.float32(zfar)),
                  bg=np.asarray(bg, dtype=np.float32))


def orbit_camera(k: int, width: int, height: int, radius: float = 4.0, elevation_deg: float = 15.0,
                 step_deg: float = 12.0, znear: float = 0.2, zfar: float = 56.5, bg=(0.0, 0.0, 0.0)) -> Camera:
    """Pose k of the orbit: azimuth step_deg * k, camera above the scene (world -y is up)."""
    az = math.radians(step_deg * k)
    el = math.radians(elevation_deg)
    pos = (radius * math.cos(el) * math.sin(az), -radius * math.sin(el), -radius * math.cos(el) * math.cos(az))
    return look_at_camera(pos, width, height, 60.0, znear, zfar, bg=bg)


def tiny_camera(width: int = 256, height: int = 256, bg=(0.0, 0.0, 0.0)) -> Camera:
    """The tiny configuration's camera: distance 3 on the -z axis, hfov 60 deg, z in (0.2, 3 + sqrt 3]."""
    return look_at_camera((0.0, 0.0, -3.0), width, height, 60.0, 0.2, 3.0 + math.sqrt(3.0), bg=bg)


# Workloads: name -> (scene factory, camera factory, description)
WORKLOADS = {
    "tiny_256": dict(n=10_000, seed=0, width=256, height=256,
                     desc="10k Gaussians in [-1,1]^3, 256x256, 16x16 tiles"),
    "clustered_1080p": dict(n=500_000, seed=1, width=1920, height=1080,
                            desc="500k Gaussians, 20 clusters + shell r=50, 1920x1080, orbit pose 0"),
    "clustered_4k": dict(n=3_000_000, seed=2, width=3840, height=2160,
                         desc="3M Gaussians, 20 clusters + shell r=50, 3840x2160, 30 orbit poses"),
}


def workload(name: str, n: int | None = None):
    """(scene, [cameras]) of a named workload; n overrides the Gaussian count."""
    w = WORKLOADS[name]
    if name == "tiny_256":
        return tiny_scene(n or w["n"], w["seed"]), [tiny_camera(w["width"], w["height"])]
    scene = clustered_scene(n or w["n"], w["seed"])
    poses = 1 if name == "clustered_1080p" else 30
    return scene, [orbit_camera(k, w["width"], w["height"]) for k in range(poses)]


def prune_by_footprint(scene: Scene, keep: float) -> Scene:
    """Keep the fraction `keep` of the Gaussians with the largest o * s1 * s2
    (opacity times the area spanned by the two largest axes), in their original
    order: a synthetic stand-in for a learned pruning method, used to check that
    the renderer's savings compose with pruning."""
    s = np.sort(scene.scales, axis=1)
    score = scene.opacities * s[:, 2] * s[:, 1]
    k = max(1, int(round(keep * scene.n)))
    idx = np.sort(np.argsort(-score, kind="stable")[:k])
    return scene.subset(idx)

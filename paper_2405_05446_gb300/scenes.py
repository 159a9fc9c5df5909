"""Seeded synthetic inputs: gradient-Gaussian scenes and pinhole cameras.

This module only draws inputs. It holds none of the method's arithmetic
(no covariance, projection Jacobian, compositing or Poisson step), so both the
CUDA path and the FP64 oracle can be fed from it without sharing code.

Layouts (all float32, C-contiguous, structure of arrays):
  mean    [N][3]   world-space centre tau_k               (Eq. 3dgs / Eq. gdgs)
  scale   [N][3]   linear per-axis scale, S = diag(scale)  (Sigma = R S S^T R^T)
  quat    [N][4]   rotation as (w, x, y, z), not necessarily unit length
  opacity [N]      alpha_k in (0, 1)
  grad    [N][C][2] per-channel image-gradient attribute (gx, gy)

Cameras follow the OpenCV convention (x right, y down, z forward); the
world-to-camera transform is a row-major 3x4 matrix [R | t].

The recipes mirror the workloads the paper trains on (edge-concentrated sparse
splats; particle counts 1e3..1e6, Table 2) with seeded random draws instead of
the paper's datasets, which are not available here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Scene:
    mean: np.ndarray
    scale: np.ndarray
    quat: np.ndarray
    opacity: np.ndarray
    grad: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    @property
    def channels(self) -> int:
        return int(self.grad.shape[1])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(*(np.ascontiguousarray(a[idx]) for a in
                       (self.mean, self.scale, self.quat, self.opacity, self.grad)))

    def astype(self, dtype) -> "Scene":
        return Scene(*(np.ascontiguousarray(a, dtype=dtype) for a in
                       (self.mean, self.scale, self.quat, self.opacity, self.grad)))


@dataclasses.dataclass
class Camera:
    world_to_cam: np.ndarray  # (3, 4) float32
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    width: int
    height: int


def look_at_camera(eye, target, width: int, height: int, hfov_deg: float = 50.0,
                   near: float = 0.2, up=(0.0, 1.0, 0.0)) -> Camera:
    """Pinhole camera at `eye` looking at `target`, world `up` mapped to image up.

    fx = fy = (width / 2) / tan(hfov / 2); principal point at the image centre.
    """
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    up = np.asarray(up, dtype=np.float64)
    z = target - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, up)
    if np.linalg.norm(x) < 1e-8:  # looking along `up`: pick another reference
        x = np.cross(z, np.array([0.0, 0.0, 1.0]))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    rot = np.stack([x, y, z], axis=0)
    t = -rot @ eye
    w2c = np.concatenate([rot, t[:, None]], axis=1).astype(np.float32)
    f = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return Camera(w2c, float(f), float(f), width / 2.0, height / 2.0, float(near),
                  int(width), int(height))


def tiny_camera(width: int = 64, height: int = 64) -> Camera:
    """Camera at distance 3 on the -z axis looking at the origin, fov 50 deg."""
    return look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), width, height)


def metric_camera(width: int = 1920, height: int = 1080) -> Camera:
    """The 1920x1080 view of the primitive scenes (same pose as `tiny_camera`)."""
    return look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), width, height)


def ring_cameras(n_views: int = 8, radius: float = 3.0, width: int = 1280,
                 height: int = 720) -> list[Camera]:
    """Cameras evenly spaced on a ring of `radius` in the xz-plane, facing the origin."""
    cams = []
    for v in range(n_views):
        a = 2.0 * math.pi * v / n_views
        eye = (radius * math.sin(a), 0.0, -radius * math.cos(a))
        cams.append(look_at_camera(eye, (0.0, 0.0, 0.0), width, height))
    return cams


def sphere_camera(rng: np.random.Generator, width: int, height: int,
                  radius: float = 3.0) -> Camera:
    """Camera at a uniformly random point on the sphere of `radius`, facing the origin."""
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    return look_at_camera(radius * d, (0.0, 0.0, 0.0), width, height)


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def tiny_scene(seed: int = 0, n: int = 1000, channels: int = 3,
               grad_scale: float = 0.05) -> Scene:
    """Uniform cloud: means U[-1,1]^3, log-scales N(-3, 0.5), opacities U[0.2,0.9],
    gradients i.i.d. Laplace(0, grad_scale)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mean = rng.uniform(-1.0, 1.0, (n, 3))
    scale = np.exp(rng.normal(-3.0, 0.5, (n, 3)))
    quat = _unit_quats(rng, n)
    opacity = rng.uniform(0.2, 0.9, n)
    grad = rng.laplace(0.0, grad_scale, (n, channels, 2))
    return Scene(mean, scale, quat, opacity, grad).astype(np.float32)


def _image_direction(cam: Camera, p: np.ndarray, nrm: np.ndarray,
                     rng: np.random.Generator) -> np.ndarray:
    """Unit image-plane direction in which the surface normal `nrm` at `p` points.

    Found by mapping p and p + eps*nrm through the pinhole camera and normalising
    the pixel displacement; random where the displacement vanishes.
    """
    w2c = cam.world_to_cam.astype(np.float64)

    def pix(q):
        c = q @ w2c[:, :3].T + w2c[:, 3]
        z = np.where(np.abs(c[:, 2]) < 1e-9, 1e-9, c[:, 2])
        return np.stack([cam.fx * c[:, 0] / z, cam.fy * c[:, 1] / z], axis=1)

    eps = 1e-4
    d = pix(p + eps * nrm) - pix(p)
    ln = np.linalg.norm(d, axis=1, keepdims=True)
    bad = ln[:, 0] < 1e-6 * eps * cam.fx
    rnd = rng.standard_normal((p.shape[0], 2))
    rnd /= np.linalg.norm(rnd, axis=1, keepdims=True)
    out = np.where(bad[:, None], rnd, d / np.maximum(ln, 1e-30))
    return out


def primitives_scene(seed: int = 0, n: int = 200_000, n_prims: int = 20,
                     channels: int = 3, grad_scale: float = 0.1,
                     log_scale_mu: float = -5.0, log_scale_sigma: float = 0.7,
                     surface_fraction: float = 0.9,
                     orient_camera: Camera | None = None) -> Scene:
    """Edge-concentrated scene: Gaussians on the surfaces of random boxes and spheres.

    `n_prims` primitives, each a sphere or an axis-aligned cube with p = 1/2, centre
    U[-0.6, 0.6]^3, radius / half-extent U[0.05, 0.25]. A `surface_fraction` of the
    Gaussians are area-weighted uniform samples on the primitive surfaces (normal =
    surface normal); the rest are uniform in [-1,1]^3 with random normals. Scales are
    log-normal(log_scale_mu, log_scale_sigma) per axis, rotations uniform, opacities
    U[0.2, 0.9]. Per Gaussian and channel a magnitude m ~ Laplace(0, grad_scale) is
    drawn and the gradient is m times the unit image-plane direction of the normal as
    seen by `orient_camera` (default: the 1920x1080 metric camera).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = orient_camera if orient_camera is not None else metric_camera()
    is_sphere = rng.random(n_prims) < 0.5
    centre = rng.uniform(-0.6, 0.6, (n_prims, 3))
    size = rng.uniform(0.05, 0.25, n_prims)
    area = np.where(is_sphere, 4.0 * math.pi * size ** 2, 24.0 * size ** 2)

    n_surf = int(round(surface_fraction * n))
    n_bg = n - n_surf
    prim = rng.choice(n_prims, size=n_surf, p=area / area.sum())
    pos = np.empty((n_surf, 3))
    nrm = np.empty((n_surf, 3))
    # spheres: uniform direction
    dirs = rng.standard_normal((n_surf, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    # cubes: uniform face, uniform point on the face
    face = rng.integers(0, 6, n_surf)
    uv = rng.uniform(-1.0, 1.0, (n_surf, 2))
    axis = face // 2
    sign = np.where(face % 2 == 0, 1.0, -1.0)
    cube_local = np.empty((n_surf, 3))
    cube_nrm = np.zeros((n_surf, 3))
    for a in range(3):
        o1, o2 = [b for b in range(3) if b != a]
        sel = axis == a
        cube_local[sel, a] = sign[sel]
        cube_local[sel, o1] = uv[sel, 0]
        cube_local[sel, o2] = uv[sel, 1]
        cube_nrm[sel, a] = sign[sel]
    sph = is_sphere[prim]
    r = size[prim][:, None]
    pos[:] = np.where(sph[:, None], centre[prim] + r * dirs, centre[prim] + r * cube_local)
    nrm[:] = np.where(sph[:, None], dirs, cube_nrm)

    bg_pos = rng.uniform(-1.0, 1.0, (n_bg, 3))
    bg_nrm = rng.standard_normal((n_bg, 3))
    bg_nrm /= np.linalg.norm(bg_nrm, axis=1, keepdims=True)
    mean = np.concatenate([pos, bg_pos], axis=0)
    normal = np.concatenate([nrm, bg_nrm], axis=0)

    scale = np.exp(rng.normal(log_scale_mu, log_scale_sigma, (n, 3)))
    quat = _unit_quats(rng, n)
    opacity = rng.uniform(0.2, 0.9, n)
    mag = rng.laplace(0.0, grad_scale, (n, channels))
    d = _image_direction(cam, mean, normal, rng)
    grad = mag[:, :, None] * d[:, None, :]
    # shuffle so that surface and background Gaussians are interleaved in memory
    perm = rng.permutation(n)
    return Scene(mean[perm], scale[perm], quat[perm], opacity[perm],
                 grad[perm]).astype(np.float32)


def image_from_gradients_test_image(h: int, w: int, seed: int = 0) -> np.ndarray:
    """A known FP64 test image (smooth part plus white noise) of shape (h, w)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    smooth = 0.5 + 0.3 * np.sin(2 * math.pi * xx / max(w, 2)) * np.cos(math.pi * yy / max(h, 2))
    return smooth + 0.05 * rng.standard_normal((h, w))


def with_laplacian_attribute(scene: Scene, seed: int = 0, value_scale: float = 0.05) -> Scene:
    """The same Gaussians carrying one Laplacian value per channel (the A_k of Eq. gdgs,
    drawn i.i.d. Laplace(0, value_scale)) instead of a gradient."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    vals = rng.laplace(0.0, value_scale, (scene.n, scene.channels))
    return Scene(scene.mean, scene.scale, scene.quat, scene.opacity,
                 np.ascontiguousarray(vals, dtype=np.float32))


# Named workloads -----------------------------------------------------------------

def workload(name: str):
    """Returns (scene, camera, per-channel mean, solver rtol) of a named workload."""
    if name == "tiny64":
        return tiny_scene(0), tiny_camera(), np.full(3, 0.5), 1e-6
    if name == "prims1080p":
        return primitives_scene(0), metric_camera(), np.full(3, 0.5), 1e-6
    if name == "lap1080p":
        sc, cam, mean, rtol = workload("prims1080p")
        return with_laplacian_attribute(sc), cam, mean, rtol
    if name == "prims4k":
        cam = metric_camera(3840, 2160)
        return (primitives_scene(0, n=1_000_000, n_prims=50, orient_camera=cam), cam,
                np.full(3, 0.5), 1e-6)
    raise KeyError(name)

"""FP64 CPU oracle for the GDGS view-synthesis path.

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
reference the CUDA path is checked against. Only the tests, the smoke check and
the CPU-baseline leg of the benchmark may import it; the product path never
does, and it imports nothing from the product package.

What it computes, step by step, all in float64:
  project           Sigma = R S S^T R^T (Sec. 1.2, Eq. 3dgs), camera transform,
                    Sigma2D = J W Sigma W^T J^T (Eq. sig2d and Sec. 2.2 "Projection")
  render_gradients  front-to-back alpha composite of the gradient attribute in
                    view-depth order (Eq. color, Eq. gdgs2d)
  divergence        rho = div(g): the Laplacian field is the divergence of the
                    gradient field (Sec. 1.5 "Sparsity", Sec. 2.1 "Poisson Equation")
  poisson_neumann   the exact solution of the discrete Neumann Poisson problem
                    Delta c = rho (Eq. p2d) by the DCT-II, which diagonalises the
                    Neumann 5-point Laplacian; the constant left free by the
                    Neumann problem (Sec. 2.1, "with possible constant difference")
                    is fixed by a supplied per-channel mean
  threshold         the hard threshold T of Eq. thresh
  render_view       the three render steps of Algorithm 1 in order, for gradient
                    Gaussians (divergence first) or Laplacian Gaussians (Eq. gdgs)

Parity against values printed in the paper is unpinned for the whole pipeline:
the paper prints no worked example. Each function is pinned instead by closed
forms, brute force and invariants in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_raster.c")
_LIB = os.path.join(_HERE, "_oracle_raster.so")
_lib = None

# column indices of a projected-Gaussian row (mirrors the enum in oracle_raster.c)
(VALID, DEPTH, MX, MY, CA, CB, CC, OPA, XMIN, XMAX, YMIN, YMAX, S00, S01, S11, DERR, KAPPA,
 GHOST, NEARAMB, BOXW, TZ0, TZ1, TZ2, LMAX) = range(24)
STRIDE = 24


@dataclasses.dataclass
class RasterOpts:
    """Readings of points the paper leaves open (paper-literal exponent by default)."""
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    dilation: float = 0.3
    exp_coef: float = 1.0


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        lib.oracle_project.argtypes = [ctypes.c_int64, p, p, p, p, p, p, p]
        lib.oracle_project.restype = None
        lib.oracle_composite.argtypes = [p, p, ctypes.c_int, p, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, p, p,
                                         ctypes.c_int64, ctypes.c_int, p, p]
        lib.oracle_composite.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def camera_array(cam) -> np.ndarray:
    """The camera as the float32 values the C ABI's gdgs_camera carries (pose,
    intrinsics, near plane), promoted to float64 like every other input."""
    w = np.asarray(cam.world_to_cam, dtype=np.float32).reshape(12)
    intr = np.array([cam.fx, cam.fy, cam.cx, cam.cy, cam.near], dtype=np.float32)
    return np.concatenate([w, intr]).astype(np.float64)


# relative precision of a plain float32 evaluation of the depth w20 x + w21 y + w22 z + w23
DEPTH_REL_F32 = 4.0 * 2.0 ** -24 / (1.0 - 4.0 * 2.0 ** -24)


def project(scene, cam, opts: RasterOpts = RasterOpts(),
            depth_rel: float = DEPTH_REL_F32) -> np.ndarray:
    """Per-Gaussian projection rows [N][STRIDE] (Eq. 3dgs, Eq. sig2d).

    Culls: non-normalisable quaternion, camera-space depth <= near, det(Sigma2D) <= 0,
    opacity < alpha_min. Footprint box: the exact bounding box of the ellipse where
    opacity * exp(-exp_coef * d^T Sigma2D^-1 d) >= alpha_min.
    depth_rel: relative precision of the depth in the implementation under test (for
    the ambiguity flags only: depth errors up to depth_rel times the sum of the depth's
    term magnitudes can swap two Gaussians or flip the near cull).
    """
    lib = _load()
    mean, scale, quat, opa = (_f32(scene.mean), _f32(scene.scale), _f32(scene.quat),
                              _f32(scene.opacity))
    n = mean.shape[0]
    out = np.zeros((n, STRIDE), dtype=np.float64)
    camv = camera_array(cam)
    optv = np.array([opts.dilation, opts.exp_coef, opts.alpha_min, depth_rel], dtype=np.float64)
    lib.oracle_project(n, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(opa), _ptr(camv),
                       _ptr(optv), _ptr(out))
    return out


def depth_order(proj: np.ndarray, ghosts: bool = False) -> np.ndarray:
    """Valid Gaussians sorted front to back ("sorted from the view direction", Eq. color):
    ascending FP64 camera depth, equal depths by ascending index.

    ghosts=True also lists the Gaussians the near cull removed only within the float32
    error bound of the depth (see oracle_raster.c); the composite uses them for the
    ambiguity flag and nothing else.
    """
    keep = proj[:, VALID] > 0
    if ghosts:
        keep |= proj[:, GHOST] > 0
    idx = np.nonzero(keep)[0]
    return idx[np.lexsort((idx, proj[idx, DEPTH]))].astype(np.int64)


def render_gradients(scene, cam, opts: RasterOpts = RasterOpts(), mode: str = "box",
                     pixels=None, nthreads: int = 0, err_scale: float = 1.0, proj=None,
                     depth_rel: float = DEPTH_REL_F32):
    """Composite the per-Gaussian attributes front to back (Eq. gdgs2d, Eq. color).

    At pixel centre p: for each Gaussian k in depth order, G = exp(-exp_coef d^T conic d)
    with d = p - mean2d, a = min(alpha_max, alpha_k G); a < alpha_min is skipped;
    acc += c_k * a * T; T *= (1 - a); stop once T < t_min.

    The attribute c_k is scene.grad: [N][C][2] gradients (gx, gy) or [N][C] Laplacian
    values (Eq. gdgs). mode "all_pairs" visits every Gaussian at every pixel (the plain
    definition); mode "box" skips Gaussians whose footprint box misses the pixel (same
    result). Returns (maps, ambiguous): maps [C][2][H][W] or [C][H][W] (or [P][C][2] /
    [P][C] for a pixel list), ambiguous a uint8 flag per pixel: one of the discontinuous
    decisions (near cull, depth order of two contributing Gaussians, alpha vs alpha_min,
    T vs T_min) lies within its float32 error bound of the threshold (oracle_raster.c
    derives the bounds; err_scale multiplies them, 0 turns the flags off).
    """
    lib = _load()
    if proj is None:
        proj = project(scene, cam, opts, depth_rel)
    grad = _f32(scene.grad)
    C = grad.shape[1]
    K = grad.shape[2] if grad.ndim == 3 else 1
    Q = C * K
    order = depth_order(proj, ghosts=True)
    W, H = cam.width, cam.height
    optv = np.array([opts.exp_coef, opts.alpha_min, opts.alpha_max, opts.t_min, err_scale],
                    dtype=np.float64)
    use_box = 1 if mode == "box" else 0
    if mode not in ("box", "all_pairs"):
        raise ValueError(mode)
    if pixels is None:
        out = np.zeros((H * W, Q), dtype=np.float64)
        amb = np.zeros(H * W, dtype=np.uint8)
        lib.oracle_composite(_ptr(proj), _ptr(grad), Q, _ptr(order), order.shape[0], W, H,
                             use_box, _ptr(optv), None, 0, nthreads, _ptr(out), _ptr(amb))
        if K == 2:
            maps = out.reshape(H, W, C, 2).transpose(2, 3, 0, 1).copy()
        else:
            maps = out.reshape(H, W, C).transpose(2, 0, 1).copy()
        return maps, amb.reshape(H, W)
    pix = np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.zeros((pix.shape[0], Q), dtype=np.float64)
    amb = np.zeros(pix.shape[0], dtype=np.uint8)
    lib.oracle_composite(_ptr(proj), _ptr(grad), Q, _ptr(order), order.shape[0], W, H,
                         use_box, _ptr(optv), _ptr(pix), pix.shape[0], nthreads, _ptr(out),
                         _ptr(amb))
    return (out.reshape(-1, C, 2) if K == 2 else out.reshape(-1, C)), amb


def threshold(rho: np.ndarray, t: float) -> np.ndarray:
    """T(x) = x if |x| >= t else 0, elementwise (Eq. thresh)."""
    rho = np.asarray(rho, dtype=np.float64)
    return np.where(np.abs(rho) >= t, rho, 0.0)


def divergence(maps: np.ndarray) -> np.ndarray:
    """rho = div(gx, gy) with zero flux through the image border.

    gx(i, j) is the flux through the face between pixels (i, j) and (i, j+1), gy(i, j)
    the one between (i, j) and (i+1, j); fluxes on border faces are dropped, so
    rho(i,j) = [j<W-1] gx(i,j) - [j>=1] gx(i,j-1) + [i<H-1] gy(i,j) - [i>=1] gy(i-1,j).
    For forward-difference gradients of an image I this is exactly the Neumann
    5-point Laplacian of I, and sum(rho) = 0.
    """
    maps = np.asarray(maps, dtype=np.float64)
    gx, gy = maps[:, 0], maps[:, 1]
    rho = np.zeros_like(gx)
    rho[:, :, :-1] += gx[:, :, :-1]
    rho[:, :, 1:] -= gx[:, :, :-1]
    rho[:, :-1, :] += gy[:, :-1, :]
    rho[:, 1:, :] -= gy[:, :-1, :]
    return rho


def forward_gradients(img: np.ndarray) -> np.ndarray:
    """Forward differences of a [C][H][W] image into [C][2][H][W] maps
    (last column of gx and last row of gy are zero: those faces are on the border)."""
    img = np.asarray(img, dtype=np.float64)
    g = np.zeros((img.shape[0], 2) + img.shape[1:], dtype=np.float64)
    g[:, 0, :, :-1] = img[:, :, 1:] - img[:, :, :-1]
    g[:, 1, :-1, :] = img[:, 1:, :] - img[:, :-1, :]
    return g


def laplacian_neumann(u: np.ndarray) -> np.ndarray:
    """L_N u (i,j) = sum over in-grid 4-neighbours n of (u_n - u_ij), per channel."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    out[..., :, :-1] += u[..., :, 1:] - u[..., :, :-1]
    out[..., :, 1:] += u[..., :, :-1] - u[..., :, 1:]
    out[..., :-1, :] += u[..., 1:, :] - u[..., :-1, :]
    out[..., 1:, :] += u[..., :-1, :] - u[..., 1:, :]
    return out


def dct_matrix(n: int) -> np.ndarray:
    """Orthonormal DCT-II matrix D[k, j] = s_k cos(pi k (2j+1) / (2n))."""
    k = np.arange(n, dtype=np.float64)[:, None]
    j = np.arange(n, dtype=np.float64)[None, :]
    d = np.cos(np.pi * k * (2.0 * j + 1.0) / (2.0 * n))
    d *= np.sqrt(2.0 / n)
    d[0, :] = np.sqrt(1.0 / n)
    return d


def poisson_neumann(rho: np.ndarray, mean) -> np.ndarray:
    """Solve L_N u = rho exactly (Eq. p2d, Neumann boundary), then set mean(u_c) = m_c.

    The DCT-II diagonalises L_N: the 1D Neumann second difference has eigenvectors
    cos(pi k (j + 1/2) / n) with eigenvalues 2 cos(pi k / n) - 2. The (0, 0) mode is the
    constant the Neumann problem leaves free; it is set to zero and the supplied mean
    added afterwards. If sum(rho) != 0 this is the least-squares solution.
    """
    rho = np.asarray(rho, dtype=np.float64)
    C, H, W = rho.shape
    dh, dw = dct_matrix(H), dct_matrix(W)
    lam = ((2.0 * np.cos(np.pi * np.arange(H) / H) - 2.0)[:, None]
           + (2.0 * np.cos(np.pi * np.arange(W) / W) - 2.0)[None, :])
    lam[0, 0] = 1.0
    mean = np.broadcast_to(np.asarray(mean, dtype=np.float64), (C,))
    out = np.empty_like(rho)
    for c in range(C):
        rh = dh @ rho[c] @ dw.T
        uh = rh / lam
        uh[0, 0] = 0.0
        u = dh.T @ uh @ dw
        out[c] = u + (mean[c] - u.mean())
    return out


def render_view(scene, cam, mean, opts: RasterOpts = RasterOpts(), nthreads: int = 0,
                rho_threshold: float = 0.0, depth_rel: float = DEPTH_REL_F32):
    """Algorithm 1's render steps: project + composite (Eq. gdgs2d), the Laplacian field
    (the divergence of gradient maps, or the composite itself for Laplacian Gaussians,
    Eq. gdgs), the hard threshold T when rho_threshold > 0 (Eq. thresh), and the Neumann
    Poisson solve (Eq. p2d) with the constant fixed by `mean`.
    Returns (image [C][H][W], maps, ambiguous [H][W])."""
    maps, amb = render_gradients(scene, cam, opts, mode="box", nthreads=nthreads,
                                 depth_rel=depth_rel)
    rho = divergence(maps) if maps.ndim == 4 else maps
    if rho_threshold > 0:
        rho = threshold(rho, rho_threshold)
    img = poisson_neumann(rho, mean)
    return img, maps, amb

"""Differentiable FP64 oracle of the view-synthesis path (plain PyTorch CPU ops).

TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`: it checks the gradients of
the CUDA path and is never imported by the product package.

The forward is the same definition as the C oracle, written with torch float64
tensors so that autograd gives its exact gradient:
  projection   Sigma = R S S^T R^T (Eq. 3dgs), t = W mu + w, J the Jacobian of the
               pinhole map at t, Sigma2D = J W Sigma W^T J^T + dil I (Eq. sig2d),
               conic = Sigma2D^-1, centre (fx t_x / t_z + c_x, fy t_y / t_z + c_y)
  composite    per pixel, Gaussians front to back: a = min(alpha_max, opacity *
               exp(-k d^T conic d)); a < alpha_min is skipped; the weight is a T
               with T the product of (1 - a) over the Gaussians before; once T
               falls below T_min the rest are not visited (Eq. gdgs2d)
  field        rho = div(maps) with zero border flux, or the composite itself for
               Laplacian Gaussians (Eq. gdgs); hard threshold T (Eq. thresh)
  solve        the exact Neumann solve by the DCT-II with the mean of rho removed
               (least squares), then the supplied per-channel mean (Eq. p2d)
The integer decisions (which Gaussians survive the culls, their depth order, and
per pixel which Gaussians pass the alpha_min test and whether the T_min stop has
happened) are taken exactly as in the C oracle; their derivative is zero almost
everywhere. With alpha_min tiny, t_min = 0 and opacities below alpha_max the map
is smooth, which is how the finite-difference pins use it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import RasterOpts, camera_array, dct_matrix, depth_order, project

PARAMS = ("mean", "scale", "quat", "opacity", "grad")


def scene_params(scene, requires_grad: bool = True) -> dict:
    """The Gaussians' parameters as float64 leaf tensors (the float32 values promoted)."""
    out = {}
    for k in PARAMS:
        t = torch.tensor(np.asarray(getattr(scene, k), dtype=np.float64))
        out[k] = t.requires_grad_(requires_grad)
    return out


def _project(p: dict, cam, opts: RasterOpts, idx: torch.Tensor):
    camv = torch.tensor(camera_array(cam), dtype=torch.float64)
    w = camv[:12].reshape(3, 4)
    fx, fy, cx, cy = camv[12], camv[13], camv[14], camv[15]
    q = p["quat"][idx]
    q = q / q.norm(dim=1, keepdim=True)
    qw, qx, qy, qz = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = torch.stack([
        torch.stack([1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)], -1),
        torch.stack([2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)], -1),
        torch.stack([2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)], -1),
    ], 1)
    s = p["scale"][idx]
    Sig = R @ torch.diag_embed(s * s) @ R.transpose(1, 2)
    t = p["mean"][idx] @ w[:, :3].T + w[:, 3]
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    z = torch.zeros_like(tz)
    J = torch.stack([torch.stack([fx / tz, z, -fx * tx / (tz * tz)], -1),
                     torch.stack([z, fy / tz, -fy * ty / (tz * tz)], -1)], 1)
    T = J @ w[:, :3]
    S2 = T @ Sig @ T.transpose(1, 2) + opts.dilation * torch.eye(2, dtype=torch.float64)
    det = S2[:, 0, 0] * S2[:, 1, 1] - S2[:, 0, 1] * S2[:, 1, 0]
    ca, cb, cc = S2[:, 1, 1] / det, -S2[:, 0, 1] / det, S2[:, 0, 0] / det
    mx, my = fx * tx / tz + cx, fy * ty / tz + cy
    return mx, my, ca, cb, cc


def composite(p: dict, scene, cam, opts: RasterOpts) -> torch.Tensor:
    """The composited attribute planes [Q][H][W] (Eq. gdgs2d), Q = grad.shape[1]."""
    proj = project(scene, cam, opts)
    order = torch.tensor(depth_order(proj), dtype=torch.int64)
    H, W = cam.height, cam.width
    Q = int(np.prod(p["grad"].shape[1:]))
    if order.numel() == 0:
        return torch.zeros((Q, H, W), dtype=torch.float64)
    mx, my, ca, cb, cc = _project(p, cam, opts, order)
    yy, xx = torch.meshgrid(torch.arange(H, dtype=torch.float64) + 0.5,
                            torch.arange(W, dtype=torch.float64) + 0.5, indexing="ij")
    dx = xx.reshape(-1, 1) - mx[None, :]
    dy = yy.reshape(-1, 1) - my[None, :]
    power = opts.exp_coef * (ca * dx * dx + 2.0 * cb * dx * dy + cc * dy * dy)
    a = p["opacity"][order][None, :] * torch.exp(-power)
    a = torch.clamp(a, max=opts.alpha_max)
    keep = (a >= opts.alpha_min).to(torch.float64).detach()
    a = a * keep
    one = torch.ones((a.shape[0], 1), dtype=torch.float64)
    T = torch.cat([one, torch.cumprod(1.0 - a, dim=1)[:, :-1]], dim=1)
    live = (T >= opts.t_min).to(torch.float64).detach()  # the T_min stop (T before the splat)
    wgt = a * T * live
    maps = wgt @ p["grad"][order].reshape(order.numel(), Q)
    return maps.T.reshape(Q, H, W)


def divergence(maps: torch.Tensor) -> torch.Tensor:
    """rho from [C][2][H][W] gradient planes, zero flux through the border."""
    gx, gy = maps[:, 0], maps[:, 1]
    rho = torch.zeros_like(gx)
    rho[:, :, :-1] = rho[:, :, :-1] + gx[:, :, :-1]
    rho[:, :, 1:] = rho[:, :, 1:] - gx[:, :, :-1]
    rho[:, :-1, :] = rho[:, :-1, :] + gy[:, :-1, :]
    rho[:, 1:, :] = rho[:, 1:, :] - gy[:, :-1, :]
    return rho


def poisson_neumann(rho: torch.Tensor, mean) -> torch.Tensor:
    """The exact Neumann solve by the DCT-II (its (0,0) mode dropped: least squares
    for a rho whose sum is not zero), then mean(u_c) = mean_c (Eq. p2d)."""
    C, H, W = rho.shape
    dh = torch.tensor(dct_matrix(H))
    dw = torch.tensor(dct_matrix(W))
    lam = ((2.0 * torch.cos(torch.pi * torch.arange(H, dtype=torch.float64) / H) - 2.0)[:, None]
           + (2.0 * torch.cos(torch.pi * torch.arange(W, dtype=torch.float64) / W) - 2.0)[None, :])
    lam[0, 0] = 1.0
    zero00 = torch.ones((H, W), dtype=torch.float64)
    zero00[0, 0] = 0.0
    out = []
    for c in range(C):
        uh = (dh @ rho[c] @ dw.T) / lam * zero00
        u = dh.T @ uh @ dw
        out.append(u + (float(mean[c]) - u.mean()))
    return torch.stack(out)


def render_view(p: dict, scene, cam, mean, opts: RasterOpts, rho_threshold: float = 0.0):
    """Algorithm 1's render steps as a differentiable FP64 function of the parameters."""
    maps = composite(p, scene, cam, opts)
    C = scene.channels
    if p["grad"].dim() == 3:  # [n][C][2]: gradient attribute
        rho = divergence(maps.reshape(C, 2, cam.height, cam.width))
    else:
        rho = maps
    if rho_threshold > 0:
        rho = rho * (rho.abs() >= rho_threshold).to(torch.float64).detach()
    return poisson_neumann(rho, mean)


def gradients(scene, cam, mean, opts: RasterOpts, d_image: np.ndarray, rho_threshold: float = 0.0):
    """d(sum(d_image * image))/d(parameters), float64 numpy arrays keyed like PARAMS."""
    p = scene_params(scene)
    img = render_view(p, scene, cam, mean, opts, rho_threshold)
    (img * torch.tensor(d_image, dtype=torch.float64)).sum().backward()
    return {k: p[k].grad.numpy().copy() for k in PARAMS}

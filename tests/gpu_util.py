"""Helpers shared by the GPU tests: build/load the library, run the CUDA path
through the C ABI, and compare with the FP64 oracle under the stated tolerances.

Tolerances (floating point):
  gradient maps  max |gpu - oracle| over non-ambiguous pixels <= 1e-5 * max |oracle|;
                 ambiguous pixels (a decision within its float32 error bound of the
                 threshold, see oracle_raster.c) are at most AMB_FRAC_MAX of all pixels
  image          max |gpu - oracle| <= 1e-3 absolute for rendered views (images near
                 [0, 1]); for solver tests on synthetic fields of arbitrary scale, and
                 for Laplacian-attribute views (whose least-squares images span
                 hundreds), 1e-3 after mapping the oracle image's range onto [0, 1]
"""
import numpy as np
import torch

import oracle as O
import paper_2405_05446_gb300 as G
from paper_2405_05446_gb300 import build as B

MAP_TOL = 1e-5
IMG_TOL = 1e-3
# measured with the oracle's float32 error model: 6.3e-4 of the 1080p workload's pixels
AMB_FRAC_MAX = 1e-3
# The library orders Gaussians by a float-float camera depth resolved to 2^-31 relative
# (include/gdgs.h, gdgs_camera); the oracle flags depth ties within 4x that.
LIB_DEPTH_REL = 2.0 ** -29


def ensure_lib():
    B.build()
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    G._abi.load()


def oracle_opts(ro) -> O.RasterOpts:
    """The oracle reads the same option values the kernel receives (float32)."""
    return O.RasterOpts(alpha_min=float(np.float32(ro.alpha_min)), alpha_max=float(np.float32(ro.alpha_max)),
                        t_min=float(np.float32(ro.t_min)), dilation=float(np.float32(ro.dilation)),
                        exp_coef=float(np.float32(ro.exp_coef)))


def oracle_maps(scene, cam, ro=None, **kw):
    """The oracle's composite for the options `ro` the kernel receives, with the depth
    ties flagged at the library's stated depth precision."""
    return O.render_gradients(scene, cam, oracle_opts(ro or G.raster_opts()),
                              depth_rel=LIB_DEPTH_REL, **kw)


def gpu_maps(scene, cam, ropts=None, with_mask=False):
    ropts = ropts or G.raster_opts()
    g = G.gaussians_to_device(scene)
    C = scene.channels
    nbytes = G.workspace_size(scene.n, C, cam.width, cam.height, ropts, None)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    shape = (C, cam.height, cam.width) if scene.grad.ndim == 2 else (C, 2, cam.height, cam.width)
    maps = torch.full(shape, float("nan"), device="cuda")
    mask = None
    if with_mask:
        mask = torch.zeros(((cam.height + 15) // 16, (cam.width + 15) // 16), dtype=torch.uint8, device="cuda")
    G.render_gradients(g, cam, maps, ws, mask=mask, ropts=ropts)
    st = G.sync_status(ws)
    return maps.cpu().numpy().astype(np.float64), (mask.cpu().numpy() if with_mask else None), st


def gpu_poisson(maps_np, mean, sopts=None, mask=None):
    C, _, H, W = maps_np.shape
    sopts = sopts or G.solver_opts()
    nbytes = G.workspace_size(0, C, W, H, None, sopts)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    maps = torch.as_tensor(np.ascontiguousarray(maps_np, dtype=np.float32)).cuda()
    m = torch.as_tensor(mask).cuda() if mask is not None else None
    img = torch.empty((C, H, W), device="cuda")
    G.poisson_reconstruct(maps, mean, img, ws, mask=m, sopts=sopts)
    st = G.sync_status(ws)
    return img.cpu().numpy().astype(np.float64), st


def map_rel_err(gpu, ora, amb):
    ok = amb == 0
    d = np.abs(gpu - ora)[:, :, ok]
    return float(d.max() / max(np.abs(ora).max(), 1e-30)) if d.size else 0.0


def img_err(gpu, ora):
    scale = max(1.0, float(ora.max() - ora.min()))
    return float(np.abs(gpu - ora).max() / scale), float(np.abs(gpu - ora).max())

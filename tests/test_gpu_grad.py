"""Gradients of the render path on the GPU (the library's backward kernels) against
the FP64 oracle gradient (oracle/diff.py, itself pinned to central differences):
64 Gaussians at 128 x 128, every parameter kind, gradient and Laplacian
attributes, with and without the hard threshold; and the autograd binding."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import diff as D
import paper_2405_05446_gb300 as G
from paper_2405_05446_gb300 import scenes as S
from gpu_util import ensure_lib

pytestmark = pytest.mark.gpu

SMOOTH = dict(alpha_min=float(np.float32(1e-10)), alpha_max=0.99, t_min=0.0)
GRAD_TOL = 1e-4  # max |gpu - oracle| <= GRAD_TOL * max |oracle|, per parameter kind (measured <= 1e-5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _scene64(seed=0, laplacian=False):
    sc = S.tiny_scene(seed, n=64)
    sc = S.Scene(sc.mean * 0.6, sc.scale * 1.6, sc.quat, np.minimum(sc.opacity, 0.9).astype(np.float32), sc.grad)
    if laplacian:
        sc = S.with_laplacian_attribute(sc)
    cam = S.look_at_camera((0.3, -0.2, -3.0), (0.0, 0.0, 0.0), 128, 128, hfov_deg=40)
    return sc, cam


def _gpu_grads(sc, cam, mean, w, ropts, sopts):
    g = G.gaussians_to_device(sc)
    C, H, W = sc.channels, cam.height, cam.width
    ws = torch.empty(G.workspace_size(sc.n, C, W, H, ropts, sopts), dtype=torch.uint8, device="cuda")
    ws_adj = torch.empty(G.workspace_size(0, C, W, H, None, sopts), dtype=torch.uint8, device="cuda")
    img = torch.empty((C, H, W), device="cuda")
    G.render_view(g, cam, mean, img, ws, ropts, sopts)
    st = G.sync_status(ws)
    assert st["status"] == 0, st
    gr = G.render_view_backward(g, cam, torch.as_tensor(w, dtype=torch.float32).cuda(), ws, ws_adj, ropts, sopts)
    sa = G.sync_status(ws_adj)
    assert sa["status"] == 0, sa
    return {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()}, img


def _compare(gpu, ref):
    for k in D.PARAMS:
        a, b = gpu[k].reshape(ref[k].shape), ref[k]
        scale = np.abs(b).max()
        err = np.abs(a - b).max()
        assert err <= GRAD_TOL * scale, (k, err, scale)


@pytest.mark.parametrize("laplacian", [False, True])
def test_gradients_match_oracle(laplacian):
    sc, cam = _scene64(1, laplacian)
    mean = [0.5, 0.5, 0.5]
    w = np.random.default_rng(7).standard_normal((3, cam.height, cam.width))
    ropts = G.raster_opts(pairs_per_gaussian=64, **SMOOTH)
    gpu, _ = _gpu_grads(sc, cam, mean, w, ropts, G.solver_opts(rtol=1e-7))
    ref = D.gradients(sc, cam, mean, O.RasterOpts(**SMOOTH), w)
    _compare(gpu, ref)


def test_gradients_through_the_threshold():
    """Laplacian field with the hard threshold T: t is chosen (from the oracle's
    field) so that no pixel's decision is within the composite error of t."""
    from test_gpu_parity import _well_posed_threshold
    sc, cam = _scene64(2, laplacian=True)
    mean = [0.5, 0.5, 0.5]
    rho, amb = O.render_gradients(sc, cam, O.RasterOpts(**SMOOTH))
    t = _well_posed_threshold(sc, rho, amb, [0.004 * (1 + 0.005 * i) for i in range(400)])
    assert t is not None and 0.1 < (np.abs(rho) < t).mean() < 0.9
    w = np.random.default_rng(8).standard_normal((3, cam.height, cam.width))
    ropts = G.raster_opts(pairs_per_gaussian=64, **SMOOTH)
    gpu, _ = _gpu_grads(sc, cam, mean, w, ropts, G.solver_opts(rtol=1e-7, rho_threshold=t))
    ref = D.gradients(sc, cam, mean, O.RasterOpts(**SMOOTH), w, rho_threshold=t)
    _compare(gpu, ref)


def test_autograd_function_and_descent():
    from paper_2405_05446_gb300 import autograd as A
    sc, cam = _scene64(3)
    mean = [0.5, 0.5, 0.5]
    ropts = G.raster_opts(pairs_per_gaussian=64, **SMOOTH)
    params = {k: torch.tensor(np.asarray(getattr(sc, k)), device="cuda", requires_grad=True)
              for k in D.PARAMS}
    target = A.render_view(*(params[k].detach() * (1.0 + 0.05 * (k == "grad")) for k in D.PARAMS),
                           cam, mean, ropts).detach()
    img = A.render_view(*(params[k] for k in D.PARAMS), cam, mean, ropts)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    direct, _ = _gpu_grads(sc, cam, mean, w.cpu().numpy(), ropts, G.solver_opts())
    for k in D.PARAMS:  # equal up to the order of the backward's atomic sums
        a, b = params[k].grad.cpu().numpy().reshape(-1), direct[k].reshape(-1)
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max(), k
    # a few steps of gradient descent on the attribute lower an image loss
    x = params["grad"].detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([x], lr=2e-3)
    losses = []
    for _ in range(8):
        opt.zero_grad()
        img = A.render_view(params["mean"].detach(), params["scale"].detach(), params["quat"].detach(),
                            params["opacity"].detach(), x, cam, mean, ropts)
        loss = ((img - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert losses[-1] < 0.5 * losses[0], losses


def test_autograd_raises_on_device_errors():
    """The binding reads both solves' statuses: a forward that did not converge in its
    cycle budget raises at backward, and so does an adjoint solve that did not."""
    from paper_2405_05446_gb300 import autograd as A
    sc, cam = _scene64(4)
    mean = [0.5, 0.5, 0.5]
    ropts = G.raster_opts(pairs_per_gaussian=64, **SMOOTH)
    one_cycle = G.solver_opts(max_cycles=1, rtol=1e-7)

    def params_of(scene):
        return [torch.tensor(np.asarray(getattr(scene, k)), device="cuda", requires_grad=True)
                for k in D.PARAMS]

    # forward: one V-cycle cannot reach 1e-7 on this view
    params = params_of(sc)
    img = A.render_view(*params, cam, mean, ropts, one_cycle)
    w = torch.randn_like(img)
    with pytest.raises(G.GDGSError) as ei:
        (img * w).sum().backward()
    assert ei.value.code == G._abi.ERR_NO_CONVERGE
    # adjoint only: every Gaussian behind the camera gives rho = 0, which the forward
    # solves at once; the adjoint of a random d image needs more than one cycle
    behind = S.Scene(sc.mean - np.float32([0.0, 0.0, 10.0]), sc.scale, sc.quat, sc.opacity, sc.grad)
    params = params_of(behind)
    img = A.render_view(*params, cam, mean, ropts, one_cycle)
    torch.cuda.synchronize()
    assert torch.allclose(img, torch.full_like(img, 0.5))
    with pytest.raises(G.GDGSError) as ei:
        (img * w).sum().backward()
    assert ei.value.code == G._abi.ERR_NO_CONVERGE
    # with the check off the same call returns (unchecked) gradients
    img = A.render_view(*params, cam, mean, ropts, one_cycle, check_status=False)
    (img * w).sum().backward()
    assert all(p.grad is not None for p in params)

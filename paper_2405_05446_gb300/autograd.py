"""torch.autograd binding of the render path: image = render(mean, scale, quat,
opacity, attribute) with gradients from the library's backward kernels.

Forward: gdgs_render_view into a workspace of its own (one per call, so several
views can be rendered before one backward). Backward: gdgs_render_view_backward,
i.e. the adjoint Poisson solve (the same zero-mean Neumann solve applied to
d loss / d image), the transpose of the threshold and of the divergence, the
rasteriser's back-to-front pass per tile and the projection's backward. All of
it runs in the CUDA library; this module only moves tensors.

Status: before the backward the forward's device status is read (a forward that
ran out of pair capacity, met a non-finite input or did not converge raises
GDGSError instead of being differentiated), and after it the adjoint solve's
status. Both reads wait for the stream; check_status=False skips them.
"""
from __future__ import annotations

import torch

import paper_2405_05446_gb300 as G


class _RenderView(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean, scale, quat, opacity, grad, cam, img_mean, ropts, sopts, check_status):
        g = G.DeviceGaussians(mean.detach().contiguous(), scale.detach().contiguous(),
                              quat.detach().contiguous(), opacity.detach().contiguous(),
                              grad.detach().contiguous())
        C, H, W = g.channels, cam.height, cam.width
        ws = torch.empty(G.workspace_size(g.n, C, W, H, ropts, sopts), dtype=torch.uint8,
                         device=mean.device)
        image = torch.empty((C, H, W), device=mean.device)
        G.render_view(g, cam, img_mean, image, ws, ropts, sopts)
        ctx.g, ctx.cam, ctx.ws, ctx.ropts, ctx.sopts = g, cam, ws, ropts, sopts
        ctx.check_status = check_status
        return image

    @staticmethod
    def backward(ctx, d_image):
        g, cam = ctx.g, ctx.cam
        ws_adj = torch.empty(G.workspace_size(0, g.channels, cam.width, cam.height, None, ctx.sopts),
                             dtype=torch.uint8, device=d_image.device)
        if ctx.check_status:
            G.sync_status(ctx.ws, raise_on_error=True)  # the forward being differentiated
        gr = G.render_view_backward(g, cam, d_image.float(), ctx.ws, ws_adj, ctx.ropts, ctx.sopts)
        if ctx.check_status:
            G.sync_status(ws_adj, raise_on_error=True)  # the adjoint solve
        ctx.ws = None
        return (gr["mean"], gr["scale"], gr["quat"], gr["opacity"], gr["grad"],
                None, None, None, None, None)


def render_view(mean, scale, quat, opacity, grad, cam, img_mean, ropts=None, sopts=None,
                check_status: bool = True):
    """Differentiable render of one view: float32 CUDA tensors in (the layouts of
    DeviceGaussians), the image [C][H][W] out. With check_status (the default) the
    backward raises GDGSError when the forward or the adjoint solve reported a device
    error (see the module docstring)."""
    return _RenderView.apply(mean, scale, quat, opacity, grad, cam, img_mean, ropts, sopts,
                             check_status)

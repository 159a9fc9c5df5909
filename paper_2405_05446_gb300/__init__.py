"""GDGS view synthesis on one GB300: Python binding of libgdgs (include/gdgs.h).

The functions here have the names of the C calls without the `gdgs_` prefix and
only marshal arguments: device buffers are torch CUDA tensors, the stream is the
current torch stream, and every step of the path runs in the CUDA library.
"""
from __future__ import annotations

import dataclasses

from . import _abi

__all__ = ["GDGSError", "raster_opts", "solver_opts", "workspace_size", "project",
           "render_gradients", "poisson_reconstruct", "poisson_reconstruct_rho", "render_view",
           "sync_status",
           "status_string", "Renderer", "gaussians_to_device", "kernel_launch_count",
           "profile_begin", "profile_end"]


class GDGSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


def _lib():
    return _abi.load()


def status_string(code: int) -> str:
    return _lib().gdgs_status_string(int(code)).decode()


def raster_opts(**kw) -> _abi.RasterOpts:
    o = _abi.RasterOpts()
    _lib().gdgs_default_raster_opts(o)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def solver_opts(**kw) -> _abi.SolverOpts:
    o = _abi.SolverOpts()
    _lib().gdgs_default_solver_opts(o)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes_void(s.cuda_stream)


def ctypes_void(v):
    import ctypes
    return ctypes.c_void_p(int(v)) if v else None


def _ptr(t):
    return ctypes_void(t.data_ptr()) if t is not None else None


@dataclasses.dataclass
class DeviceGaussians:
    """Gaussian attribute tensors resident on the device (layouts of gdgs_gaussians).

    grad is [n][C][2] (gradient Gaussians) or [n][C] (Laplacian Gaussians)."""
    mean: "object"
    scale: "object"
    quat: "object"
    opacity: "object"
    grad: "object"

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    @property
    def channels(self) -> int:
        return int(self.grad.shape[1])

    @property
    def attribute(self) -> int:
        return _abi.ATTR_LAPLACIAN if self.grad.dim() == 2 else _abi.ATTR_GRADIENT

    def struct(self) -> _abi.Gaussians:
        for t in (self.mean, self.scale, self.quat, self.opacity, self.grad):
            if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"):
                raise ValueError("Gaussian tensors must be contiguous float32 CUDA tensors")
        return _abi.Gaussians(self.n, self.channels, self.attribute, _ptr(self.mean),
                              _ptr(self.scale), _ptr(self.quat), _ptr(self.opacity),
                              _ptr(self.grad))


def gaussians_to_device(scene, device="cuda") -> DeviceGaussians:
    """Copy a host scene (numpy arrays, see scenes.Scene) into device tensors."""
    import torch
    f = lambda a: torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)  # noqa: E731
    return DeviceGaussians(f(scene.mean), f(scene.scale), f(scene.quat), f(scene.opacity),
                           f(scene.grad))


def camera_struct(cam) -> _abi.Camera:
    c = _abi.Camera()
    w = [float(x) for x in list(cam.world_to_cam.reshape(-1))]
    c.world_to_cam[:] = w
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_plane = float(cam.near)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def workspace_size(n: int, channels: int, width: int, height: int, ropts=None, sopts=None) -> int:
    return int(_lib().gdgs_workspace_size(int(n), int(channels), int(width), int(height), ropts, sopts))


def _check(code: int, where: str):
    if code != _abi.OK:
        raise GDGSError(code, where)


def project(g: DeviceGaussians, cam, ws, ropts=None, mean2d=None, cov2d=None, depth=None,
            rect=None, stream=None) -> None:
    out = _abi.Projected(_ptr(mean2d), _ptr(cov2d), _ptr(depth), _ptr(rect))
    gs = g.struct()
    _check(_lib().gdgs_project(gs, camera_struct(cam), ropts, out, _ptr(ws), ws.numel(),
                               _stream(stream)), "gdgs_project")


def render_gradients(g: DeviceGaussians, cam, maps, ws, mask=None, ropts=None, stream=None) -> None:
    gs = g.struct()
    _check(_lib().gdgs_render_gradients(gs, camera_struct(cam), ropts, _ptr(maps), _ptr(mask),
                                        _ptr(ws), ws.numel(), _stream(stream)),
           "gdgs_render_gradients")


def _mean_array(mean, C):
    import ctypes
    arr = (ctypes.c_float * C)(*[float(m) for m in list(mean)[:C]])
    return arr


def poisson_reconstruct(maps, mean, image, ws, mask=None, sopts=None, stream=None) -> None:
    C, _, H, W = maps.shape
    _check(_lib().gdgs_poisson_reconstruct(_ptr(maps), _ptr(mask), int(C), int(H), int(W),
                                           _mean_array(mean, C), sopts, _ptr(image), _ptr(ws),
                                           ws.numel(), _stream(stream)), "gdgs_poisson_reconstruct")


def poisson_reconstruct_rho(rho, mean, image, ws, mask=None, sopts=None, stream=None) -> None:
    """Solve L u = T(rho) for a Laplacian field given directly ([C][H][W])."""
    C, H, W = rho.shape
    _check(_lib().gdgs_poisson_reconstruct_rho(_ptr(rho), _ptr(mask), int(C), int(H), int(W),
                                               _mean_array(mean, C), sopts, _ptr(image), _ptr(ws),
                                               ws.numel(), _stream(stream)),
           "gdgs_poisson_reconstruct_rho")


def render_view(g: DeviceGaussians, cam, mean, image, ws, ropts=None, sopts=None, stream=None) -> None:
    gs = g.struct()
    _check(_lib().gdgs_render_view(gs, camera_struct(cam), _mean_array(mean, g.channels), ropts,
                                   sopts, _ptr(image), _ptr(ws), ws.numel(), _stream(stream)),
           "gdgs_render_view")


def camera_bytes(cam) -> bytes:
    """The gdgs_camera struct of `cam` as bytes (to fill a device camera buffer)."""
    import ctypes
    c = camera_struct(cam)
    return ctypes.string_at(ctypes.addressof(c), ctypes.sizeof(c))


def render_view_devcam(g: DeviceGaussians, cam, cam_dev, mean, image, ws, ropts=None, sopts=None,
                       stream=None) -> None:
    """render_view with the pose and intrinsics read from `cam_dev` (a device tensor
    holding one gdgs_camera, see camera_bytes) when the kernels run; `cam` gives
    the image size. A CUDA graph captured from this call replays for any camera."""
    gs = g.struct()
    _check(_lib().gdgs_render_view_devcam(gs, camera_struct(cam), _ptr(cam_dev),
                                          _mean_array(mean, g.channels), ropts, sopts,
                                          _ptr(image), _ptr(ws), ws.numel(), _stream(stream)),
           "gdgs_render_view_devcam")


def render_view_backward(g: DeviceGaussians, cam, d_image, ws, ws_adj, ropts=None, sopts=None,
                         stream=None) -> dict:
    """d loss / d (mean, scale, quat, opacity, grad) from d_image = d loss / d image, for
    the gdgs_render_view call that last used `ws` (same g, cam and options).
    ws_adj: a Poisson workspace (workspace_size(0, ...)) for the adjoint solve."""
    import torch
    gr = {k: torch.empty_like(getattr(g, k)) for k in ("mean", "scale", "quat", "opacity", "grad")}
    gg = _abi.GaussianGrads(_ptr(gr["mean"]), _ptr(gr["scale"]), _ptr(gr["quat"]),
                            _ptr(gr["opacity"]), _ptr(gr["grad"]))
    d_image = d_image.contiguous()
    _check(_lib().gdgs_render_view_backward(g.struct(), camera_struct(cam), ropts, sopts,
                                            _ptr(d_image), gg, _ptr(ws), ws.numel(), _ptr(ws_adj),
                                            ws_adj.numel(), _stream(stream)),
           "gdgs_render_view_backward")
    return gr


def sync_status(ws, stream=None, raise_on_error: bool = False) -> dict:
    st = _abi.SolveStats()
    code = _lib().gdgs_sync_status(_ptr(ws), st, _stream(stream))
    out = {"status": int(code), "status_string": status_string(code), "cycles": st.cycles,
           "rel_residual": st.rel_residual, "rho_norm": st.rho_norm,
           "mean_set": list(st.mean_set), "n_pairs": int(st.n_pairs),
           "n_active_tiles": int(st.n_active_tiles), "n_visible": int(st.n_visible)}
    if raise_on_error and code != _abi.OK:
        raise GDGSError(code, "gdgs_sync_status")
    return out


def kernel_launch_count() -> int:
    """Kernels this library has enqueued in this process (all streams)."""
    return int(_lib().gdgs_kernel_launch_count())


def profile_begin() -> None:
    _check(_lib().gdgs_profile_begin(), "gdgs_profile_begin")


def profile_end(max_entries: int = 64) -> dict:
    """Per-kernel {name: (launches, total_ms)} from CUDA events on the launch streams."""
    import ctypes
    arr = (_abi.KernelTime * max_entries)()
    n = ctypes.c_int32(0)
    _check(_lib().gdgs_profile_end(arr, max_entries, ctypes.byref(n)), "gdgs_profile_end")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


class Renderer:
    """Owns one workspace and renders views of scenes with up to `n` Gaussians.

    With graphs (the default) a view is one replay of a CUDA graph captured from
    render_view_devcam: one graph per (Gaussian tensors, output, image size, mean),
    captured at its first use after one ordinary render, replayed for any camera
    (written to a device buffer first, in stream order). It runs the same kernels
    as render_view without the gaps between launches."""

    def __init__(self, n: int, channels: int, width: int, height: int, ropts=None, sopts=None,
                 device="cuda", graphs: bool = True):
        import torch
        self.ropts = ropts if ropts is not None else raster_opts()
        self.sopts = sopts if sopts is not None else solver_opts()
        self.shape = (channels, height, width)
        nbytes = workspace_size(n, channels, width, height, self.ropts, self.sopts)
        if nbytes == 0:
            raise ValueError("unsupported sizes or options")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.device = device
        self.graphs = graphs
        self._views = {}

    def _view_graph(self, g: DeviceGaussians, cam, mean, out, stream):
        import ctypes
        import torch
        key = (tuple(t.data_ptr() for t in (g.mean, g.scale, g.quat, g.opacity, g.grad)), g.n,
               out.data_ptr(), cam.width, cam.height, tuple(float(m) for m in mean))
        entry = self._views.get(key)
        if entry is None:
            cam_dev = torch.empty(ctypes.sizeof(_abi.Camera), dtype=torch.uint8, device=self.device)
            cam_dev.copy_(torch.frombuffer(bytearray(camera_bytes(cam)), dtype=torch.uint8))
            s = torch.cuda.Stream(device=out.device)
            s.wait_stream(stream)
            with torch.cuda.stream(s):
                render_view_devcam(g, cam, cam_dev, mean, out, self.ws, self.ropts, self.sopts)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
                render_view_devcam(g, cam, cam_dev, mean, out, self.ws, self.ropts, self.sopts)
            stream.wait_stream(s)
            entry = self._views[key] = (graph, cam_dev)
        return entry

    def render_view(self, g: DeviceGaussians, cam, mean, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        if not self.graphs:
            render_view(g, cam, mean, out, self.ws, self.ropts, self.sopts, stream)
            return out
        st = stream if stream is not None else torch.cuda.current_stream()
        graph, cam_dev = self._view_graph(g, cam, mean, out, st)
        with torch.cuda.stream(st):
            cam_dev.copy_(torch.frombuffer(bytearray(camera_bytes(cam)), dtype=torch.uint8),
                          non_blocking=True)
            graph.replay()
        return out

    def render_gradients(self, g: DeviceGaussians, cam, maps=None, mask=None, stream=None):
        import torch
        C, H, W = self.shape
        if maps is None:
            shape = (C, H, W) if g.attribute == _abi.ATTR_LAPLACIAN else (C, 2, H, W)
            maps = torch.empty(shape, dtype=torch.float32, device=self.device)
        render_gradients(g, cam, maps, self.ws, mask, self.ropts, stream)
        return maps

    def poisson_reconstruct(self, maps, mean, mask=None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        poisson_reconstruct(maps, mean, out, self.ws, mask, self.sopts, stream)
        return out

    def stats(self, stream=None) -> dict:
        return sync_status(self.ws, stream)

"""CPU-only checks of the C ABI: the library builds, loads and exports every
symbol include/*.h declares; host-side argument checks and workspace sizing work
without touching a GPU (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2405_05446_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"GDGS_API[^;(]*?\b(gdgs_\w+)\s*\(", text, flags=re.S))
    return names


def test_header_declares_the_four_calls():
    names = _declared_symbols()
    for n in ("gdgs_project", "gdgs_render_gradients", "gdgs_poisson_reconstruct",
              "gdgs_render_view", "gdgs_workspace_size", "gdgs_sync_status"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert names
    for n in names:
        assert hasattr(lib, n), n
        assert n in _abi.PROTOTYPES, f"binding lacks {n}"


def test_abi_version_and_defaults(lib):
    assert lib.gdgs_abi_version() == _abi.ABI_VERSION
    r = _abi.RasterOpts()
    lib.gdgs_default_raster_opts(r)
    assert r.alpha_min == pytest.approx(1 / 255) and r.alpha_max == pytest.approx(0.99)
    assert r.t_min == pytest.approx(1e-4) and r.exp_coef == 1.0 and r.pairs_per_gaussian == 16
    s = _abi.SolverOpts()
    lib.gdgs_default_solver_opts(s)
    assert (s.nu1, s.nu2, s.coarse_max_dim) == (2, 1, 8) and s.rtol == pytest.approx(1e-6)
    for code in range(8):
        assert lib.gdgs_status_string(code)
    assert lib.gdgs_status_string(99) == b"unknown status"


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(_abi.Gaussians) == 8 + 4 + 4 + 5 * 8
    assert ctypes.sizeof(_abi.Camera) == 17 * 4 + 8
    assert ctypes.sizeof(_abi.RasterOpts) == 24
    assert ctypes.sizeof(_abi.SolverOpts) == 32
    assert ctypes.sizeof(_abi.SolveStats) == 4 + 4 + 8 + 8 + 32 + 8 + 4 + 4


def test_workspace_size_host_logic(lib):
    ws = lambda *a: lib.gdgs_workspace_size(*a, None, None)  # noqa: E731
    assert ws(1000, 3, 64, 64) > 0
    assert ws(200_000, 3, 1920, 1080) > ws(1000, 3, 1920, 1080) > ws(0, 3, 1920, 1080) > 0
    assert ws(0, 1, 1920, 1080) < ws(0, 3, 1920, 1080)
    for bad in [(-1, 3, 64, 64), (10, 0, 64, 64), (10, 5, 64, 64), (10, 3, 0, 64), (10, 3, 64, -2)]:
        assert ws(*bad) == 0
    so = _abi.SolverOpts()
    lib.gdgs_default_solver_opts(so)
    so.nu1 = 4
    assert lib.gdgs_workspace_size(10, 3, 64, 64, None, so) == 0
    so.nu1, so.max_cycles = 2, 0
    assert lib.gdgs_workspace_size(10, 3, 64, 64, None, so) == 0
    ro = _abi.RasterOpts()
    lib.gdgs_default_raster_opts(ro)
    ro.alpha_min = 0.0
    assert lib.gdgs_workspace_size(10, 3, 64, 64, ro, None) == 0


def test_argument_errors_return_before_any_gpu_work(lib):
    """Null pointers, bad sizes and a missing workspace are rejected on the host."""
    cam = _abi.Camera()
    cam.fx = cam.fy = 50.0
    cam.cx = cam.cy = 32.0
    cam.near_plane = 0.2
    cam.width = cam.height = 64
    g = _abi.Gaussians(10, 3, 0, None, None, None, None, None)
    assert lib.gdgs_render_view(g, cam, (ctypes.c_float * 3)(0.5, 0.5, 0.5), None, None,
                                ctypes.c_void_p(256), None, 0, None) == _abi.ERR_INVALID_ARG
    g0 = _abi.Gaussians(0, 3, 0, None, None, None, None, None)
    assert lib.gdgs_render_view(g0, cam, (ctypes.c_float * 3)(0.5, 0.5, 0.5), None, None,
                                ctypes.c_void_p(256), None, 0, None) == _abi.ERR_WORKSPACE
    assert lib.gdgs_render_view(g0, cam, (ctypes.c_float * 3)(0.5, 0.5, 0.5), None, None,
                                ctypes.c_void_p(8), ctypes.c_void_p(4096), 1 << 40,
                                None) == _abi.ERR_INVALID_ARG  # image not 16-byte aligned
    cam.width = 0
    assert lib.gdgs_render_view(g0, cam, (ctypes.c_float * 3)(0.5, 0.5, 0.5), None, None,
                                ctypes.c_void_p(256), ctypes.c_void_p(4096), 1 << 40,
                                None) == _abi.ERR_INVALID_ARG
    assert lib.gdgs_poisson_reconstruct(None, None, 3, 8, 8, (ctypes.c_float * 3)(), None,
                                        ctypes.c_void_p(256), ctypes.c_void_p(4096), 1 << 40,
                                        None) == _abi.ERR_INVALID_ARG
    # overlapping image and maps
    assert lib.gdgs_poisson_reconstruct(ctypes.c_void_p(4096), None, 1, 8, 8,
                                        (ctypes.c_float * 1)(), None, ctypes.c_void_p(4096 + 64),
                                        ctypes.c_void_p(1 << 20), 1 << 40, None) == _abi.ERR_INVALID_ARG
    assert lib.gdgs_sync_status(None, None, None) == _abi.ERR_WORKSPACE

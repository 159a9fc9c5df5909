"""ctypes mirror of include/gdgs.h (structs, status codes, prototypes).

Argument marshalling only: every step of the render path runs in libgdgs.so.
Loading fails loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libgdgs.so")

ABI_VERSION = 2
TILE = 16
MAX_CHANNELS = 4

OK = 0
ERR_INVALID_ARG = 1
ERR_WORKSPACE = 2
ERR_CUDA = 3
ERR_NO_CONVERGE = 4
ERR_NONFINITE = 5
ERR_TIMEOUT = 6
ERR_CAPACITY = 7

_p = ctypes.c_void_p
_f = ctypes.c_float
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


STORAGE_F32, STORAGE_BF16, STORAGE_F16 = 0, 1, 2
ATTR_GRADIENT = 0
ATTR_LAPLACIAN = 1


class Gaussians(ctypes.Structure):
    _fields_ = [("n", _i64), ("channels", _i32), ("attribute", _i32), ("mean", _p),
                ("scale", _p), ("quat", _p), ("opacity", _p), ("grad", _p)]


class Camera(ctypes.Structure):
    _fields_ = [("world_to_cam", _f * 12), ("fx", _f), ("fy", _f), ("cx", _f), ("cy", _f),
                ("near_plane", _f), ("width", _i32), ("height", _i32)]


class RasterOpts(ctypes.Structure):
    _fields_ = [("alpha_min", _f), ("alpha_max", _f), ("t_min", _f), ("dilation", _f),
                ("exp_coef", _f), ("pairs_per_gaussian", _i32)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("nu1", _i32), ("nu2", _i32), ("max_cycles", _i32), ("rtol", _f),
                ("coarse_max_dim", _i32), ("rho_threshold", _f), ("omega", _f),
                ("storage", _i32)]


class GaussianGrads(ctypes.Structure):
    _fields_ = [("d_mean", _p), ("d_scale", _p), ("d_quat", _p), ("d_opacity", _p), ("d_attr", _p)]


class SolveStats(ctypes.Structure):
    _fields_ = [("status", _i32), ("cycles", _i32), ("rel_residual", ctypes.c_double),
                ("rho_norm", ctypes.c_double), ("mean_set", ctypes.c_double * MAX_CHANNELS),
                ("n_pairs", _i64), ("n_active_tiles", _i32), ("n_visible", _i32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", _i64), ("total_ms", ctypes.c_double)]


class Projected(ctypes.Structure):
    _fields_ = [("mean2d", _p), ("cov2d", _p), ("depth", _p), ("rect", _p)]


# name -> (restype, argtypes); the set the header declares
PROTOTYPES = {
    "gdgs_abi_version": (ctypes.c_int, []),
    "gdgs_default_raster_opts": (None, [ctypes.POINTER(RasterOpts)]),
    "gdgs_default_solver_opts": (None, [ctypes.POINTER(SolverOpts)]),
    "gdgs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gdgs_workspace_size": (ctypes.c_size_t, [_i64, _i32, _i32, _i32, ctypes.POINTER(RasterOpts),
                                              ctypes.POINTER(SolverOpts)]),
    "gdgs_project": (ctypes.c_int, [ctypes.POINTER(Gaussians), ctypes.POINTER(Camera),
                                    ctypes.POINTER(RasterOpts), ctypes.POINTER(Projected), _p,
                                    ctypes.c_size_t, _p]),
    "gdgs_render_gradients": (ctypes.c_int, [ctypes.POINTER(Gaussians), ctypes.POINTER(Camera),
                                             ctypes.POINTER(RasterOpts), _p, _p, _p,
                                             ctypes.c_size_t, _p]),
    "gdgs_poisson_reconstruct": (ctypes.c_int, [_p, _p, _i32, _i32, _i32, ctypes.POINTER(_f),
                                                ctypes.POINTER(SolverOpts), _p, _p, ctypes.c_size_t,
                                                _p]),
    "gdgs_poisson_reconstruct_rho": (ctypes.c_int, [_p, _p, _i32, _i32, _i32, ctypes.POINTER(_f),
                                                    ctypes.POINTER(SolverOpts), _p, _p,
                                                    ctypes.c_size_t, _p]),
    "gdgs_render_view": (ctypes.c_int, [ctypes.POINTER(Gaussians), ctypes.POINTER(Camera),
                                        ctypes.POINTER(_f), ctypes.POINTER(RasterOpts),
                                        ctypes.POINTER(SolverOpts), _p, _p, ctypes.c_size_t, _p]),
    "gdgs_render_view_devcam": (ctypes.c_int, [ctypes.POINTER(Gaussians), ctypes.POINTER(Camera),
                                               _p, ctypes.POINTER(_f), ctypes.POINTER(RasterOpts),
                                               ctypes.POINTER(SolverOpts), _p, _p, ctypes.c_size_t,
                                               _p]),
    "gdgs_render_view_backward": (ctypes.c_int, [ctypes.POINTER(Gaussians), ctypes.POINTER(Camera),
                                                 ctypes.POINTER(RasterOpts), ctypes.POINTER(SolverOpts),
                                                 _p, ctypes.POINTER(GaussianGrads), _p, ctypes.c_size_t,
                                                 _p, ctypes.c_size_t, _p]),
    "gdgs_sync_status": (ctypes.c_int, [_p, ctypes.POINTER(SolveStats), _p]),
    "gdgs_poisson_reconstruct_static": (ctypes.c_int, [_p, _p, _i32, _i32, _i32, ctypes.POINTER(_f),
                                                       ctypes.POINTER(SolverOpts), _p,
                                                       ctypes.POINTER(SolveStats), _p]),
    "gdgs_poisson_static_status": (ctypes.c_int, [ctypes.POINTER(SolveStats), _p]),
    "gdgs_kernel_launch_count": (ctypes.c_uint64, []),
    "gdgs_profile_begin": (ctypes.c_int, []),
    "gdgs_profile_end": (ctypes.c_int, [ctypes.POINTER(KernelTime), _i32, ctypes.POINTER(_i32)]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgdgs.so and bind every prototype. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; call paper_2405_05446_gb300.build.build() "
                           "(needs nvcc). There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.gdgs_abi_version() != ABI_VERSION:
        raise RuntimeError("libgdgs ABI version mismatch")
    _lib = lib
    return lib

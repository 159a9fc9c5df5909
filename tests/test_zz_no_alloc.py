"""The allocation-free Poisson entry point (gdgs_poisson_reconstruct_static).

Some callers cannot allocate device memory where they need the solve (inside a
stream capture, inside a host application that owns the allocator, in loops that
forbid allocation after start-up). The static entry point takes only inputs and
outputs and keeps its scratch in a fixed device array of the library. These
tests call it through the C ABI and compare it with gdgs_poisson_reconstruct,
twice in a row (the array keeps the previous call's contents). The file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import paper_2405_05446_gb300 as G
from paper_2405_05446_gb300 import _abi

from gpu_util import IMG_TOL, ensure_lib, img_err

pytestmark = pytest.mark.gpu


def _static_call(lib, maps, mean, img, stats=None, sopts=None):
    C, _, H, W = maps.shape
    return lib.gdgs_poisson_reconstruct_static(
        ctypes.c_void_p(maps.data_ptr()), None, C, H, W, (ctypes.c_float * C)(*mean), sopts,
        ctypes.c_void_p(img.data_ptr()), stats,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_entry_point_matches_workspace_entry_point_twice():
    ensure_lib()
    lib = _abi.load()
    rng = np.random.default_rng(21)
    means = [[0.5, 0.25, -0.1], [0.1, 0.9, 0.3]]
    for call, (H, W) in enumerate([(240, 320), (200, 300)]):
        maps = torch.as_tensor(rng.laplace(0, 0.1, (3, 2, H, W)).astype(np.float32)).cuda()
        mean = means[call]
        ref = torch.empty((3, H, W), device="cuda")
        ws = torch.empty(G.workspace_size(0, 3, W, H), dtype=torch.uint8, device="cuda")
        G.poisson_reconstruct(maps, mean, ref, ws)
        assert G.sync_status(ws)["status"] == 0
        got = torch.full((3, H, W), float("nan"), device="cuda")
        st = _abi.SolveStats()
        assert _static_call(lib, maps, mean, got, st) == _abi.OK
        assert st.status == _abi.OK and st.rel_residual <= 1e-6
        a, b = got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(a).all()
        assert np.abs(a - b).max() <= IMG_TOL
        oracle = O.poisson_neumann(O.divergence(maps.cpu().numpy().astype(np.float64)), mean)
        assert img_err(a, oracle)[0] <= IMG_TOL


def test_static_entry_point_inside_a_stream_capture():
    """Inside a capture the call only enqueues (stats must be NULL); the replayed solve
    equals the workspace path and its status is read afterwards."""
    ensure_lib()
    lib = _abi.load()
    rng = np.random.default_rng(5)
    H, W = 150, 220
    mean = [0.3, 0.6, 0.45]
    maps = torch.as_tensor(rng.laplace(0, 0.1, (3, 2, H, W)).astype(np.float32)).cuda()
    ref = torch.empty((3, H, W), device="cuda")
    ws = torch.empty(G.workspace_size(0, 3, W, H), dtype=torch.uint8, device="cuda")
    G.poisson_reconstruct(maps, mean, ref, ws)
    assert G.sync_status(ws)["status"] == 0
    got = torch.full((3, H, W), float("nan"), device="cuda")
    # one call outside the capture first: the array's address is looked up there
    assert _static_call(lib, maps, mean, got) == _abi.OK
    torch.cuda.synchronize()
    got.fill_(float("nan"))
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
        # a caller that asks for stats would need to wait: refused, nothing enqueued
        assert _static_call(lib, maps, mean, got, _abi.SolveStats()) == _abi.ERR_INVALID_ARG
        assert _static_call(lib, maps, mean, got) == _abi.OK
    torch.cuda.synchronize()
    assert torch.isnan(got).all()  # captured, not run
    for _ in range(2):
        got.fill_(float("nan"))
        graph.replay()
        st = _abi.SolveStats()
        assert lib.gdgs_poisson_static_status(
            st, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == _abi.OK
        torch.cuda.synchronize()
        assert st.status == _abi.OK and 0 < st.cycles and st.rel_residual <= 1e-6
        a, b = got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.abs(a - b).max() <= IMG_TOL


def test_static_entry_point_takes_no_device_memory_on_repeat():
    """Repeated calls of one size leave the device's free memory unchanged."""
    ensure_lib()
    lib = _abi.load()
    H, W = 128, 96
    maps = torch.zeros((3, 2, H, W), device="cuda")
    img = torch.empty((3, H, W), device="cuda")
    st = _abi.SolveStats()
    assert _static_call(lib, maps, [0.5] * 3, img, st) == _abi.OK  # first call of this size
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _static_call(lib, maps, [0.5] * 3, img, st) == _abi.OK
        assert st.status == _abi.OK
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.allclose(img, torch.full_like(img, 0.5))


def test_static_entry_point_rejects_sizes_beyond_its_array():
    ensure_lib()
    lib = _abi.load()
    maps = torch.zeros((3, 2, 1080, 1920), device="cuda")
    img = torch.empty((3, 1080, 1920), device="cuda")
    assert _static_call(lib, maps, [0.5] * 3, img) == _abi.ERR_WORKSPACE

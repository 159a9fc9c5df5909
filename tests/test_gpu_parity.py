"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2405_05446_gb300 as G
from paper_2405_05446_gb300 import scenes as S

from gpu_util import (AMB_FRAC_MAX, IMG_TOL, LIB_DEPTH_REL, MAP_TOL, ensure_lib, gpu_maps,
                      gpu_poisson, img_err, map_rel_err, oracle_maps, oracle_opts)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _small_prims(n=20000, w=330, h=190, seed=0, channels=3):
    cam = S.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), w, h)
    return S.primitives_scene(seed, n=n, orient_camera=cam, channels=channels), cam


# ------------------------------------------------------------------ projection

def test_projection_matches_oracle():
    scene = S.tiny_scene(3, n=2000)
    cam = S.look_at_camera((0.7, -0.4, -2.8), (0.1, 0.0, 0.2), 96, 72, hfov_deg=55)
    ro = G.raster_opts()
    g = G.gaussians_to_device(scene)
    ws = torch.empty(G.workspace_size(scene.n, 3, cam.width, cam.height, ro, None), dtype=torch.uint8, device="cuda")
    m2 = torch.zeros((scene.n, 2), device="cuda")
    cv = torch.zeros((scene.n, 3), device="cuda")
    dp = torch.zeros(scene.n, device="cuda")
    rc = torch.zeros((scene.n, 4), dtype=torch.int32, device="cuda")
    G.project(g, cam, ws, ro, m2, cv, dp, rc)
    st = G.sync_status(ws)
    assert st["status"] == 0
    proj = O.project(scene, cam, oracle_opts(ro), depth_rel=LIB_DEPTH_REL)
    vis = rc[:, 2].cpu().numpy() > rc[:, 0].cpu().numpy()
    ok = proj[:, O.VALID] > 0
    # the returned depth is the float-float camera depth rounded to float: within
    # half an ulp of the FP64 depth, plus the pair's own error (2^-44 of its terms)
    dpn = dp.cpu().numpy().astype(np.float64)
    t = proj[vis, O.DEPTH]
    half_ulp = np.spacing(np.float32(t)).astype(np.float64) / 2
    assert np.all(np.abs(dpn[vis] - t) <= half_ulp + 2.0 ** -44 * 8 * np.abs(t))
    # the near cull agrees with the FP64 depth except within the depth bound
    sure = proj[:, O.NEARAMB] == 0
    assert not np.any(vis & ~ok & sure)
    m2 = m2.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(m2[vis, 0], proj[vis, O.MX], atol=1e-4, rtol=0)
    np.testing.assert_allclose(m2[vis, 1], proj[vis, O.MY], atol=1e-4, rtol=0)
    cv = cv.cpu().numpy().astype(np.float64)
    for k, col in enumerate([O.S00, O.S01, O.S11]):
        scale = np.maximum(proj[vis, O.S00], proj[vis, O.S11])
        assert np.max(np.abs(cv[vis, k] - proj[vis, col]) / scale) < 1e-5
    # the tile rectangle covers every pixel of the exact footprint box
    rc = rc.cpu().numpy()
    W, H = cam.width, cam.height
    for i in np.nonzero(ok)[0]:
        j0 = int(np.ceil(proj[i, O.XMIN] - 0.5)); j1 = int(np.floor(proj[i, O.XMAX] - 0.5))
        i0 = int(np.ceil(proj[i, O.YMIN] - 0.5)); i1 = int(np.floor(proj[i, O.YMAX] - 0.5))
        j0, j1, i0, i1 = max(j0, 0), min(j1, W - 1), max(i0, 0), min(i1, H - 1)
        if j0 > j1 or i0 > i1:
            continue
        assert rc[i, 0] <= j0 // 16 and rc[i, 2] > j1 // 16, i
        assert rc[i, 1] <= i0 // 16 and rc[i, 3] > i1 // 16, i
    assert st["n_visible"] == int(vis.sum())


# ------------------------------------------------------------------ rasteriser

@pytest.mark.parametrize("channels", [3, 1, 4])
def test_gradient_maps_tiny(channels):
    scene = S.tiny_scene(0, channels=channels)
    cam = S.tiny_camera()
    gm, _, st = gpu_maps(scene, cam)
    assert st["status"] == 0
    om, amb = oracle_maps(scene, cam)
    assert amb.mean() <= AMB_FRAC_MAX
    assert map_rel_err(gm, om, amb) <= MAP_TOL


def test_gradient_maps_ragged_prims_several_tiles():
    scene, cam = _small_prims()
    gm, _, st = gpu_maps(scene, cam)
    assert st["status"] == 0 and st["n_pairs"] > 0
    om, amb = oracle_maps(scene, cam)
    assert amb.mean() <= AMB_FRAC_MAX
    assert map_rel_err(gm, om, amb) <= MAP_TOL


def test_gradient_maps_half_exponent_option():
    scene = S.tiny_scene(5, n=500)
    cam = S.tiny_camera(80, 48)
    ro = G.raster_opts(exp_coef=0.5, dilation=0.1)
    gm, _, st = gpu_maps(scene, cam, ro)
    om, amb = oracle_maps(scene, cam, ro)
    assert map_rel_err(gm, om, amb) <= MAP_TOL


def test_tile_mask_and_untouched_tiles():
    scene = S.tiny_scene(1, n=60)  # sparse: most tiles empty
    cam = S.tiny_camera(100, 70)
    gm, mask, st = gpu_maps(scene, cam, with_mask=True)
    om, amb = oracle_maps(scene, cam)
    H, W = cam.height, cam.width
    pix_mask = np.kron(mask, np.ones((16, 16), np.uint8))[:H, :W].astype(bool)
    # every pixel the oracle sees non-zero lies in an active tile
    assert not np.any((np.abs(om).sum((0, 1)) > 0) & ~pix_mask)
    # active tiles are written and match; inactive ones are left untouched (NaN fill)
    assert np.all(np.isnan(gm[:, :, ~pix_mask]))
    assert np.isfinite(gm[:, :, pix_mask]).all()
    gm0 = np.where(np.isnan(gm), 0.0, gm)
    assert map_rel_err(gm0, om, amb) <= MAP_TOL
    assert st["n_active_tiles"] == int(mask.sum()) < mask.size


def test_gradient_maps_1080p_whole_image():
    """Every pixel of the 1920x1080 workload's six gradient planes against the oracle."""
    scene, cam, _, _ = S.workload("prims1080p")
    gm, _, st = gpu_maps(scene, cam)
    assert st["status"] == 0
    om, amb = oracle_maps(scene, cam)
    print(f"1080p maps: {int(amb.sum())} ambiguous pixels ({amb.mean():.2e}), "
          f"max rel err {map_rel_err(gm, om, amb):.2e}")
    assert amb.mean() <= AMB_FRAC_MAX
    assert map_rel_err(gm, om, amb) <= MAP_TOL
    # ambiguous pixels differ by at most one decision's worth of a splat's attribute
    d = np.abs(gm - om)[:, :, amb > 0]
    assert d.size == 0 or d.max() <= 2 * np.abs(scene.grad).max()


def test_raster_deterministic():
    scene, cam = _small_prims(n=5000)
    a, _, _ = gpu_maps(scene, cam)
    b, _, _ = gpu_maps(scene, cam)
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ Poisson

@pytest.mark.parametrize("hw", [(64, 64), (135, 240), (17, 9), (3, 200), (1, 1), (2, 2), (100, 37),
                                (33, 16), (270, 481), (97, 114), (25, 58), (48, 56), (49, 2),
                                (1, 130), (99, 203), (61, 483)])
def test_poisson_matches_dct_oracle(hw):
    H, W = hw
    rng = np.random.default_rng(H * 1000 + W)
    maps = rng.laplace(0, 0.1, (3, 2, H, W)).astype(np.float32)
    mean = [0.5, 0.1, -0.2]
    img, st = gpu_poisson(maps, mean)
    ref = O.poisson_neumann(O.divergence(maps.astype(np.float64)), mean)
    assert st["status"] == 0, st
    assert img_err(img, ref)[0] <= IMG_TOL
    assert st["rel_residual"] <= 1e-6
    np.testing.assert_allclose(img.mean(axis=(1, 2)), mean, atol=1e-6)


def test_pixel_kernels_alignment_contract():
    """Maps and image must be 16-byte aligned (then rows of a multiple of 4 floats take
    the four-pixel divergence and finalisation; other widths the one-pixel kernels, both
    covered against the oracle by the shapes above). A pointer one float past a 16-byte
    boundary is rejected on the host with GDGS_ERR_INVALID_ARG, before anything runs."""
    H, W = 270, 480
    rng = np.random.default_rng(7)
    maps = torch.from_numpy(rng.laplace(0, 0.1, (3, 2, H, W)).astype(np.float32)).cuda()
    mean = [0.5, 0.1, -0.2]
    sopts = G.solver_opts()
    ws = torch.empty(G.workspace_size(0, 3, W, H, None, sopts), dtype=torch.uint8, device="cuda")
    img = torch.empty((3, H, W), device="cuda")
    G.poisson_reconstruct(maps, mean, img, ws, sopts=sopts)
    st = G.sync_status(ws)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
    ref = O.poisson_neumann(O.divergence(maps.cpu().numpy().astype(np.float64)), mean)
    assert img_err(img.cpu().numpy().astype(np.float64), ref)[0] <= IMG_TOL
    mbuf = torch.empty(maps.numel() + 1, device="cuda")
    maps_s = mbuf[1:].view(maps.shape)
    ibuf = torch.empty(img.numel() + 1, device="cuda")
    img_s = ibuf[1:].view(img.shape)
    for m, o in ((maps_s, img), (maps, img_s)):
        with pytest.raises(G.GDGSError) as ei:
            G.poisson_reconstruct(m, mean, o, ws, sopts=sopts)
        assert ei.value.code == 1  # GDGS_ERR_INVALID_ARG


@pytest.mark.parametrize("hw", [(2, 12000), (12000, 2)])
def test_poisson_long_strip(hw):
    """Strips whose small levels do not fit the one-CTA tail with their coefficient
    tables (the tail then starts one level lower): the FP64 residual of the image
    and its mean, checked against the Neumann Laplacian of Eq. p2d."""
    rng = np.random.default_rng(hw[0])
    H, W = hw
    img0 = rng.random((1, H, W))
    maps = O.forward_gradients(img0)
    rho = O.divergence(maps)
    img, st = gpu_poisson(maps.astype(np.float32), [0.5])
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
    r = rho - O.laplacian_neumann(img)
    assert np.linalg.norm(r) <= 2e-6 * np.linalg.norm(rho)
    assert abs(img.mean() - 0.5) <= 1e-6


def test_poisson_recovers_known_image_1080p():
    H, W = 1080, 1920
    img0 = np.stack([S.image_from_gradients_test_image(H, W, seed=s) for s in range(3)])
    maps = O.forward_gradients(img0).astype(np.float32)
    img, st = gpu_poisson(maps, img0.mean(axis=(1, 2)))
    ref = O.poisson_neumann(O.divergence(maps.astype(np.float64)), img0.mean(axis=(1, 2)))
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6
    assert st["cycles"] <= 12
    assert img_err(img, ref)[1] <= IMG_TOL


@pytest.mark.parametrize("max_cycles", [1, 30])
def test_identical_channels_give_identical_images_1080p(max_cycles):
    """Channels are independent problems: four copies of one field at 1080p (enough
    CTAs for several waves per level) must come out bit-identical. A kernel that
    reads cells another CTA of the same launch rewrites (an in-place level update)
    breaks this, even where the solve still converges."""
    rng = np.random.default_rng(5)
    H, W, C = 1080, 1920, 4
    one = rng.laplace(0, 0.1, (1, 2, H, W)).astype(np.float32)
    maps = np.repeat(one, C, axis=0)
    img, st = gpu_poisson(maps, [0.5] * C, G.solver_opts(max_cycles=max_cycles, rtol=0.0 if max_cycles == 1 else 1e-6))
    for c in range(1, C):
        assert np.array_equal(img[c], img[0]), c
    if max_cycles > 1:
        assert st["status"] == 0 and st["cycles"] <= 5, st


def test_channel_split_equals_one_channel_solves():
    """A multi-channel solve runs one cycle loop per channel (each on a stream of its own,
    stopping on its own residual): every channel's image equals the 1-channel solve of
    that channel bit for bit, and the channels' different cycle counts merge correctly
    (a zero channel stops at once, a larger one needs more cycles)."""
    rng = np.random.default_rng(9)
    H, W = 540, 960
    maps = np.stack([rng.laplace(0, 0.1, (2, H, W)), np.zeros((2, H, W)),
                     rng.laplace(0, 3.0, (2, H, W))]).astype(np.float32)
    mean = [0.5, 0.2, -0.3]
    img, st = gpu_poisson(maps, mean)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
    cycles = []
    for c in range(3):
        one, st1 = gpu_poisson(maps[c:c + 1], [mean[c]])
        assert st1["status"] == 0
        assert np.array_equal(one[0], img[c]), c
        cycles.append(st1["cycles"])
    assert cycles[1] == 0 and st["cycles"] == max(cycles)
    assert np.all(img[1] == np.float32(0.2))


STORAGES = {"f32": 0, "bf16": 1, "f16": 2}


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_poisson_16bit_storage_reaches_tolerance_1080p(storage):
    """BF16 / FP16 storage of the multigrid corrections and coarse right-hand sides:
    the FP32 residual recurrence refines the float-float iterate to rtol all the same."""
    H, W = 1080, 1920
    img0 = np.stack([S.image_from_gradients_test_image(H, W, seed=s) for s in range(3)])
    maps = O.forward_gradients(img0).astype(np.float32)
    img, st = gpu_poisson(maps, img0.mean(axis=(1, 2)), G.solver_opts(storage=STORAGES[storage]))
    ref = O.poisson_neumann(O.divergence(maps.astype(np.float64)), img0.mean(axis=(1, 2)))
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
    assert st["cycles"] <= 12
    assert img_err(img, ref)[1] <= IMG_TOL


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_poisson_storage_4k_against_oracle(storage):
    """The 4K grid (3840 x 2160, 10 levels) in every storage format, one channel,
    against the exact DCT solve."""
    H, W = 2160, 3840
    img0 = S.image_from_gradients_test_image(H, W, seed=11)[None]
    maps = O.forward_gradients(img0).astype(np.float32)
    img, st = gpu_poisson(maps, [float(img0.mean())], G.solver_opts(storage=STORAGES[storage]))
    ref = O.poisson_neumann(O.divergence(maps.astype(np.float64)), [float(img0.mean())])
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
    assert img_err(img, ref)[1] <= IMG_TOL


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_render_view_16bit_storage(storage):
    scene, cam = _small_prims(n=8000)
    mean = [0.5, 0.5, 0.5]
    img, st = _render(scene, cam, mean, sopts=G.solver_opts(storage=STORAGES[storage]))
    ref, _, _ = O.render_view(scene, cam, mean, oracle_opts(G.raster_opts()))
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
    assert img_err(img, ref)[1] <= IMG_TOL


def test_storage_scaling_keeps_fp32_bitwise():
    """The per-cycle power-of-two scaling is exact: FP32 storage gives the same bits
    for a field and for the same field times 2^20 (then divided back)."""
    rng = np.random.default_rng(17)
    maps = rng.laplace(0, 0.1, (2, 2, 150, 211)).astype(np.float32)
    a, sa = gpu_poisson(maps, [0.0, 0.0])
    b, sb = gpu_poisson(maps * np.float32(2.0 ** 20), [0.0, 0.0])
    assert sa["status"] == sb["status"] == 0 and sa["cycles"] == sb["cycles"]
    assert np.array_equal(a * 2.0 ** 20, b)


def test_poisson_zero_field_gives_mean():
    img, st = gpu_poisson(np.zeros((2, 2, 40, 50), np.float32), [0.25, 0.75])
    assert st["status"] == 0 and st["cycles"] == 0
    np.testing.assert_array_equal(img[0], 0.25)
    np.testing.assert_array_equal(img[1], 0.75)


def test_poisson_no_converge_status():
    rng = np.random.default_rng(1)
    maps = rng.laplace(0, 0.1, (1, 2, 200, 300)).astype(np.float32)
    img, st = gpu_poisson(maps, [0.5], G.solver_opts(max_cycles=1, rtol=1e-9))
    assert st["status"] == G._abi.ERR_NO_CONVERGE
    assert st["cycles"] == 1 and st["rel_residual"] > 1e-9


def test_poisson_nonfinite_status():
    maps = np.zeros((1, 2, 32, 32), np.float32)
    maps[0, 0, 5, 5] = np.nan
    _, st = gpu_poisson(maps, [0.5])
    assert st["status"] == G._abi.ERR_NONFINITE


def test_poisson_mask_reads_inactive_tiles_as_zero():
    rng = np.random.default_rng(2)
    H, W = 70, 90
    maps = rng.laplace(0, 0.1, (3, 2, H, W)).astype(np.float32)
    mask = (rng.random(((H + 15) // 16, (W + 15) // 16)) < 0.5).astype(np.uint8)
    pix = np.kron(mask, np.ones((16, 16), np.uint8))[:H, :W].astype(bool)
    garbage = maps.copy()
    garbage[:, :, ~pix] = 1e30
    clean = np.where(pix, maps, 0).astype(np.float32)
    a, st = gpu_poisson(garbage, [0.5] * 3, mask=mask)
    b, _ = gpu_poisson(clean, [0.5] * 3)
    assert st["status"] == 0
    np.testing.assert_allclose(a, b, atol=1e-6)


def test_poisson_coarse_cache_reused_across_sizes():
    """One workspace solving two different grid shapes in turn (the cached coarse
    factor is keyed by the shape) gives the same answers as fresh workspaces."""
    rng = np.random.default_rng(3)
    m1 = rng.laplace(0, 0.1, (1, 2, 90, 130)).astype(np.float32)
    m2 = rng.laplace(0, 0.1, (1, 2, 64, 64)).astype(np.float32)
    nbytes = max(G.workspace_size(0, 1, 130, 90, None, None), G.workspace_size(0, 1, 64, 64, None, None))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = []
    for m in (m1, m2, m1):
        t = torch.as_tensor(m).cuda()
        img = torch.empty((1,) + m.shape[2:], device="cuda")
        G.poisson_reconstruct(t, [0.5], img, ws)
        assert G.sync_status(ws)["status"] == 0
        out.append(img.cpu().numpy())
    assert np.array_equal(out[0], out[2])
    ref = O.poisson_neumann(O.divergence(m2.astype(np.float64)), [0.5])
    assert img_err(out[1], ref)[0] <= IMG_TOL


# ------------------------------------------------------------------ whole view

def _render(scene, cam, mean, ropts=None, sopts=None, nbytes=None):
    g = G.gaussians_to_device(scene)
    ropts = ropts or G.raster_opts()
    sopts = sopts or G.solver_opts()
    nb = nbytes or G.workspace_size(scene.n, scene.channels, cam.width, cam.height, ropts, sopts)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    img = torch.empty((scene.channels, cam.height, cam.width), device="cuda")
    G.render_view(g, cam, mean, img, ws, ropts, sopts)
    return img.cpu().numpy().astype(np.float64), G.sync_status(ws)


def test_render_view_tiny_matches_oracle():
    scene, cam, mean, rtol = S.workload("tiny64")
    img, st = _render(scene, cam, mean, sopts=G.solver_opts(rtol=rtol))
    ref, _, _ = O.render_view(scene, cam, mean, oracle_opts(G.raster_opts()))
    assert st["status"] == 0, st
    assert img_err(img, ref)[1] <= IMG_TOL


def test_render_view_1080p_matches_oracle():
    scene, cam, mean, rtol = S.workload("prims1080p")
    img, st = _render(scene, cam, mean, sopts=G.solver_opts(rtol=rtol))
    ref, _, amb = O.render_view(scene, cam, mean, oracle_opts(G.raster_opts()))
    assert st["status"] == 0 and st["rel_residual"] <= rtol, st
    rel, absolute = img_err(img, ref)
    print(f"1080p view: max |gpu - oracle| = {absolute:.2e}, ambiguous pixels {int(amb.sum())}")
    assert absolute <= IMG_TOL, (rel, absolute)
    assert st["n_visible"] > 0.9 * scene.n


def test_render_view_empty_and_culled_scenes_give_mean():
    cam = S.tiny_camera(48, 40)
    empty = S.tiny_scene(0, n=0)
    img, st = _render(empty, cam, [0.5, 0.2, 0.1])
    assert st["status"] == 0
    np.testing.assert_array_equal(img[1], np.float32(0.2))
    behind = S.tiny_scene(0, n=50)
    behind.mean[:, 2] = -10.0  # behind the camera at z = -3
    img, st = _render(behind, cam, [0.5, 0.2, 0.1])
    assert st["status"] == 0 and st["n_visible"] == 0
    np.testing.assert_array_equal(img[0], np.float32(0.5))


def test_render_view_capacity_overflow_is_reported():
    scene, cam, mean, _ = S.workload("tiny64")
    scene.scale *= 4  # large splats: many tiles each
    img, st = _render(scene, cam, mean, ropts=G.raster_opts(pairs_per_gaussian=1))
    assert st["status"] == G._abi.ERR_CAPACITY
    assert st["n_pairs"] > scene.n


def test_render_view_nonfinite_gaussian_is_reported():
    scene, cam, mean, _ = S.workload("tiny64")
    scene.mean[7, 1] = np.inf
    _, st = _render(scene, cam, mean)
    assert st["status"] == G._abi.ERR_NONFINITE


def test_render_view_workspace_too_small_raises():
    scene, cam, mean, _ = S.workload("tiny64")
    with pytest.raises(G.GDGSError) as e:
        _render(scene, cam, mean, nbytes=4096)
    assert e.value.code == G._abi.ERR_WORKSPACE


def test_renderer_graph_replays_match_direct_renders():
    """Renderer replays one captured graph per (Gaussians, output, size, mean) for any
    camera: every replay equals a direct render_view of that camera bit for bit."""
    scene, cam0 = _small_prims(n=8000)
    g = G.gaussians_to_device(scene)
    r = G.Renderer(scene.n, 3, cam0.width, cam0.height)
    ws = torch.empty_like(r.ws)
    out = torch.empty((3, cam0.height, cam0.width), device="cuda")
    ref = torch.empty_like(out)
    rng = np.random.default_rng(2)
    for i in range(4):
        cam = S.sphere_camera(rng, cam0.width, cam0.height) if i else cam0
        r.render_view(g, cam, [0.5, 0.4, 0.6], out)
        st = r.stats()
        G.render_view(g, cam, [0.5, 0.4, 0.6], ref, ws)
        st2 = G.sync_status(ws)
        assert st["status"] == st2["status"] == 0 and st["cycles"] == st2["cycles"]
        assert torch.equal(out, ref), i
    assert len(r._views) == 1


def test_graph_and_direct_cycle_loops_agree():
    """The cycle loop launched as a CUDA graph (WHILE node, default) and as direct
    launches (used while profiling) give bit-identical images and cycle counts."""
    scene, cam = _small_prims(n=8000)
    mean = [0.5, 0.5, 0.5]
    a, sa = _render(scene, cam, mean)
    G.profile_begin()
    b, sb = _render(scene, cam, mean)
    prof = G.profile_end()
    assert "mg0_up" in prof and prof["mg0_up"][0] >= sb["cycles"]
    assert sa["status"] == sb["status"] == 0
    assert sa["cycles"] == sb["cycles"]
    assert np.array_equal(a, b)


def test_kernel_launch_count_covers_graph_kernels():
    scene, cam, mean, _ = S.workload("tiny64")
    _render(scene, cam, mean)  # warm: builds the cycle graph for this shape
    n0 = G.kernel_launch_count()
    img, st = _render(scene, cam, mean)
    n1 = G.kernel_launch_count()
    # projection, sorts, raster, divergence, setup, finalize + per cycle kernels
    assert n1 - n0 >= 10 + 4 * st["cycles"]


def test_graph_cache_distinguishes_workspace_layouts():
    """A Poisson-only workspace and a render workspace of the same image size have
    different layouts; reusing one address for both must not reuse a stale graph."""
    scene, cam = _small_prims(n=3000, w=200, h=120)
    mean = [0.5, 0.5, 0.5]
    C, H, W = 3, cam.height, cam.width
    big = G.workspace_size(scene.n, C, W, H, None, None)
    ws = torch.empty(big, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(4)
    maps = torch.as_tensor(rng.laplace(0, 0.1, (C, 2, H, W)).astype(np.float32)).cuda()
    img = torch.empty((C, H, W), device="cuda")
    small = ws[:G.workspace_size(0, C, W, H, None, None)]
    G.poisson_reconstruct(maps, mean, img, small)  # builds a graph for the Poisson-only layout
    assert G.sync_status(small)["status"] == 0
    g = G.gaussians_to_device(scene)
    G.render_view(g, cam, mean, img, ws)  # same base address, render layout
    st = G.sync_status(ws)
    assert st["status"] == 0
    ref, _, _ = O.render_view(scene, cam, mean, oracle_opts(G.raster_opts()))
    assert np.isfinite(img.cpu().numpy()).all()
    assert img_err(img.cpu().numpy().astype(np.float64), ref)[1] <= IMG_TOL


@pytest.mark.parametrize("coarse", [2, 16])
@pytest.mark.parametrize("nu", [(1, 1), (3, 2)])
@pytest.mark.parametrize("omega", [1.0, 1.2])
def test_poisson_solver_options(coarse, nu, omega):
    """Other coarsest-grid sizes (down to 2x2, up to 16x16), sweep counts and
    smoother relaxations reach the same solution."""
    rng = np.random.default_rng(coarse * 10 + nu[0])
    H, W = 150, 211
    maps = rng.laplace(0, 0.1, (2, 2, H, W)).astype(np.float32)
    so = G.solver_opts(coarse_max_dim=coarse, nu1=nu[0], nu2=nu[1], omega=omega)
    img, st = gpu_poisson(maps, [0.5, 0.5], so)
    ref = O.poisson_neumann(O.divergence(maps.astype(np.float64)), [0.5, 0.5])
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
    assert img_err(img, ref)[0] <= IMG_TOL


def test_relaxation_changes_speed_not_the_answer():
    """omega = 1 (plain Gauss-Seidel) and omega = 1.2 give images that agree to the
    solver tolerance; with one workspace, the graph cache keeps the two apart."""
    rng = np.random.default_rng(21)
    C, H, W = 3, 270, 480
    maps = torch.as_tensor(rng.laplace(0, 0.1, (C, 2, H, W)).astype(np.float32)).cuda()
    ws = torch.empty(G.workspace_size(0, C, W, H, None, None), dtype=torch.uint8, device="cuda")

    def solve(omega):
        img = torch.empty((C, H, W), device="cuda")
        G.poisson_reconstruct(maps, [0.5] * C, img, ws, sopts=G.solver_opts(omega=omega))
        st = G.sync_status(ws)
        assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
        return img.cpu().numpy().astype(np.float64), st["cycles"]

    i1, k1 = solve(1.0)
    i2, k2 = solve(1.2)
    i3, k3 = solve(1.0)
    assert k2 <= k1 == k3
    assert np.array_equal(i1, i3)
    assert not np.array_equal(i1, i2)  # a stale graph would have repeated omega = 1
    assert np.abs(i1 - i2).max() <= IMG_TOL
    ref = O.poisson_neumann(O.divergence(maps.cpu().numpy().astype(np.float64)), [0.5] * C)
    assert img_err(i2, ref)[0] <= IMG_TOL


def test_coarse_factor_cache_survives_other_layouts_and_detects_corruption():
    """The FP64 coarse factor cached in the workspace is reused only when it is
    intact: solves of other shapes in the same buffer, or bytes overwritten inside
    the cached factor, lead to a rebuild and the same answer."""
    rng = np.random.default_rng(8)
    mA = rng.laplace(0, 0.1, (2, 2, 120, 170)).astype(np.float32)
    mB = rng.laplace(0, 0.1, (1, 2, 300, 90)).astype(np.float32)
    soA = G.solver_opts(coarse_max_dim=16)
    soB = G.solver_opts(coarse_max_dim=2)
    nb = max(G.workspace_size(0, 2, 170, 120, None, soA), G.workspace_size(0, 1, 90, 300, None, soB))
    ws = torch.zeros(nb, dtype=torch.uint8, device="cuda")

    def solve(m, so):
        t = torch.as_tensor(m).cuda()
        img = torch.empty((m.shape[0],) + m.shape[2:], device="cuda")
        G.poisson_reconstruct(t, [0.5] * m.shape[0], img, ws, sopts=so)
        st = G.sync_status(ws)
        assert st["status"] == 0, st
        return img.cpu().numpy()

    a1 = solve(mA, soA)
    solve(mB, soB)
    a2 = solve(mA, soA)
    assert np.array_equal(a1, a2)
    ws[8192:8192 + 4096] = torch.randint(0, 255, (4096,), dtype=torch.uint8, device="cuda")
    a3 = solve(mA, soA)
    assert np.array_equal(a1, a3)
    ref = O.poisson_neumann(O.divergence(mA.astype(np.float64)), [0.5, 0.5])
    assert img_err(a1.astype(np.float64), ref)[0] <= IMG_TOL


# ------------------------------------------------------------------ Laplacian Gaussians (Eq. gdgs)

def test_laplacian_field_matches_oracle():
    scene = S.with_laplacian_attribute(S.tiny_scene(2))
    cam = S.tiny_camera(96, 64)
    gm, _, st = gpu_maps(scene, cam)
    om, amb = oracle_maps(scene, cam)
    assert st["status"] == 0 and gm.shape == om.shape == (3, 64, 96)
    ok = amb == 0
    assert np.abs(gm - om)[:, ok].max() <= MAP_TOL * np.abs(om).max()


def _well_posed_threshold(scene, rho, amb, candidates):
    """A threshold t for which no pixel's decision |rho| >= t lies within the composite
    error bound the map parity test enforces (MAP_TOL * max|rho| for clear pixels, plus
    alpha_min * max|A| where a Gaussian sits at the alpha_min cut). The decision is
    discrete: at such a t both sides must take the same one at every pixel."""
    a = np.abs(rho)
    ref = a.max()
    margin = np.where(amb[None] > 0, np.abs(scene.grad).max() / 255.0 + MAP_TOL * ref, MAP_TOL * ref)
    for t in candidates:
        t = float(np.float32(t))
        if np.all(np.abs(a - t) > margin):
            return t
    return None


@pytest.mark.parametrize("t", [0.0, 0.004])
def test_render_view_laplacian_with_threshold(t):
    # a small ragged view: few enough pixels that thresholds with a decision margin exist
    scene, cam = _small_prims(n=3000, w=136, h=100)
    scene = S.with_laplacian_attribute(scene)
    mean = [0.5, 0.4, 0.6]
    if t > 0:
        rho, amb = oracle_maps(scene, cam)
        t = _well_posed_threshold(scene, rho, amb, [t * (1 + 0.005 * i) for i in range(400)])
        assert t is not None
        assert 0.2 < (np.abs(rho) < t).mean() < 0.9  # the threshold removes a real share
    img, st = _render(scene, cam, mean, sopts=G.solver_opts(rho_threshold=t))
    ref, _, _ = O.render_view(scene, cam, mean, oracle_opts(G.raster_opts()), rho_threshold=t)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-6, st
    assert img_err(img, ref)[1] <= IMG_TOL


def test_poisson_reconstruct_rho_entry_point():
    rng = np.random.default_rng(12)
    rho = rng.laplace(0, 0.05, (2, 70, 90)).astype(np.float32)
    ws = torch.empty(G.workspace_size(0, 2, 90, 70), dtype=torch.uint8, device="cuda")
    img = torch.empty((2, 70, 90), device="cuda")
    G.poisson_reconstruct_rho(torch.as_tensor(rho).cuda(), [0.5, 0.5], img, ws,
                              sopts=G.solver_opts(rho_threshold=0.03))
    st = G.sync_status(ws)
    ref = O.poisson_neumann(O.threshold(rho.astype(np.float64), np.float32(0.03)), [0.5, 0.5])
    assert st["status"] == 0
    assert img_err(img.cpu().numpy().astype(np.float64), ref)[0] <= IMG_TOL

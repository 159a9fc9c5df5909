"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each pin checks the oracle through a route that does not retype its formula:
closed forms, library routines (scipy rotations, scipy DCT, dense numpy solves),
finite differences, Monte Carlo, brute force on tiny inputs, and invariants.
The paper prints no worked numerical example, so whole-pipeline parity against the
paper itself is unpinned; the hand-worked composite fixture follows Eq. gdgs2d.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.linalg
import scipy.sparse
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2405_05446_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _one(mean, scale, quat, opacity=0.8, grad=None, C=3):
    g = np.zeros((1, C, 2), np.float32) if grad is None else np.asarray(grad, np.float32).reshape(1, C, 2)
    return S.Scene(np.asarray([mean], np.float32), np.asarray([scale], np.float32),
                   np.asarray([quat], np.float32), np.asarray([opacity], np.float32), g)


def _w2c(cam):
    return np.asarray(cam.world_to_cam, np.float32).astype(np.float64)


def _f32(v):  # the camera reaches the library as float32 (gdgs_camera)
    return float(np.float32(v))


def _pinhole(cam, x_cam):
    return np.array([_f32(cam.fx) * x_cam[0] / x_cam[2] + _f32(cam.cx),
                     _f32(cam.fy) * x_cam[1] / x_cam[2] + _f32(cam.cy)])


# ------------------------------------------------------------------ projection (Eq. sig2d)

def test_isotropic_on_axis_closed_form():
    """Isotropic Gaussian of scale s at depth z on the optical axis:
    Sigma2D = (f s / z)^2 I + dil I and the centre maps to the principal point."""
    cam = S.tiny_camera(64, 64)
    s, opts = 0.02, O.RasterOpts(dilation=0.3)
    r = O.project(_one([0, 0, 0], [s, s, s], [1, 0, 0, 0]), cam, opts)[0]
    z = 3.0
    exp = (cam.fx * s / z) ** 2 + 0.3
    assert r[O.VALID] == 1
    assert r[O.DEPTH] == pytest.approx(z, abs=1e-12)
    assert r[O.S00] == pytest.approx(exp, rel=1e-6) and r[O.S11] == pytest.approx(exp, rel=1e-6)
    assert abs(r[O.S01]) < 1e-9
    assert r[O.MX] == pytest.approx(cam.cx, abs=1e-9) and r[O.MY] == pytest.approx(cam.cy, abs=1e-9)


def test_rotation_about_view_axis_swaps_axes():
    """A 90 degree turn about the view axis swaps the projected variances."""
    cam = S.tiny_camera(64, 64)
    opts = O.RasterOpts(dilation=0.0)
    sc = (0.05, 0.01, 0.02)
    a = O.project(_one([0, 0, 0], sc, [1, 0, 0, 0]), cam, opts)[0]
    c45 = math.cos(math.pi / 4)
    b = O.project(_one([0, 0, 0], sc, [c45, 0, 0, c45]), cam, opts)[0]
    fz = cam.fx / 3.0
    assert a[O.S00] == pytest.approx((fz * 0.05) ** 2, rel=1e-6)
    assert a[O.S11] == pytest.approx((fz * 0.01) ** 2, rel=1e-6)
    assert b[O.S00] == pytest.approx(a[O.S11], rel=1e-5)
    assert b[O.S11] == pytest.approx(a[O.S00], rel=1e-5)


@pytest.mark.parametrize("seed", range(5))
def test_sigma2d_matches_fd_jacobian_and_scipy_rotation(seed):
    """Sigma2D = J W Sigma W^T J^T with J from central differences of the pinhole map
    and Sigma built from scipy's quaternion rotation (scalar-last convention)."""
    rng = np.random.default_rng(seed)
    cam = S.look_at_camera(rng.normal(size=3) * 0.3 + [0.2, -0.1, -3.0], [0.1, 0.2, 0.0], 96, 80,
                           hfov_deg=60.0)
    mean = rng.uniform(-0.7, 0.7, 3)
    scale = np.exp(rng.normal(-3.0, 0.5, 3))
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    r = O.project(_one(mean.astype(np.float32), scale.astype(np.float32), q.astype(np.float32)),
                  cam, O.RasterOpts(dilation=0.0))[0]
    mean32 = mean.astype(np.float32).astype(np.float64)
    s32 = scale.astype(np.float32).astype(np.float64)
    q32 = q.astype(np.float32).astype(np.float64)
    rot = Rotation.from_quat([q32[1], q32[2], q32[3], q32[0]]).as_matrix()
    sigma = rot @ np.diag(s32 ** 2) @ rot.T
    w = _w2c(cam)
    t = w[:, :3] @ mean32 + w[:, 3]
    h = 1e-5
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (_pinhole(cam, t + e) - _pinhole(cam, t - e)) / (2 * h)
    s2 = J @ w[:, :3] @ sigma @ w[:, :3].T @ J.T
    got = np.array([[r[O.S00], r[O.S01]], [r[O.S01], r[O.S11]]])
    np.testing.assert_allclose(got, s2, rtol=1e-6, atol=1e-9 * np.abs(s2).max())
    np.testing.assert_allclose([r[O.MX], r[O.MY]], _pinhole(cam, t), rtol=0, atol=1e-9)
    # conic is the inverse of Sigma2D
    conic = np.array([[r[O.CA], r[O.CB]], [r[O.CB], r[O.CC]]])
    np.testing.assert_allclose(conic @ got, np.eye(2), atol=1e-9)


def test_sigma2d_monte_carlo():
    """The projected covariance equals the covariance of projected samples (small
    Gaussian, so the local affine approximation of Eq. sig2d is accurate)."""
    rng = np.random.default_rng(7)
    cam = S.look_at_camera((0.4, 0.3, -3.0), (0.0, 0.0, 0.0), 128, 128)
    mean = np.array([0.3, -0.2, 0.1])
    scale = np.array([0.01, 0.004, 0.007])
    q = np.array([0.9, 0.2, -0.3, 0.25])
    q /= np.linalg.norm(q)
    r = O.project(_one(mean, scale, q), cam, O.RasterOpts(dilation=0.0))[0]
    m32 = mean.astype(np.float32).astype(np.float64)
    s32 = scale.astype(np.float32).astype(np.float64)
    q32 = q.astype(np.float32).astype(np.float64)
    rot = Rotation.from_quat([q32[1], q32[2], q32[3], q32[0]]).as_matrix()
    x = m32 + (rng.standard_normal((400_000, 3)) * s32) @ rot.T
    w = _w2c(cam)
    xc = x @ w[:, :3].T + w[:, 3]
    uv = np.stack([cam.fx * xc[:, 0] / xc[:, 2], cam.fy * xc[:, 1] / xc[:, 2]], axis=1)
    cov = np.cov(uv.T)
    got = np.array([[r[O.S00], r[O.S01]], [r[O.S01], r[O.S11]]])
    np.testing.assert_allclose(got, cov, rtol=2e-2, atol=2e-2 * np.abs(cov).max())


def test_near_cull_and_behind_camera():
    cam = S.tiny_camera()
    r = O.project(_one([0, 0, -2.9], [0.01] * 3, [1, 0, 0, 0]), cam)[0]  # depth 0.1 < near
    assert r[O.VALID] == 0
    r = O.project(_one([0, 0, -4.0], [0.01] * 3, [1, 0, 0, 0]), cam)[0]  # behind
    assert r[O.VALID] == 0
    r = O.project(_one([0, 0, 0], [0.01] * 3, [0, 0, 0, 0]), cam)[0]  # no rotation
    assert r[O.VALID] == 0
    r = O.project(_one([0, 0, 0], [0.01] * 3, [1, 0, 0, 0], opacity=0.001), cam)[0]
    assert r[O.VALID] == 0  # never reaches alpha_min


# ------------------------------------------------------------------ footprint

@pytest.mark.parametrize("kexp", [1.0, 0.5])
def test_footprint_box_tight_and_conservative(kexp):
    """The box is the exact bounding box of {opacity * exp(-k d^T conic d) >= alpha_min}:
    no sampled point outside has alpha >= alpha_min and the extreme ellipse points sit
    exactly on alpha_min."""
    rng = np.random.default_rng(3)
    cam = S.tiny_camera(64, 64)
    opts = O.RasterOpts(exp_coef=kexp)
    for _ in range(5):
        q = rng.normal(size=4)
        sc = _one(rng.uniform(-0.3, 0.3, 3), np.exp(rng.normal(-3, 0.5, 3)), q,
                  opacity=rng.uniform(0.2, 0.9))
        r = O.project(sc, cam, opts)[0]
        sig = np.array([[r[O.S00], r[O.S01]], [r[O.S01], r[O.S11]]])
        lev = math.log(r[O.OPA] / opts.alpha_min)
        # extreme point in x of the ellipse d^T Sigma^-1 d = lev / k: d = Sigma e_x * c
        for ax, (lo, hi) in enumerate([(O.XMIN, O.XMAX), (O.YMIN, O.YMAX)]):
            e = np.zeros(2)
            e[ax] = 1
            d = sig @ e * math.sqrt(lev / kexp / (e @ sig @ e))
            conic = np.linalg.inv(sig)
            a = r[O.OPA] * math.exp(-kexp * d @ conic @ d)
            assert a == pytest.approx(opts.alpha_min, rel=1e-9)
            centre = r[O.MX] if ax == 0 else r[O.MY]
            assert centre + d[ax] == pytest.approx(r[hi], rel=1e-12)
            assert centre - d[ax] == pytest.approx(r[lo], rel=1e-12)
        # brute force on a fine grid around the splat
        xs = np.linspace(r[O.XMIN] - 5, r[O.XMAX] + 5, 301)
        ys = np.linspace(r[O.YMIN] - 5, r[O.YMAX] + 5, 301)
        X, Y = np.meshgrid(xs, ys)
        dx, dy = X - r[O.MX], Y - r[O.MY]
        conic = np.linalg.inv(sig)
        a = r[O.OPA] * np.exp(-kexp * (conic[0, 0] * dx * dx + 2 * conic[0, 1] * dx * dy
                                       + conic[1, 1] * dy * dy))
        outside = (X < r[O.XMIN]) | (X > r[O.XMAX]) | (Y < r[O.YMIN]) | (Y > r[O.YMAX])
        assert not np.any(a[outside] >= opts.alpha_min)


# ------------------------------------------------------------------ compositing (Eq. gdgs2d)

def _hand_rows(alphas, depths, centres, W=8):
    rows = np.zeros((len(alphas), O.STRIDE))
    for k, (a, d, (x, y)) in enumerate(zip(alphas, depths, centres)):
        rows[k, O.VALID] = 1
        rows[k, O.DEPTH] = d
        rows[k, O.DERR] = 4 * 2.0 ** -24 * abs(d)
        rows[k, O.KAPPA] = 1.0
        rows[k, O.LMAX] = 2.0  # Sigma2D = 2 I (conic 0.5 I)
        rows[k, O.BOXW] = 1.0
        rows[k, O.TZ0], rows[k, O.TZ1], rows[k, O.TZ2] = x, y, d  # terms of the depth
        rows[k, O.MX], rows[k, O.MY] = x, y
        rows[k, O.CA], rows[k, O.CB], rows[k, O.CC] = 0.5, 0.0, 0.5
        rows[k, O.OPA] = a
        rows[k, O.XMIN], rows[k, O.XMAX] = -1e9, 1e9
        rows[k, O.YMIN], rows[k, O.YMAX] = -1e9, 1e9
    return rows


def _hand_scene(g):
    n = len(g)
    grad = np.zeros((n, 1, 2), np.float32)
    grad[:, 0, 0] = g
    grad[:, 0, 1] = -np.asarray(g)
    return S.Scene(np.zeros((n, 3), np.float32), np.ones((n, 3), np.float32),
                   np.tile(np.float32([1, 0, 0, 0]), (n, 1)), np.ones(n, np.float32), grad)


def test_composite_hand_worked_fixture():
    fx = json.load(open(os.path.join(GOLDEN, "composite_hand.json")))
    cam = S.tiny_camera(8, 8)
    centre = (3.5, 2.5)  # pixel (row 2, col 3)
    # given in reverse: the composite must follow depth, not input order
    rows = _hand_rows(fx["alpha"][::-1], fx["depth"][::-1], [centre] * 3)
    sc = _hand_scene(fx["g"][::-1])
    out, amb = O.render_gradients(sc, cam, mode="all_pairs", pixels=[2 * 8 + 3], proj=rows)
    assert out[0, 0, 0] == pytest.approx(fx["expected"], abs=1e-15)
    assert out[0, 0, 1] == pytest.approx(-fx["expected"], abs=1e-15)
    rows2 = _hand_rows(fx["alpha"][:2], fx["depth"][:2], [centre] * 2)
    out2, _ = O.render_gradients(_hand_scene(fx["g"][:2]), cam, mode="all_pairs",
                                 pixels=[2 * 8 + 3], proj=rows2)
    assert out2[0, 0, 0] == pytest.approx(fx["expected_two_front"], abs=1e-15)


def test_composite_equal_depths_keep_ascending_index():
    """Equal view depths are composited in ascending Gaussian index (the tie-break
    reading of "sorted from the view direction", Eq. color), whatever the input."""
    fx = json.load(open(os.path.join(GOLDEN, "composite_tie.json")))
    cam = S.tiny_camera(8, 8)
    c = (3.5, 2.5)
    # three different centres that all sit on the pixel centre in the hand rows, so
    # the depth ties are real ties of different Gaussians, not one mean repeated
    rows = _hand_rows(fx["alpha"], [fx["depth"]] * 3, [c] * 3)
    rows[:, O.MX] += np.array([0.0, 1e-10, 2e-10])  # distinct; exp(-0.5 dx^2) is 1 in FP64
    rows[:, O.TZ0] = np.array([0.1, -0.2, 0.3])  # different means whose depths tie
    out, amb = O.render_gradients(_hand_scene(fx["g"]), cam, mode="all_pairs", pixels=[19],
                                  proj=rows)
    assert out[0, 0, 0] == pytest.approx(fx["expected"], abs=1e-15)
    assert out[0, 0, 0] != pytest.approx(fx["expected_descending"], abs=1e-3)
    assert amb[0] == 1  # ties between different Gaussians: a float32 sort may order them either way
    # listing the same three Gaussians in reverse must reverse the composite order
    rows_r, g_r = rows[::-1].copy(), fx["g"][::-1]
    out_r, _ = O.render_gradients(_hand_scene(g_r), cam, mode="all_pairs", pixels=[19], proj=rows_r)
    a, g = fx["alpha"][::-1], g_r
    want = g[0] * a[0] + g[1] * a[1] * (1 - a[0]) + g[2] * a[2] * (1 - a[0]) * (1 - a[1])
    assert out_r[0, 0, 0] == pytest.approx(want, abs=1e-15)
    assert want == pytest.approx(fx["expected_descending"], abs=1e-15)
    # the same mean twice: equal float32 depths on any evaluation, so no ambiguity
    rows_same = _hand_rows(fx["alpha"][:2], [fx["depth"]] * 2, [c] * 2)
    _, amb_same = O.render_gradients(_hand_scene(fx["g"][:2]), cam, mode="all_pairs",
                                     pixels=[19], proj=rows_same)
    assert amb_same[0] == 0


def test_composite_near_equal_depths_follow_fp64_and_are_flagged():
    fx = json.load(open(os.path.join(GOLDEN, "composite_tie.json")))
    cam = S.tiny_camera(8, 8)
    c = (3.5, 2.5)
    rows = _hand_rows([0.5, 0.25], [2.0 + 1e-12, 2.0], [c, (3.5 + 1e-10, 2.5)])
    rows[:, O.TZ0] = [0.1, -0.2]
    out, amb = O.render_gradients(_hand_scene([1.0, 2.0]), cam, mode="all_pairs", pixels=[19],
                                  proj=rows)
    assert out[0, 0, 0] == pytest.approx(fx["near_expected"], abs=1e-15)
    assert amb[0] == 1
    # well separated depths: same order, no flag
    rows = _hand_rows([0.5, 0.25], [2.5, 2.0], [c, (3.5 + 1e-10, 2.5)])
    out, amb = O.render_gradients(_hand_scene([1.0, 2.0]), cam, mode="all_pairs", pixels=[19],
                                  proj=rows)
    assert out[0, 0, 0] == pytest.approx(fx["near_expected"], abs=1e-15)
    assert amb[0] == 0


def test_projected_equal_depths_sort_by_index():
    """Through the projection: Gaussians at one camera depth (same z, camera looking
    along +z) get equal FP64 depths and are ordered by index; a farther one goes last."""
    cam = S.tiny_camera(64, 64)
    assert _w2c(cam)[2, 0] == 0 and _w2c(cam)[2, 1] == 0
    n = 4
    sc = S.Scene(np.float32([[0.05, 0.0, 0.1], [-0.05, 0.02, 0.1], [0.0, -0.03, 0.1],
                             [0.0, 0.0, 0.0]]),
                 np.full((n, 3), 0.05, np.float32), np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
                 np.full(n, 0.5, np.float32), np.zeros((n, 1, 2), np.float32))
    rows = O.project(sc, cam)
    assert rows[0, O.DEPTH] == rows[1, O.DEPTH] == rows[2, O.DEPTH] > rows[3, O.DEPTH]
    np.testing.assert_array_equal(O.depth_order(rows), [3, 0, 1, 2])
    perm = [2, 0, 3, 1]
    np.testing.assert_array_equal(O.depth_order(rows[perm]), [2, 0, 1, 3])


def test_near_cull_within_float32_bound_is_flagged():
    """A Gaussian whose FP64 depth is within the float32 depth error bound of the near
    plane is culled (depth <= near) but kept as a ghost that flags the pixels it would
    reach; one just in front contributes and flags them too."""
    cam = S.tiny_camera(16, 16)
    cam.near = 3.0 - 0.0  # the origin sits at depth 3.0 exactly
    for z, valid in ((0.0, 0), (1e-7, 1)):
        sc = _one([0, 0, z], [0.05] * 3, [1, 0, 0, 0], opacity=0.8,
                  grad=np.full((3, 2), 0.5, np.float32))
        r = O.project(sc, cam)[0]
        assert r[O.NEARAMB] == 1 and r[O.VALID] == valid and r[O.GHOST] == 1 - valid
        maps, amb = O.render_gradients(sc, cam)
        assert amb[8, 8] == 1
        assert (np.abs(maps).max() > 0) == bool(valid)
    sc = _one([0, 0, 0.5], [0.05] * 3, [1, 0, 0, 0], opacity=0.8, grad=np.full((3, 2), 0.5, np.float32))
    r = O.project(sc, cam)[0]
    assert r[O.NEARAMB] == 0 and r[O.VALID] == 1
    maps, amb = O.render_gradients(sc, cam)
    assert amb.max() == 0 and np.abs(maps).max() > 0


def test_composite_off_centre_two_splats():
    """Two splats off the pixel centre: g1 a1 + g2 a2 (1 - a1), a = alpha exp(-d^T Q d)."""
    cam = S.tiny_camera(8, 8)
    rows = _hand_rows([0.6, 0.7], [1.0, 1.5], [(3.0, 2.5), (4.5, 3.5)])
    p = (3.5, 2.5)
    a1 = 0.6 * math.exp(-(0.5 * 0.25))
    a2 = 0.7 * math.exp(-(0.5 * 1.0 + 0.5 * 1.0))
    out, _ = O.render_gradients(_hand_scene([0.3, -0.8]), cam, mode="all_pairs", pixels=[2 * 8 + 3],
                                proj=rows)
    g1, g2 = float(np.float32(0.3)), float(np.float32(-0.8))  # attributes are stored as float32
    assert out[0, 0, 0] == pytest.approx(g1 * a1 + g2 * a2 * (1 - a1), rel=1e-14)


def test_composite_alpha_min_skip_and_t_min_stop():
    cam = S.tiny_camera(8, 8)
    c = (3.5, 2.5)
    # opacity below alpha_min at the centre: skipped, does not attenuate
    rows = _hand_rows([0.003, 0.5], [1.0, 2.0], [c, c])
    out, _ = O.render_gradients(_hand_scene([10.0, 1.0]), cam, mode="all_pairs", pixels=[19],
                                proj=rows)
    assert out[0, 0, 0] == pytest.approx(0.5, abs=1e-15)
    # T drops below t_min after the second splat (T = 0.01 * 0.005 < 1e-4): third ignored
    rows = _hand_rows([0.99, 0.995, 0.5], [1.0, 2.0, 3.0], [c, c, c])
    opts = O.RasterOpts(alpha_max=0.999)
    out, _ = O.render_gradients(_hand_scene([1.0, 1.0, 100.0]), cam, opts, mode="all_pairs",
                                pixels=[19], proj=rows)
    assert out[0, 0, 0] == pytest.approx(0.99 + 0.995 * 0.01, abs=1e-14)
    # alpha_max clamps
    rows = _hand_rows([1.0], [1.0], [c])
    out, _ = O.render_gradients(_hand_scene([1.0]), cam, mode="all_pairs", pixels=[19], proj=rows)
    assert out[0, 0, 0] == pytest.approx(0.99, abs=1e-15)


def test_single_splat_peak_is_alpha_times_g():
    """A splat whose centre falls on a pixel centre peaks at alpha * g there."""
    cam = S.tiny_camera(64, 64)
    cam.cx, cam.cy = 32.5, 20.5  # the origin projects onto the centre of pixel (20, 32)
    g = np.array([[0.3, -0.2], [0.1, 0.05], [-0.4, 0.7]], np.float32)
    sc = _one([0, 0, 0], [0.02, 0.03, 0.01], [0.9, 0.1, 0.3, -0.2], opacity=0.7, grad=g)
    maps, amb = O.render_gradients(sc, cam)
    peak = maps[:, :, 20, 32]
    np.testing.assert_allclose(peak, np.float32(0.7) * g.astype(np.float64), rtol=1e-12)
    assert np.abs(maps).max() == pytest.approx(np.abs(peak).max(), rel=1e-12)


@pytest.mark.parametrize("seed", range(100))
def test_box_mode_equals_all_pairs(seed):
    """Brute force over all Gaussians equals the footprint-box pre-filter exactly."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 65))
    sc = S.tiny_scene(seed, n=n)
    sc.scale *= np.float32(rng.uniform(0.5, 3.0))
    cam = S.tiny_camera(32, 32)
    a, amb_a = O.render_gradients(sc, cam, mode="all_pairs")
    b, amb_b = O.render_gradients(sc, cam, mode="box")
    assert np.array_equal(a, b)
    assert np.array_equal(amb_a, amb_b)


def test_pixel_list_equals_full_image():
    sc, cam = S.tiny_scene(1, n=200), S.tiny_camera(48, 40)
    full, amb = O.render_gradients(sc, cam)
    pix = np.array([0, 5, 47, 48 * 20 + 7, 48 * 40 - 1])
    part, pamb = O.render_gradients(sc, cam, pixels=pix, mode="all_pairs")
    C = full.shape[0]
    for k, p in enumerate(pix):
        i, j = divmod(int(p), 48)
        np.testing.assert_array_equal(part[k], full[:, :, i, j])
        assert pamb[k] == amb[i, j]


# ------------------------------------------------------------------ divergence and Poisson (Eq. p2d)

def _neumann_matrix(h, w):
    """Neumann 5-point Laplacian built from 1D second differences with a Kronecker sum."""
    def d1(n):
        m = np.zeros((n, n))
        for i in range(n):
            if i > 0:
                m[i, i - 1] = 1
                m[i, i] -= 1
            if i < n - 1:
                m[i, i + 1] = 1
                m[i, i] -= 1
        return m
    return np.kron(np.eye(h), d1(w)) + np.kron(d1(h), np.eye(w))


def test_divergence_of_forward_gradients_is_laplacian():
    rng = np.random.default_rng(0)
    img = rng.normal(size=(2, 9, 13))
    rho = O.divergence(O.forward_gradients(img))
    lap = (_neumann_matrix(9, 13) @ img.reshape(2, -1).T).T.reshape(img.shape)
    np.testing.assert_allclose(rho, lap, atol=1e-12)
    np.testing.assert_allclose(O.laplacian_neumann(img), lap, atol=1e-12)
    # any gradient field: sum(rho) = 0 (zero flux through the border)
    g = rng.normal(size=(3, 2, 11, 7))
    assert abs(O.divergence(g).sum()) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 7, 16, 135])
def test_dct_matrix_matches_scipy(n):
    x = np.random.default_rng(n).normal(size=(n, 3))
    ref = scipy.fft.dct(x, type=2, norm="ortho", axis=0)
    np.testing.assert_allclose(O.dct_matrix(n) @ x, ref, atol=1e-12)
    np.testing.assert_allclose(O.dct_matrix(n) @ O.dct_matrix(n).T, np.eye(n), atol=1e-12)


@pytest.mark.parametrize("hw", [(1, 1), (1, 5), (4, 4), (9, 15), (16, 16), (7, 3)])
def test_poisson_matches_dense_bordered_solve(hw):
    """Against a dense solve of [L 1; 1^T 0][u; lam] = [rho - mean(rho); 0]."""
    h, w = hw
    rng = np.random.default_rng(h * 100 + w)
    rho = rng.normal(size=(2, h, w))
    u = O.poisson_neumann(rho, [0.0, 0.0])
    n = h * w
    L = _neumann_matrix(h, w)
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = L
    A[:n, n] = 1
    A[n, :n] = 1
    for c in range(2):
        f = rho[c].reshape(-1)
        x = np.linalg.solve(A, np.concatenate([f, [0.0]]))
        np.testing.assert_allclose(u[c].reshape(-1), x[:n], atol=1e-10)


@pytest.mark.parametrize("hw", [(64, 64), (45, 70), (17, 9)])
def test_poisson_recovers_image_from_fd_gradients(hw):
    """FD gradients of a known image -> divergence -> solve -> the image (to 1e-9)
    once the constant is fixed (Sec. 2.1: exact up to a constant difference)."""
    h, w = hw
    img = np.stack([S.image_from_gradients_test_image(h, w, seed=s) for s in range(3)])
    rho = O.divergence(O.forward_gradients(img))
    u = O.poisson_neumann(rho, img.mean(axis=(1, 2)))
    np.testing.assert_allclose(u, img, atol=1e-9)


def test_poisson_residual_zero_mean_and_channels_independent():
    rng = np.random.default_rng(5)
    g = rng.laplace(0, 0.1, size=(3, 2, 30, 40))
    rho = O.divergence(g)
    assert abs(rho.sum()) < 1e-12
    u = O.poisson_neumann(rho, [0.5, 0.2, -0.1])
    r = rho - O.laplacian_neumann(u)
    assert np.abs(r).max() < 1e-11
    assert abs(r.mean()) < 1e-14
    np.testing.assert_allclose(u.mean(axis=(1, 2)), [0.5, 0.2, -0.1], atol=1e-14)
    u1 = O.poisson_neumann(rho[1:2], [0.2])
    np.testing.assert_allclose(u1[0], u[1], atol=1e-13)


def test_poisson_inconsistent_rhs_is_least_squares():
    """With sum(rho) != 0 the result solves L u = rho - mean(rho)."""
    rng = np.random.default_rng(9)
    rho = rng.normal(size=(1, 12, 10)) + 0.3
    u = O.poisson_neumann(rho, [0.0])
    r = rho - O.laplacian_neumann(u)
    np.testing.assert_allclose(r, np.full_like(r, rho.mean()), atol=1e-10)


def test_poisson_minimises_variational_energy():
    """The solution minimises E(u) = 1/2 sum_faces (u_n - u)^2 + sum u rho, the discrete
    form of the energy whose Euler-Lagrange equation is Eq. p2d (Sec. 3.2.4, L_e)."""
    rng = np.random.default_rng(11)
    rho = O.divergence(rng.normal(size=(1, 2, 20, 24)))

    def energy(u):
        return 0.5 * (np.sum(np.diff(u, axis=-1) ** 2) + np.sum(np.diff(u, axis=-2) ** 2)) + np.sum(u * rho)

    u = O.poisson_neumann(rho, [0.0])
    e0 = energy(u)
    for _ in range(20):
        d = rng.normal(size=u.shape) * 1e-3
        assert energy(u + d) > e0


def test_poisson_rejects_planted_sign_error():
    """A plausible mistake planted in the oracle (wrong eigenvalue sign) fails the pins."""
    rho = O.divergence(O.forward_gradients(np.stack([S.image_from_gradients_test_image(20, 30)])))
    good = O.poisson_neumann(rho, [0.5])
    orig = O.poisson_neumann

    def planted(rho, mean):
        return -orig(rho, [0.0]) + np.asarray(mean)[:, None, None]

    bad = planted(rho, [0.5])
    assert np.abs(rho - O.laplacian_neumann(good)).max() < 1e-10
    assert np.abs(rho - O.laplacian_neumann(bad)).max() > 1e-3


def test_divergence_rejects_planted_index_error():
    img = np.stack([S.image_from_gradients_test_image(10, 12)])
    g = O.forward_gradients(img)
    bad = g.copy()
    bad[:, 0] = np.roll(bad[:, 0], 1, axis=-1)  # gx taken at the wrong column
    assert np.abs(O.divergence(g) - O.laplacian_neumann(img)).max() < 1e-12
    assert np.abs(O.divergence(bad) - O.laplacian_neumann(img)).max() > 1e-3


# ------------------------------------------------------------------ whole tiny pipeline

def test_tiny_pipeline_golden_samples():
    """Regression of the tiny 64x64 workload against samples written by
    tests/golden/make_golden.py (which calls only the oracle)."""
    path = os.path.join(GOLDEN, "tiny64_oracle_samples.json")
    ref = json.load(open(path))
    sc, cam, mean, _ = S.workload("tiny64")
    img, maps, amb = O.render_view(sc, cam, mean)
    for s in ref["samples"]:
        c, i, j = s["c"], s["i"], s["j"]
        assert maps[c, 0, i, j] == pytest.approx(s["gx"], abs=1e-12)
        assert maps[c, 1, i, j] == pytest.approx(s["gy"], abs=1e-12)
        assert img[c, i, j] == pytest.approx(s["img"], abs=1e-10)
    assert int(amb.sum()) == ref["ambiguous"]


def test_laplacian_attribute_hand_fixture_and_threshold():
    """Scalar (Laplacian) attributes composite by the same rule (Eq. gdgs2d with the
    c_k of Eq. gdgs); T keeps values at or above t in magnitude (Eq. thresh)."""
    fx = json.load(open(os.path.join(GOLDEN, "composite_hand.json")))
    cam = S.tiny_camera(8, 8)
    rows = _hand_rows(fx["alpha"], fx["depth"], [(3.5, 2.5)] * 3)
    sc = _hand_scene(fx["g"])
    sc = S.Scene(sc.mean, sc.scale, sc.quat, sc.opacity, np.ascontiguousarray(sc.grad[:, :, 0]))
    out, _ = O.render_gradients(sc, cam, mode="all_pairs", pixels=[19], proj=rows)
    assert out.shape == (1, 1) and out[0, 0] == pytest.approx(fx["expected"], abs=1e-15)
    x = np.array([-0.5, -0.003, -0.002, 0.0, 0.002, 0.003, 0.7])
    np.testing.assert_array_equal(O.threshold(x, 0.003), [-0.5, -0.003, 0, 0, 0, 0.003, 0.7])


def test_laplacian_scene_box_equals_all_pairs():
    sc = S.with_laplacian_attribute(S.tiny_scene(4, n=40))
    cam = S.tiny_camera(32, 32)
    a, _ = O.render_gradients(sc, cam, mode="all_pairs")
    b, _ = O.render_gradients(sc, cam, mode="box")
    assert a.shape == (3, 32, 32) and np.array_equal(a, b)
    img, maps, _ = O.render_view(sc, cam, [0.5, 0.5, 0.5])
    r = maps - O.laplacian_neumann(img)
    np.testing.assert_allclose(r, np.broadcast_to(maps.mean(axis=(1, 2), keepdims=True), r.shape),
                               atol=1e-10)

"""Pins of the differentiable FP64 oracle (oracle/diff.py), CPU only: its forward is
the C oracle's, its gradient matches central finite differences in FP64, and the
adjoint of the Poisson stage is the same zero-mean solve (L is symmetric)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import diff as D
from paper_2405_05446_gb300 import scenes as S

SMOOTH = O.RasterOpts(alpha_min=1e-10, alpha_max=0.99, t_min=0.0)


def _scene64(seed=0, laplacian=False):
    sc = S.tiny_scene(seed, n=64)
    sc = S.Scene(sc.mean * 0.6, sc.scale * 1.6, sc.quat, np.minimum(sc.opacity, 0.9).astype(np.float32), sc.grad)
    if laplacian:
        sc = S.with_laplacian_attribute(sc)
    cam = S.look_at_camera((0.3, -0.2, -3.0), (0.0, 0.0, 0.0), 128, 128, hfov_deg=40)
    return sc, cam


@pytest.mark.parametrize("laplacian,t", [(False, 0.0), (True, 0.0), (True, 0.004)])
def test_forward_equals_c_oracle(laplacian, t):
    sc = S.tiny_scene(4, n=300)
    if laplacian:
        sc = S.with_laplacian_attribute(sc)
    cam = S.look_at_camera((0.2, 0.1, -3.0), (0.0, 0.0, 0.0), 48, 40)
    mean = [0.5, 0.3, 0.7]
    ref, _, _ = O.render_view(sc, cam, mean, O.RasterOpts(), rho_threshold=t)
    got = D.render_view(D.scene_params(sc, False), sc, cam, mean, O.RasterOpts(), rho_threshold=t)
    np.testing.assert_allclose(got.detach().numpy(), ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("laplacian", [False, True])
def test_gradient_matches_central_differences(laplacian):
    """64 Gaussians, 128 x 128, FP64: autograd against (f(x+h) - f(x-h)) / 2h on a
    sample of parameters of every kind."""
    sc, cam = _scene64(1, laplacian)
    mean = [0.5, 0.5, 0.5]
    rng = np.random.default_rng(7)
    w = rng.standard_normal((3, cam.height, cam.width))
    g = D.gradients(sc, cam, mean, SMOOTH, w)
    wt = torch.tensor(w)

    def loss(p):
        return float((D.render_view(p, sc, cam, mean, SMOOTH) * wt).sum())

    checked = 0
    for k in D.PARAMS:
        base = D.scene_params(sc, False)
        flat = base[k].reshape(-1)
        picks = rng.choice(flat.numel(), size=6, replace=False)
        for i in picks:
            x0 = float(flat[i])
            h = 1e-6 * max(1.0, abs(x0))
            p = {kk: vv.clone() for kk, vv in base.items()}
            p[k].reshape(-1)[i] = x0 + h
            fp = loss(p)
            p[k].reshape(-1)[i] = x0 - h
            fm = loss(p)
            fd = (fp - fm) / (2 * h)
            an = float(g[k].reshape(-1)[i])
            scale = max(np.abs(g[k]).max(), 1e-12)
            assert abs(fd - an) <= 2e-6 * scale + 1e-7 * abs(an), (k, int(i), fd, an)
            checked += 1
    assert checked == 6 * len(D.PARAMS)


def test_poisson_adjoint_is_the_zero_mean_solve():
    """d<w, solve(rho)>/d rho = solve(w) with mean 0, for any rho (also one whose sum
    is not zero, which the solve treats in the least-squares sense)."""
    rng = np.random.default_rng(3)
    rho = torch.tensor(rng.standard_normal((2, 17, 23)), requires_grad=True)
    w = rng.standard_normal((2, 17, 23))
    (D.poisson_neumann(rho, [0.3, -0.1]) * torch.tensor(w)).sum().backward()
    expect = O.poisson_neumann(w, [0.0, 0.0])
    np.testing.assert_allclose(rho.grad.numpy(), expect, rtol=0, atol=1e-12)

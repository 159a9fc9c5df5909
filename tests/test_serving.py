"""Serving (resident scenes, continuous batching of mixed-resolution views replayed
as captured CUDA graphs, admission under a memory budget). GPU tests compare every
served image with the same view rendered alone; the request generator is checked
on the CPU."""
import numpy as np
import pytest

from paper_2405_05446_gb300 import scenes as S


def test_mixed_requests_are_a_poisson_process():
    from paper_2405_05446_gb300 import serving as SV
    reqs = SV.mixed_requests(4000, rate=500.0, seed=3)
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(t)
    assert t[0] == 0.0 and np.all(gaps >= 0)
    assert abs(gaps.mean() - 1 / 500.0) < 0.1 / 500.0          # mean gap 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1           # exponential: cv = 1
    sizes = [(r.cam.width, r.cam.height) for r in reqs]
    counts = {s: sizes.count(s) for s in SV.SIZES}
    assert all(600 < c < 1000 for c in counts.values())        # uniform over 5 sizes
    scenes = [r.scene for r in reqs]
    assert set(scenes) == {0, 1, 2, 3}
    eyes = np.array([-r.cam.world_to_cam[:, :3].astype(np.float64).T @ r.cam.world_to_cam[:, 3] for r in reqs[:500]])
    np.testing.assert_allclose(np.linalg.norm(eyes, axis=1), 3.0, rtol=1e-5)
    assert np.abs(eyes.mean(axis=0)).max() < 0.25              # uniform on the sphere


torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def _lib():
    from gpu_util import ensure_lib
    ensure_lib()


def _scenes():
    cam = S.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 200, 120)
    return [S.primitives_scene(0, n=5000, orient_camera=cam), S.primitives_scene(1, n=20000, orient_camera=cam)]


SMALL_SIZES = [(64, 64), (128, 96), (200, 120)]


def _requests(n, seed, keep=True):
    from paper_2405_05446_gb300 import serving as SV
    reqs = SV.mixed_requests(n, rate=1e6, seed=seed, n_scenes=2, sizes=SMALL_SIZES)
    for r in reqs:
        r.keep = keep
    return reqs


@pytest.mark.gpu
def test_captured_view_graph_replays_any_camera(_lib):
    import paper_2405_05446_gb300 as G
    scene = _scenes()[1]
    g = G.gaussians_to_device(scene)
    W, H = 200, 120
    camA = S.look_at_camera((0.5, 0.2, -3.0), (0.0, 0.0, 0.0), W, H)
    camB = S.look_at_camera((-1.0, 0.8, -2.6), (0.1, 0.0, 0.0), W, H)
    ro, so = G.raster_opts(), G.solver_opts()
    nb = G.workspace_size(scene.n, 3, W, H, ro, so)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    img = torch.empty((3, H, W), device="cuda")
    cam_dev = torch.as_tensor(np.frombuffer(G.camera_bytes(camA), dtype=np.uint8).copy()).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        G.render_view_devcam(g, camA, cam_dev, [0.5] * 3, img, ws, ro, so)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
        G.render_view_devcam(g, camA, cam_dev, [0.5] * 3, img, ws, ro, so)
    cam_dev.copy_(torch.as_tensor(np.frombuffer(G.camera_bytes(camB), dtype=np.uint8).copy()))
    with torch.cuda.stream(s):
        graph.replay()
    s.synchronize()
    st = G.sync_status(ws)
    ref = torch.empty_like(img)
    ws2 = torch.empty_like(ws)
    G.render_view(g, camB, [0.5] * 3, ref, ws2, ro, so)
    st2 = G.sync_status(ws2)
    assert st["status"] == 0 and st["cycles"] == st2["cycles"] and st["rel_residual"] == st2["rel_residual"]
    assert torch.equal(img, ref)


@pytest.mark.gpu
def test_device_camera_near_plane_below_zero_reads_as_zero(_lib):
    """The device camera cannot be validated on the host: a negative (or NaN) near
    plane is read as 0, which gives exactly the view of a camera with near = 0."""
    import dataclasses
    import paper_2405_05446_gb300 as G
    scene = _scenes()[1]
    g = G.gaussians_to_device(scene)
    W, H = 160, 96
    cam0 = S.look_at_camera((0.4, 0.1, -2.0), (0.0, 0.0, 0.0), W, H, near=0.0)
    ro, so = G.raster_opts(), G.solver_opts()
    nb = G.workspace_size(scene.n, 3, W, H, ro, so)
    out = {}
    for name, near in (("zero", 0.0), ("negative", -1.0), ("nan", float("nan"))):
        cam = dataclasses.replace(cam0, near=near)
        cam_dev = torch.as_tensor(np.frombuffer(G.camera_bytes(cam), dtype=np.uint8).copy()).cuda()
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        img = torch.empty((3, H, W), device="cuda")
        G.render_view_devcam(g, cam0, cam_dev, [0.5] * 3, img, ws, ro, so)
        st = G.sync_status(ws)
        assert st["status"] == 0, (name, st)
        out[name] = img.cpu()
    assert torch.equal(out["negative"], out["zero"])
    assert torch.equal(out["nan"], out["zero"])


@pytest.mark.gpu
def test_served_views_identical_alone_and_in_the_mix(_lib):
    from paper_2405_05446_gb300 import serving as SV
    scenes = _scenes()
    reqs = _requests(24, seed=5)
    mix = SV.ViewServer(budget_bytes=8 << 30, slots=3)
    alone = SV.ViewServer(budget_bytes=8 << 30, slots=1)
    for i, sc in enumerate(scenes):
        mix.add_scene(i, sc, [0.5] * 3)
        alone.add_scene(i, sc, [0.5] * 3)
    mixed = mix.run(reqs, realtime=False)
    for i, r in enumerate(reqs):
        solo = alone.run([r], realtime=False)[0]
        assert mixed[i].status == 0 and solo.status == 0
        assert torch.equal(mixed[i].image, solo.image), i
    assert mix.plans_built >= 3


@pytest.mark.gpu
def test_served_view_matches_direct_render(_lib):
    import paper_2405_05446_gb300 as G
    from paper_2405_05446_gb300 import serving as SV
    scenes = _scenes()
    srv = SV.ViewServer(budget_bytes=4 << 30, slots=2)
    for i, sc in enumerate(scenes):
        srv.add_scene(i, sc, [0.5] * 3)
    reqs = _requests(6, seed=9)
    res = srv.run(reqs, realtime=False)
    for r, out in zip(reqs, res):
        sc = scenes[r.scene]
        g = G.gaussians_to_device(sc)
        ro = G.raster_opts()
        ws = torch.empty(G.workspace_size(sc.n, 3, r.cam.width, r.cam.height, ro, None), dtype=torch.uint8, device="cuda")
        ref = torch.empty((3, r.cam.height, r.cam.width), device="cuda")
        G.render_view(g, r.cam, [0.5] * 3, ref, ws, ro)
        assert G.sync_status(ws)["status"] == 0
        assert torch.equal(out.image, ref)


@pytest.mark.gpu
def test_budget_admission_evicts_and_still_serves(_lib):
    from paper_2405_05446_gb300 import serving as SV
    scenes = _scenes()
    srv = SV.ViewServer(budget_bytes=1 << 30, slots=2)
    for i, sc in enumerate(scenes):
        srv.add_scene(i, sc, [0.5] * 3)
    biggest = max(srv.plan_bytes(i, w, h) for i in range(2) for w, h in SMALL_SIZES)
    srv.budget = srv.used + 3 * biggest  # room for about three plans at once
    reqs = _requests(30, seed=11, keep=False)
    res = srv.run(reqs, realtime=False)
    assert all(r.status == 0 for r in res)
    assert srv.evictions > 0 and srv.used <= srv.budget
    tiny = SV.ViewServer(budget_bytes=srv.scenes[0].nbytes + 1024, slots=1)
    tiny.add_scene(0, scenes[0], [0.5] * 3)
    req = _requests(1, seed=1, keep=False)[0]
    req.scene = 0
    with pytest.raises(MemoryError):
        tiny.run([req], realtime=False)

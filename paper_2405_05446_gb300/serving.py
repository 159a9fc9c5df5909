"""Serving views of resident scenes: continuous batching of mixed-resolution requests.

A scene is uploaded once and stays resident. A request names a scene, a camera
(pose, intrinsics, image size) and arrives at some time. The server keeps `slots`
CUDA streams busy: whenever a slot is free and a request has arrived, the request
is dispatched at once (no waiting to fill a batch), so views of different sizes
and scenes overlap on the GPU.

One view is one CUDA graph replay. For each (scene, image size, slot) the server
keeps a *view plan*: a workspace, an output image, a device camera buffer and a
graph captured from `render_view_devcam` (the projection reads the camera from
the buffer, and the multigrid cycle loop is recorded as a conditional WHILE
node), so a dispatch is a 76-byte host-to-device copy of the camera, the replay
and an 8-byte read-back of the status word. Plans are created on demand under a
device-memory budget that also holds the resident scenes; when a new plan does
not fit, idle plans are evicted least-recently-used first, and a request whose
plan cannot be admitted waits for memory to free up.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

import paper_2405_05446_gb300 as G
from paper_2405_05446_gb300 import _abi

CAMERA_BYTES = 76  # sizeof(gdgs_camera)


@dataclass
class Request:
    scene: int
    cam: object          # scenes.Camera
    arrival: float = 0.0  # seconds after the start of run()
    keep: bool = False    # copy the image out (tests); otherwise it stays in the plan


@dataclass
class Result:
    request: int
    status: int
    latency_ms: float
    image: torch.Tensor | None = None


@dataclass
class _Plan:
    key: tuple
    ws: torch.Tensor
    image: torch.Tensor
    cam_dev: torch.Tensor
    cam_host: torch.Tensor
    status_host: torch.Tensor
    graph: torch.cuda.CUDAGraph
    nbytes: int
    busy: bool = False
    last_use: int = 0


@dataclass
class _Scene:
    g: G.DeviceGaussians
    n: int
    channels: int
    mean: list
    nbytes: int


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    request: int = -1
    plan: _Plan | None = None
    done: torch.cuda.Event | None = None
    keep_out: torch.Tensor | None = None
    arrival: float = 0.0


class ViewServer:
    def __init__(self, budget_bytes: int = 60 << 30, slots: int = 4, sopts=None,
                 pairs_per_gaussian=lambda w, h: 32 if w * h > 4_000_000 else 16, device="cuda"):
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.used = 0
        self.sopts = sopts if sopts is not None else G.solver_opts()
        self.ppg = pairs_per_gaussian
        self.scenes: dict[int, _Scene] = {}
        self.plans: collections.OrderedDict[tuple, _Plan] = collections.OrderedDict()
        self.slots = [_Slot(torch.cuda.Stream(device=self.device)) for _ in range(slots)]
        self.clock = 0
        self.evictions = 0
        self.plans_built = 0

    # -------------------------------------------------------------- scenes
    def add_scene(self, scene_id: int, scene, mean) -> None:
        nbytes = sum(np.asarray(getattr(scene, k)).nbytes
                     for k in ("mean", "scale", "quat", "opacity", "grad"))
        if self.used + nbytes > self.budget:
            raise MemoryError(f"scene {scene_id} ({nbytes} B) exceeds the memory budget")
        g = G.gaussians_to_device(scene, self.device)
        self.scenes[scene_id] = _Scene(g, scene.n, scene.channels, list(mean), nbytes)
        self.used += nbytes

    # -------------------------------------------------------------- plans
    def _ropts(self, w, h):
        return G.raster_opts(pairs_per_gaussian=self.ppg(w, h))

    def plan_bytes(self, scene_id: int, w: int, h: int) -> int:
        sc = self.scenes[scene_id]
        ws = G.workspace_size(sc.n, sc.channels, w, h, self._ropts(w, h), self.sopts)
        return ws + 4 * sc.channels * w * h + 256

    def _admit(self, need: int) -> bool:
        """Make room for `need` bytes by evicting idle plans, LRU first."""
        if self.used + need <= self.budget:
            return True
        for key in list(self.plans.keys()):
            if self.used + need <= self.budget:
                break
            p = self.plans[key]
            if p.busy:
                continue
            del self.plans[key]
            self.used -= p.nbytes
            self.evictions += 1
        return self.used + need <= self.budget

    def _build(self, key, slot: _Slot) -> _Plan | None:
        scene_id, w, h, _ = key
        sc = self.scenes[scene_id]
        need = self.plan_bytes(scene_id, w, h)
        if not self._admit(need):
            return None
        ro = self._ropts(w, h)
        ws = torch.empty(G.workspace_size(sc.n, sc.channels, w, h, ro, self.sopts),
                         dtype=torch.uint8, device=self.device)
        image = torch.empty((sc.channels, h, w), device=self.device)
        cam_dev = torch.empty(CAMERA_BYTES, dtype=torch.uint8, device=self.device)
        cam_host = torch.empty(CAMERA_BYTES, dtype=torch.uint8).pin_memory()
        status_host = torch.empty(8, dtype=torch.uint8).pin_memory()
        cam_shape = _shape_camera(w, h)
        cam_host.numpy()[:] = np.frombuffer(G.camera_bytes(cam_shape), dtype=np.uint8)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(slot.stream):
            cam_dev.copy_(cam_host, non_blocking=True)
            # one uncaptured view first: kernel attributes and the coarse factor are set up
            G.render_view_devcam(sc.g, cam_shape, cam_dev, sc.mean, image, ws, ro, self.sopts)
        slot.stream.synchronize()
        st = G.sync_status(ws, stream=slot.stream)
        if st["status"] != _abi.OK:
            raise RuntimeError(f"view plan {key}: {st['status_string']}")
        with torch.cuda.graph(graph, stream=slot.stream, capture_error_mode="thread_local"):
            G.render_view_devcam(sc.g, cam_shape, cam_dev, sc.mean, image, ws, ro, self.sopts)
        plan = _Plan(key, ws, image, cam_dev, cam_host, status_host, graph, need)
        self.plans[key] = plan
        self.used += need
        self.plans_built += 1
        return plan

    def _plan(self, req: Request, slot_index: int) -> _Plan | None:
        key = (req.scene, req.cam.width, req.cam.height, slot_index)
        p = self.plans.get(key)
        if p is None:
            p = self._build(key, self.slots[slot_index])
            if p is None:
                return None
        self.plans.move_to_end(key)
        self.clock += 1
        p.last_use = self.clock
        return p

    # -------------------------------------------------------------- serving
    def _dispatch(self, slot_index: int, req_index: int, req: Request, plan: _Plan) -> None:
        slot = self.slots[slot_index]
        plan.busy = True
        plan.cam_host.numpy()[:] = np.frombuffer(G.camera_bytes(req.cam), dtype=np.uint8)
        with torch.cuda.stream(slot.stream):
            plan.cam_dev.copy_(plan.cam_host, non_blocking=True)
            plan.graph.replay()
            plan.status_host.copy_(plan.ws[:8], non_blocking=True)
            slot.keep_out = plan.image.clone() if req.keep else None
            slot.done = torch.cuda.Event()
            slot.done.record(slot.stream)
        slot.request, slot.plan, slot.arrival = req_index, plan, req.arrival

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve `requests` (arrival times in seconds from now; realtime=False
        treats every request as already arrived). Returns one Result per request,
        in request order."""
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        pending = collections.deque(order)
        results: list[Result | None] = [None] * len(requests)
        t0 = time.perf_counter()
        waiting = 0
        while pending or any(s.request >= 0 for s in self.slots):
            now = time.perf_counter() - t0
            progressed = False
            for si, slot in enumerate(self.slots):
                if slot.request >= 0 and slot.done.query():
                    status = int(np.frombuffer(slot.plan.status_host.numpy().tobytes()[:4], dtype=np.int32)[0])
                    t_done = time.perf_counter() - t0
                    arrival = slot.arrival if realtime else 0.0
                    results[slot.request] = Result(slot.request, status, 1e3 * (t_done - arrival),
                                                   slot.keep_out)
                    slot.plan.busy = False
                    slot.request, slot.plan, slot.done, slot.keep_out = -1, None, None, None
                    progressed = True
            for si, slot in enumerate(self.slots):
                if slot.request >= 0 or not pending:
                    continue
                ri = pending[0]
                if realtime and requests[ri].arrival > now:
                    break
                plan = self._plan(requests[ri], si)
                if plan is None:  # not admitted: wait for memory to free up
                    if not any(s.request >= 0 for s in self.slots):
                        raise MemoryError(f"request {ri}: its view plan does not fit the budget "
                                          f"({self.plan_bytes(requests[ri].scene, requests[ri].cam.width, requests[ri].cam.height)} B)")
                    waiting += 1
                    break
                pending.popleft()
                self._dispatch(si, ri, requests[ri], plan)
                progressed = True
            if not progressed:
                time.sleep(0)
        self.waits = waiting
        return results

    def warm(self, requests: list[Request]) -> None:
        """Build the view plans the requests need (captures happen outside timing)."""
        for si in range(len(self.slots)):
            for req in requests:
                key = (req.scene, req.cam.width, req.cam.height, si)
                if key not in self.plans:
                    self._plan(req, si)


def _shape_camera(w: int, h: int):
    from paper_2405_05446_gb300 import scenes as S
    return S.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), w, h)


# -------------------------------------------------------------- the mixed workload

SIZES = [(256, 256), (512, 512), (1280, 720), (1920, 1080), (3840, 2160)]
SCENE_SIZES = [100_000, 400_000, 1_000_000, 2_000_000]


def mixed_requests(n: int, rate: float, seed: int = 0, n_scenes: int = 4, sizes=SIZES) -> list[Request]:
    """n requests with Poisson arrivals at `rate` per second; scene uniform over the
    resident scenes, image size uniform over `sizes`, camera uniform on the sphere
    of radius 3 looking at the origin."""
    from paper_2405_05446_gb300 import scenes as S
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(n):
        w, h = sizes[rng.integers(len(sizes))]
        reqs.append(Request(int(rng.integers(n_scenes)), S.sphere_camera(rng, w, h), float(t[i])))
    return reqs

"""Child process of test_gpu_stream.py: one seeded Poisson solve, image saved.

The library reads GDGS_STREAM (finest-level path: streaming warps or tiles) and
GDGS_STREAM_ROWS (segment height of the streaming path) once, when it first
launches a solve, so every setting under test runs in a process of its own.

usage: python _stream_child.py H W C storage max_cycles out.npy
"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_2405_05446_gb300 as G  # noqa: E402

STORAGES = {"f32": 0, "bf16": 1, "f16": 2}


def main():
    H, W, C = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3])
    storage, max_cycles, out = sys.argv[4], int(sys.argv[5]), sys.argv[6]
    rng = np.random.default_rng(H * 7919 + W * 31 + C)
    maps = torch.from_numpy(rng.laplace(0, 0.1, (C, 2, H, W)).astype(np.float32)).cuda()
    mean = [0.5, 0.1, -0.2, 0.3][:C]
    so = G.solver_opts(storage=STORAGES[storage], max_cycles=max_cycles, rtol=1e-9)
    ws = torch.empty(G.workspace_size(0, C, W, H, None, so), dtype=torch.uint8, device="cuda")
    img = torch.empty((C, H, W), device="cuda")
    G.poisson_reconstruct(maps, mean, img, ws, sopts=so)
    st = G.sync_status(ws)
    np.save(out, img.cpu().numpy())
    print(st["status"], st["cycles"], st["rel_residual"])


if __name__ == "__main__":
    main()

"""Host-side logic of bench.py: its model of the solver's levels must follow the
library, its byte counts follow their stated formulas, and a profiled DRAM-traffic
figure is only used while the kernel's source file is the one that was profiled."""
import hashlib
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tail_threshold_matches_the_library():
    src = open(os.path.join(ROOT, "paper_2405_05446_gb300", "csrc", "poisson.cu")).read()
    m = re.search(r"constexpr long long kTailCells = (\d+);", src)
    assert m, "kTailCells not found"
    assert int(m.group(1)) == bench.TAIL_CELLS


def test_levels_of_the_1080p_view():
    lv, t = bench.mg_levels(1080, 1920)
    assert lv == [(1080, 1920), (540, 960), (270, 480), (135, 240), (68, 120), (34, 60),
                  (17, 30), (9, 15), (5, 8)]
    assert t == 5  # 60x34 is the first level with at most TAIL_CELLS cells


def test_algorithmic_bytes_formulas():
    C, H, W = 3, 64, 48
    px = C * H * W
    assert bench.algorithmic_bytes("divergence", C, H, W, 5, 0, 0) == px * 12
    assert bench.algorithmic_bytes("finalize", C, H, W, 5, 0, 0) == px * 16
    # the survey's per-unknown model: 12 B per sweep, 9 B residual + restriction, 9 B
    # prolongation + correction; V(2,1) by default
    assert bench.algorithmic_bytes("mg0_down", C, H, W, 5, 0, 0) == 5 * px * (2 * 12 + 9)
    assert bench.algorithmic_bytes("mg0_up", C, H, W, 5, 0, 0) == 5 * px * (12 + 9)
    assert bench.algorithmic_bytes("mg0_up", C, H, W, 5, 0, 0, nu1=3, nu2=2) == 5 * px * (24 + 9)
    lv, _ = bench.mg_levels(H, W)
    assert bench.algorithmic_bytes("mg1_down", C, H, W, 5, 0, 0) == 5 * C * lv[1][0] * lv[1][1] * 33
    assert bench.algorithmic_bytes("mg2_up", C, H, W, 5, 0, 0) == 5 * C * lv[2][0] * lv[2][1] * 21
    # what the fused kernels must move at least
    assert bench.min_traffic_bytes("mg0_down", C, H, W, 5, 0, 0) == 5 * px * 9
    assert bench.min_traffic_bytes("mg0_up", C, H, W, 5, 0, 0) == 5 * px * 21 + 4 * px * 8
    assert bench.algorithmic_bytes("raster", C, H, W, 5, 0, 1000) == 1000 * (36 + 8 * C) + px * 8
    assert bench.algorithmic_bytes("no_such_kernel", C, H, W, 5, 0, 0) == 0.0


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "kernel.cu"
    src.write_text("// one version of a kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "k.md").write_text(
        "# a summary\n\nbench-traffic: kernel=mg0_up bytes_per_launch=1234 cycle=1 "
        f"source=kernel.cu source_sha256={sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.profiled_traffic("mg0_up")
    assert got is not None and got["bytes_per_launch"] == 1234.0
    assert bench.profiled_traffic("raster") is None
    src.write_text("// another version\n")
    assert bench.profiled_traffic("mg0_up") is None


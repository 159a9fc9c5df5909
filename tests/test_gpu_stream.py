"""The streaming finest-level passes (one warp per 64-column strip and segment of rows).

Every cell's formula depends on its position alone, so the iterate must not depend on
how the grid is cut into segments (GDGS_STREAM_ROWS), on grids with border strips, odd
heights, a last segment shorter than the others and 16-bit storage alike: the final
residual, recomputed from the float-float iterate, must be the same, and the images may
differ only through the FP32 sums of the iterate (their roundings follow the segments),
which set the constant shift: by a few units in the last place. A halo row or column
computed differently by two segments or strips changes the residual in its leading
digits. Against the tiled passes (GDGS_STREAM=0) the image must agree to the solver's
tolerance. Each setting is read once per process, so every run
is a child process (_stream_child.py). Parity with the oracle at many shapes is in
test_gpu_parity.py, which runs the streaming path (the default for even widths).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import ensure_lib

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _solve(tmp_path, tag, env_extra, H, W, C, storage="f32", max_cycles=3):
    out = str(tmp_path / ("img_%s.npy" % tag))
    env = dict(os.environ)
    env.pop("GDGS_STREAM", None)
    env.pop("GDGS_STREAM_ROWS", None)
    env.update(env_extra)
    r = subprocess.run([sys.executable, os.path.join(HERE, "_stream_child.py"), str(H), str(W),
                        str(C), storage, str(max_cycles), out],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    status, cycles, rel = r.stdout.split()[-3:]
    return np.load(out), int(status), int(cycles), float(rel)


def _same_iterate(a, b):
    img_a, _, cyc_a, rel_a = a
    img_b, _, cyc_b, rel_b = b
    assert cyc_a == cyc_b
    assert abs(rel_a - rel_b) <= 1e-9 * rel_a, (rel_a, rel_b)
    ulp = np.spacing(np.float32(np.abs(img_a).max()))
    assert np.abs(img_a - img_b).max() <= 4 * ulp


# (99, 203): odd finest width (tiles there); level 1 has 102 columns, the last one
# narrow, and streams its up pass with the general face coefficients.
@pytest.mark.parametrize("shape", [(1080, 1920, 1), (97, 114, 2), (50, 66, 1), (25, 2, 1), (99, 203, 1)])
def test_iterate_does_not_depend_on_segment_height(tmp_path, shape):
    H, W, C = shape
    ref = _solve(tmp_path, "16", {"GDGS_STREAM_ROWS": "16"}, H, W, C)
    assert 1 <= ref[2] <= 3 and np.isfinite(ref[0]).all()
    for rows in ("24", "40"):
        _same_iterate(ref, _solve(tmp_path, rows, {"GDGS_STREAM_ROWS": rows}, H, W, C))


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_16bit_storage_does_not_depend_on_segment_height(tmp_path, storage):
    a = _solve(tmp_path, "a", {"GDGS_STREAM_ROWS": "16"}, 135, 240, 3, storage)
    b = _solve(tmp_path, "b", {"GDGS_STREAM_ROWS": "32"}, 135, 240, 3, storage)
    _same_iterate(a, b)


@pytest.mark.parametrize("shape", [(270, 480, 3), (97, 114, 1)])
def test_streaming_and_tiled_passes_agree(tmp_path, shape):
    H, W, C = shape
    s, st_s, cyc_s, rel_s = _solve(tmp_path, "s", {"GDGS_STREAM": "1"}, H, W, C, max_cycles=12)
    t, st_t, cyc_t, rel_t = _solve(tmp_path, "t", {"GDGS_STREAM": "0"}, H, W, C, max_cycles=12)
    assert rel_s <= 1e-6 and rel_t <= 1e-6
    scale = max(1.0, float(t.max() - t.min()))
    assert np.abs(s - t).max() <= 1e-5 * scale

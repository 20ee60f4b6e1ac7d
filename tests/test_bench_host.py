"""Host logic of bench.py's oracle baseline (no GPU): the bounded sample of one step.

The sample is sized from a tiny calibration run; when that run overstates the per-item cost (a
fixed cost per call, as thread start-up gives the real oracle), the first sample takes far less
than the budget, and the sampler sizes it again from the first sample's own rate.  The fake oracle
below charges a fixed 20 ms per call plus a per-item time, so the calibration overstates the cost
about 25-fold.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CALL_S, PIXEL_S, PRIM_S = 0.02, 2e-6, 1e-4


class FakeOracle:
    def __init__(self):
        self.calls = []

    def build(self):
        pass

    def render2d(self, p, H, W, pixels=None):
        pix = np.asarray(pixels)
        self.calls.append(("render", len(pix)))
        time.sleep(CALL_S + PIXEL_S * len(pix))
        return np.zeros((len(pix), 3))

    def grad2d(self, p, H, W, g):
        self.calls.append(("grad", len(p)))
        time.sleep(CALL_S + PRIM_S * len(p))
        return np.zeros_like(p, dtype=np.float64)


def test_sample_is_resized_from_its_own_rate(monkeypatch):
    fake = FakeOracle()
    monkeypatch.setitem(sys.modules, "oracle", fake)
    H, W, n, budget = 64, 64, 4000, 1.0
    p = np.zeros((n, 16), np.float32)
    target = np.zeros((H, W, 3), np.float32)
    t0 = time.perf_counter()
    per_step, desc = bench.oracle_step_sample(p, target, H, W, budget)
    wall = time.perf_counter() - t0
    # calibration (1 row, n / 2000 primitives), the first sample, then the resized one
    renders = [k for kind, k in fake.calls if kind == "render"]
    grads = [k for kind, k in fake.calls if kind == "grad"]
    assert len(renders) == 3 and len(grads) == 3
    assert renders[2] > renders[1] and grads[2] > grads[1]
    # the true cost of a full step, and the estimate from the final sample
    true_step = 2 * CALL_S + PIXEL_S * H * W + PRIM_S * n
    rows, prims = renders[2] // W, grads[2]
    est = (CALL_S + PIXEL_S * rows * W) * (H / rows) + (CALL_S + PRIM_S * prims) * (n / prims)
    assert abs(per_step - est) <= 0.5 * est  # the sleeps only overrun
    assert per_step >= 0.9 * true_step
    assert wall <= 3 * budget
    assert f"of {H} rows" in desc and f"of {n} primitives" in desc


class FakeOracle3D:
    """A 3D oracle whose calls cost a fixed set-up plus a time per pixel of the band."""

    SETUP_S, PX_S = 0.05, 2e-4

    def __init__(self):
        self.calls = []

    def build(self):
        pass

    def deform6d(self, p, t):
        return np.asarray(p, np.float64)[:, :20]

    def render3d(self, p, cam, H, W, pixels=None):
        self.calls.append(("render", len(pixels)))
        time.sleep(self.SETUP_S + self.PX_S * len(pixels))

    def grad3d(self, p, cam, H, W, g):
        n = int(np.count_nonzero(np.any(g != 0, axis=2)))
        self.calls.append(("grad", n))
        time.sleep(self.SETUP_S + self.PX_S * n)


def test_3d_sample_separates_the_fixed_cost_from_the_rows(monkeypatch):
    """The 3D baseline times bands of rows of one frame: the cost per call that does not depend on
    the band is counted once per pass, the rest scaled to every row and every sample of a step."""
    import types

    fake = FakeOracle3D()
    monkeypatch.setitem(sys.modules, "oracle", fake)
    H, W, batch, budget = 64, 40, 4, 1.5
    wl = types.SimpleNamespace(p=np.zeros((10, 32), np.float32), cams=[np.zeros(17, np.float32)],
                               samples=[(0, 0.25)], H=H, W=W, batch=batch)
    t0 = time.perf_counter()
    per_step, desc = bench.oracle_3d_sample(wl, budget)
    wall = time.perf_counter() - t0
    true_step = batch * (2 * fake.SETUP_S + 2 * fake.PX_S * H * W)
    assert 0.8 * true_step <= per_step <= 1.5 * true_step, (per_step, true_step)
    # three band heights, each pass on every pixel of the band
    grads = [k for kind, k in fake.calls if kind == "grad"]
    assert [k // W for k in grads][:2] == [1, 4] and grads[2] > grads[1]
    assert wall <= 3 * budget
    assert f"of {H} rows" in desc and "4 full frames per step" in desc

"""The oracle against the hand-derived values stored under tests/golden/ (no GPU needed).

Each fixture file states the equations its values follow from and how they were derived; the values
are closed forms written out by hand, not outputs of the oracle or of the device path.
"""
from pathlib import Path

import numpy as np

import oracle

GOLDEN = Path(__file__).parent / "golden"


def _rows(name):
    for line in (GOLDEN / name).read_text().splitlines():
        body = line.split("#", 1)[0].split()
        if body:
            yield body


def test_wavelet2d_points():
    n = 0
    for row in _rows("eq5_wavelet2d_points.txt"):
        rec = np.zeros((1, 16), np.float32)
        rec[0, :11] = [float(x) for x in row[1:12]]
        u, v, W = int(row[12]), int(row[13]), float(row[14])
        out = oracle.render2d(rec, 17, 17, truncated=False, pixels=[[u, v]])
        expect = W * rec[0, 8:11].astype(np.float64)
        np.testing.assert_allclose(out[0], expect, rtol=0, atol=1e-12, err_msg=f"case {row[0]} at ({u}, {v})")
        n += 1
    assert n == 15


def test_front_to_back_stack():
    layers, expect, bg = [], None, None
    for line in (GOLDEN / "eq3_front_to_back_stack.txt").read_text().splitlines():
        if line.startswith("# bg"):
            bg = [float(x) for x in line.split()[2:5]]
    for row in _rows("eq3_front_to_back_stack.txt"):
        if row[0] == "layer":
            z, o, r, g, b = (float(x) for x in row[1:6])
            p = np.zeros(20, np.float32)
            p[:18] = [0, 0, z, 0.1, 0.1, 0.1, 1, 0, 0, 0, 0, 0, 0, 0.0, o, r, g, b]
            layers.append(p)
        elif row[0] == "expect":
            expect = [float(x) for x in row[1:5]]
    assert len(layers) == 3 and expect is not None and bg is not None
    H = W = 17
    cam = np.zeros(17, np.float32)
    cam[:12] = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32).ravel()
    cam[12:17] = [100.0, 100.0, 8.5, 8.5, 0.2]
    opts = np.array([3.0, 0.0, 1.0, 0.0, 0.3, *bg], np.float32)
    C, T, nc, amb = oracle.render3d(np.stack(layers), cam, H, W, opts, pixels=[[8, 8]])
    np.testing.assert_allclose(C[0], expect[:3], rtol=0, atol=1e-14)
    assert abs(T[0] - expect[3]) <= 1e-14
    assert nc[0] == 3

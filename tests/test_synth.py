"""The seeded input generators follow the stated recipe (no GPU): shapes, value ranges, camera
geometry and determinism of the workloads that stand in for the paper's datasets."""
import math

import numpy as np

import synth


def test_seeded_generators_are_deterministic():
    a = synth.scene2d(500, 64, 96, 7)
    assert np.array_equal(a, synth.scene2d(500, 64, 96, 7))
    assert not np.array_equal(a, synth.scene2d(500, 64, 96, 8))
    b = synth.scene3d(500, 7)
    assert np.array_equal(b, synth.scene3d(500, 7))
    assert np.array_equal(synth.sphere_cameras(3, 64, 64, 5), synth.sphere_cameras(3, 64, 64, 5))


def test_image_fitting_workload():
    """768x512, 70,000 primitives: scales log-uniform 0.5-32 px, theta in [0, pi), |f| <= 0.5
    cycles/px, phase in [0, 2 pi), colours in [0, 1]; the target is an image in [0, 1]."""
    p, target = synth.cfg1_inputs()
    c = synth.CFG1_2D_KODAK
    assert p.shape == (70000, synth.P2D) and p.dtype == np.float32
    assert target.shape == (512, 768, 3) and c.H == 512 and c.W == 768
    assert (p[:, 0] >= 0).all() and (p[:, 0] <= 768).all() and (p[:, 1] >= 0).all() and (p[:, 1] <= 512).all()
    s = p[:, 2:4]
    assert s.min() >= 0.5 * (1 - 1e-6) and s.max() <= 32 * (1 + 1e-6)
    # log-uniform: the median scale sits near the geometric mean 4 px
    assert abs(np.median(np.log(s)) - math.log(4.0)) < 0.05
    assert (p[:, 4] >= 0).all() and (p[:, 4] < math.pi + 1e-6).all()
    assert np.hypot(p[:, 5], p[:, 6]).max() <= 0.5 + 1e-6
    assert (p[:, 7] >= 0).all() and (p[:, 7] <= 2 * math.pi + 1e-6).all()
    assert (p[:, 8:11] >= 0).all() and (p[:, 8:11] <= 1).all() and (p[:, 11:] == 0).all()
    assert target.min() >= 0 and target.max() <= 1 and target.std() > 0.01


def test_static_scene_workload_and_cameras():
    """800x800, 300,000 primitives in the unit cube; 16 cameras on the radius-4 sphere looking at
    the origin with a 50 degree field of view."""
    p, cams = synth.cfg2_inputs()
    assert p.shape == (300000, synth.P3D) and cams.shape == (16, synth.CAM_FLOATS)
    assert np.abs(p[:, 0:3]).max() <= 0.5
    assert p[:, 3:6].min() >= 0.002 * (1 - 1e-6) and p[:, 3:6].max() <= 0.05 * (1 + 1e-6)
    assert np.allclose(np.linalg.norm(p[:, 6:10], axis=1), 1.0, atol=1e-6)
    assert np.linalg.norm(p[:, 10:13], axis=1).max() <= 40 * (1 + 1e-6)
    assert (p[:, 14] > 0).all() and (p[:, 14] < 1).all()
    fx = 400.0 / math.tan(math.radians(25.0))
    for cam in cams:
        V = cam[:12].reshape(3, 4).astype(np.float64)
        R, t = V[:, :3], V[:, 3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
        eye = -R.T @ t
        assert abs(np.linalg.norm(eye) - 4.0) < 1e-5
        # the origin lies on the optical axis, in front of the camera
        o = R @ np.zeros(3) + t
        assert abs(o[0]) < 1e-5 and abs(o[1]) < 1e-5 and abs(o[2] - 4.0) < 1e-5
        assert cam[12] == np.float32(fx) and cam[13] == np.float32(fx)
        assert cam[14] == 400 and cam[15] == 400 and cam[16] == np.float32(0.2)


def test_dynamic_scene_and_variants():
    p, cams, ts = synth.cfg3_inputs(n_cams=2)
    assert p.shape == (200000, synth.P6D) and ts.shape == (300,) and ts[0] == 0 and ts[-1] == 1
    rates = p[:, 20:30]
    assert abs(rates.std() - 0.05) < 0.002 and (p[:, 30:] == 0).all()
    assert np.array_equal(p[:, :20], synth.scene3d(200000, synth.CFG3_6D.seed))
    # Cholesky record: |l1|, |l3| in the scale range, |l2| at most the range's top
    q = synth.scene2d_cholesky(5000, 64, 64, 3, (0.5, 32.0))
    assert np.abs(q[:, [2, 4]]).min() >= 0.5 * (1 - 1e-6) and np.abs(q[:, [2, 4]]).max() <= 32 * (1 + 1e-6)
    assert np.abs(q[:, 3]).max() <= 32 * (1 + 1e-6) and (q[:, 2] < 0).any() and (q[:, 4] < 0).any()
    # SH record: the degree-0 coefficients reproduce the base colour (0.5 + Y00 c00 = c)
    base = synth.scene3d(1000, 11)
    sh = synth.scene3d_sh(1000, 11, degree=3)
    y00 = 0.5 / math.sqrt(math.pi)
    assert np.allclose(0.5 + y00 * sh[:, 15:18].astype(np.float64), base[:, 15:18], atol=1e-6)
    assert np.count_nonzero(sh[:, 20:65]) == 1000 * 45 and (sh[:, 65:] == 0).all()
    # the network's packed parameters: 505,101 values, the head scaled down
    theta = synth.deform_mlp_theta(5)
    assert theta.size == sum(o * i + o for o, i in synth.MLP_SHAPES) == 505101
    assert np.abs(theta[:256 * 80]).max() <= 1 / math.sqrt(80)


def test_serving_trace():
    """Poisson arrivals at the stated rate; scenes alternate 2D and 3D; sizes from the stated set."""
    scenes, req = synth.serving_workload(n_scenes=4, rate=2000.0, seconds=1.0, n_range=(1000, 2000))
    assert [s.dims for s in scenes] == [2, 3, 2, 3]
    assert all(1000 <= s.n <= 2000 for s in scenes)
    assert abs(len(req) - 2000) < 4 * math.sqrt(2000)
    assert (np.diff(req[:, 0]) > 0).all() and req[-1, 0] < 1.0
    assert set(np.unique(req[:, 2]).astype(int)) <= {0, 1, 2, 3}
    assert scenes[0].params[3].shape == (scenes[0].n, synth.P2D) and scenes[1].cameras[2].shape == (16, 17)

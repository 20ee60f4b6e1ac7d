"""Pins of the binary64 oracle against facts the paper and the mathematics fix (no GPU needed).

Each test names the passage it rests on.  Together they are chosen so that a plausible slip in the
oracle (a dropped factor 1/2 or 2 pi, a sign of the phase or offset, Sigma in place of its inverse,
a transposed rotation, a wrong Jacobian column, front-to-back order reversed) fails one of them.
"""
import math

import numpy as np
import pytest
import scipy.stats

import oracle
import synth


def rec2d(mu, s, theta, f, phi, c):
    p = np.zeros((1, 16), np.float32)
    p[0, :11] = [mu[0], mu[1], s[0], s[1], theta, f[0], f[1], phi, c[0], c[1], c[2]]
    return p


def rec3d(mu, s, q, f, phi, o, c):
    p = np.zeros((1, 20), np.float32)
    p[0, :18] = [*mu, *s, *q, *f, phi, o, *c]
    return p


def cam_identity(H, W, fx=300.0, fy=None, near=0.2):
    cam = np.zeros(17, np.float32)
    cam[:12] = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32).ravel()
    cam[12] = fx
    cam[13] = fx if fy is None else fy
    cam[14] = W / 2
    cam[15] = H / 2
    cam[16] = near
    return cam


OPTS_EXACT = np.array([3.0, 0.0, 1.0, 0.0, 0.3, 0.0, 0.0, 0.0], np.float32)


# ---------------------------------------------------------------------------------------------
# 2D wavelet field (Sec. 4.1 Eq. 5, Sec. 4.3 with the summed field of Eq. 4)
# ---------------------------------------------------------------------------------------------

def test_zero_frequency_reduces_to_gaussian_splat():
    """Sec. 4.1: with f = 0 the wavelet is the Gaussian primitive.  The expected image is a sum of
    scipy multivariate-normal densities scaled by 2 pi sqrt(det Sigma), Sigma = R S S^T R^T."""
    H, W = 40, 56
    p = synth.scene2d(12, H, W, 3, (1.5, 6.0))
    p[:, 5:8] = 0.0
    img = oracle.render2d(p, H, W, truncated=False)
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    pts = np.stack([xx.ravel(), yy.ravel()], 1)
    ref = np.zeros((H, W, 3))
    for i in range(len(p)):
        c, s = math.cos(p[i, 4]), math.sin(p[i, 4])
        R = np.array([[c, -s], [s, c]])
        S = np.diag(p[i, 2:4].astype(np.float64))
        Sig = R @ S @ S.T @ R.T
        dens = scipy.stats.multivariate_normal(mean=p[i, :2].astype(np.float64), cov=Sig).pdf(pts)
        G = dens * 2 * math.pi * math.sqrt(np.linalg.det(Sig))
        ref += G.reshape(H, W)[..., None] * p[i, 8:11].astype(np.float64)
    np.testing.assert_allclose(img, ref, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("phi", [0.0, 1.0, math.pi / 2, 2.5, math.pi, 4.0])
@pytest.mark.parametrize("truncated", [False, True])
def test_single_primitive_value_at_centre(phi, truncated):
    """Eq. 5 at x = mu: G = 1 and the modulation is (1 + cos phi) / 2."""
    p = rec2d((10.5, 7.5), (3.0, 1.7), 0.4, (0.13, -0.21), phi, (0.2, 0.5, 0.9))
    out = oracle.render2d(p, 16, 24, truncated=truncated, pixels=[[10, 7]])
    expected = p[0, 8:11].astype(np.float64) * 0.5 * (1 + math.cos(float(p[0, 7])))
    np.testing.assert_allclose(out[0], expected, rtol=0, atol=1e-15)


def test_phase_sign_and_offset_direction():
    """Eq. 5 with d = x - mu and the phase added to 2 pi f.d: with f = (1/4, 0) cycles/px and
    phi = pi/2 the cosine is -1 one pixel to the right of the centre and +1 one pixel to the left;
    one pixel below it is cos(pi/2) = 0."""
    s = 2.0
    p = rec2d((8.5, 8.5), (s, s), 0.0, (0.25, 0.0), math.pi / 2, (1, 1, 1))
    out = oracle.render2d(p, 17, 17, truncated=False, pixels=[[9, 8], [7, 8], [8, 9]])
    G1 = math.exp(-0.5 / s ** 2)
    np.testing.assert_allclose(out[:, 0], [0.0, G1, 0.5 * G1], atol=1e-7)


@pytest.mark.parametrize("trial", range(6))
def test_pixel_sum_matches_fourier_closed_form(trial):
    """Sec. 4.2: the modulation shifts the Gaussian spectrum to +-f.  Summing W over the pixel grid
    (midpoint rule, spectrally exact for sigma >= 3 px) gives the integral
    pi sqrt(det Sigma) (1 + cos(phi) exp(-2 pi^2 f^T Sigma f))."""
    rng = np.random.default_rng(100 + trial)
    H = W = 160
    s = rng.uniform(3.0, 7.0, 2)
    th = rng.uniform(0, math.pi)
    fm, fd = rng.uniform(0, 0.45), rng.uniform(0, 2 * math.pi)
    phi = rng.uniform(0, 2 * math.pi)
    p = rec2d((80.0 + rng.uniform(-1, 1), 80.0 + rng.uniform(-1, 1)), s, th, (fm * math.cos(fd), fm * math.sin(fd)),
              phi, (1, 0, 0))
    img = oracle.render2d(p, H, W, truncated=False)
    q = p[0].astype(np.float64)
    c, sn = math.cos(q[4]), math.sin(q[4])
    R = np.array([[c, -sn], [sn, c]])
    Sig = R @ np.diag(q[2:4] ** 2) @ R.T
    f = q[5:7]
    closed = math.pi * math.sqrt(np.linalg.det(Sig)) * (1 + math.cos(q[7]) * math.exp(-2 * math.pi ** 2 * f @ Sig @ f))
    assert abs(img[..., 0].sum() - closed) <= 1e-9 * closed


def test_translation_by_whole_pixels_shifts_the_image():
    """Eq. 5 depends on x - mu only: moving every centre by (3, 2) pixels moves the image."""
    H, W = 48, 64
    p = synth.scene2d(20, H, W, 21, (1.0, 3.0))
    p[:, 0] = np.clip(p[:, 0], 14, W - 20).astype(np.float32)
    p[:, 1] = np.clip(p[:, 1], 14, H - 20).astype(np.float32)
    p[:, :2] = np.round(p[:, :2] * 4096.0) / 4096.0  # so that the shifted centres stay exact in float32
    a = oracle.render2d(p, H, W, truncated=False)
    q = p.copy()
    q[:, 0] += 3.0
    q[:, 1] += 2.0
    b = oracle.render2d(q, H, W, truncated=False)
    np.testing.assert_allclose(b[2:, 3:], a[:-2, :-3], rtol=1e-9, atol=1e-12)


def test_truncation_bound():
    """Dropping the terms outside the 3-sigma ellipse changes a pixel by at most
    sum_i |c_i| (1/2)(1 + 1) e^{-9/2} over the primitives cut at that pixel."""
    H, W = 64, 64
    p = synth.scene2d(60, H, W, 5, (1.0, 8.0))
    full = oracle.render2d(p, H, W, truncated=False)
    cut = oracle.render2d(p, H, W, truncated=True)
    bound = np.abs(p[:, 8:11]).sum(0) * math.exp(-4.5)
    assert np.all(np.abs(full - cut) <= bound + 1e-12)
    assert np.abs(full - cut).max() > 0


def _central_fd(render, p, rows, cols, rel=2.0 ** -16, floor=None):
    """Central differences of L(p) with float32-representable steps."""
    out = np.zeros((len(rows), len(cols)))
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            base = float(p[i, j])
            scale = max(abs(base), floor[j] if floor is not None else 1.0)
            h = 2.0 ** math.floor(math.log2(scale)) * rel
            pp, pm = p.copy(), p.copy()
            pp[i, j] = np.float32(base + h)
            pm[i, j] = np.float32(base - h)
            step = float(pp[i, j]) - float(pm[i, j])
            out[a, b] = (render(pp) - render(pm)) / step
    return out


def test_grad2d_matches_central_differences():
    """The analytic gradient (Sec. 1 states explicit gradients) equals central differences of
    the binary64 forward, every parameter of every primitive, no truncation."""
    H, W = 24, 28
    p = synth.scene2d(5, H, W, 11, (1.5, 5.0))
    g = synth.upstream_grad(H, W, 12)
    an = oracle.grad2d(p, H, W, g, truncated=False)
    cols = list(range(11))
    fd = _central_fd(lambda pp: float((oracle.render2d(pp, H, W, truncated=False) * g).sum()), p, range(len(p)), cols)
    ref = an[:, cols]
    err = np.abs(ref - fd)
    tol = 2e-6 * np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max(axis=0, keepdims=True))
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-300)).max()


# ---------------------------------------------------------------------------------------------
# 2D Cholesky covariance (GaussianImage's second construction, Sec. 5.1): Sigma = L L^T
# ---------------------------------------------------------------------------------------------

def _rs_to_cholesky(p):
    """The same primitives in the Cholesky record: L = chol(R diag(s^2) R^T), in binary64."""
    q = p.astype(np.float64).copy()
    for i in range(len(p)):
        c, s = math.cos(p[i, 4]), math.sin(p[i, 4])
        R = np.array([[c, -s], [s, c]])
        L = np.linalg.cholesky(R @ np.diag(p[i, 2:4].astype(np.float64) ** 2) @ R.T)
        q[i, 2], q[i, 3], q[i, 4] = L[0, 0], L[1, 0], L[1, 1]
    return q


def test_cholesky_and_rs_constructions_render_the_same_field():
    """A Cholesky record built from an RS record by numpy's Cholesky factorisation describes the
    same Sigma, so the untruncated fields agree up to the rounding of the records to binary32."""
    H, W = 40, 48
    p = synth.scene2d(40, H, W, 21, (1.0, 8.0))
    q = _rs_to_cholesky(p)
    a = oracle.render2d(p, H, W, truncated=False)
    b = oracle.render2d(q, H, W, truncated=False, cov2d=1)
    assert np.abs(a - b).max() <= 2e-5 * max(1.0, np.abs(a).max())
    ga = oracle.grad2d(p, H, W, synth.upstream_grad(H, W, 22), truncated=False)
    gb = oracle.grad2d(q, H, W, synth.upstream_grad(H, W, 22), truncated=False, cov2d=1)
    for cols in ([0, 1], [5, 6, 7], [8, 9, 10]):  # parameters the two records share
        np.testing.assert_allclose(gb[:, cols], ga[:, cols], rtol=1e-4, atol=1e-4 * np.abs(ga[:, cols]).max())


def test_cholesky_sign_flips_leave_sigma_and_the_image_unchanged():
    """(l1, l2, l3) -> (-l1, -l2, -l3) and l3 -> -l3 leave L L^T unchanged: identical images, also
    truncated (the binary32 footprint rule sees the same squares and products), and the gradient
    with respect to the flipped entries changes sign."""
    H, W = 36, 44
    p = synth.scene2d_cholesky(60, H, W, 23, (1.0, 8.0))
    g = synth.upstream_grad(H, W, 24)
    base = oracle.render2d(p, H, W, cov2d=1)
    gb = oracle.grad2d(p, H, W, g, cov2d=1)
    for flip in ([2, 3, 4], [4]):
        q = p.copy()
        q[:, flip] = -q[:, flip]
        assert np.array_equal(oracle.render2d(q, H, W, cov2d=1), base)
        assert np.array_equal(oracle.tile_lists(2, q, H, W, cov2d=1)[0], oracle.tile_lists(2, p, H, W, cov2d=1)[0])
        gq = oracle.grad2d(q, H, W, g, cov2d=1)
        np.testing.assert_allclose(gq[:, flip], -gb[:, flip], rtol=1e-9, atol=1e-12)


def test_cholesky_grad_matches_central_differences():
    """The Cholesky chain rule (dK = -K dSigma K) equals central differences of the binary64
    forward, every parameter of every primitive, no truncation."""
    H, W = 24, 28
    p = synth.scene2d_cholesky(5, H, W, 25, (1.5, 5.0))
    g = synth.upstream_grad(H, W, 26)
    an = oracle.grad2d(p, H, W, g, truncated=False, cov2d=1)
    cols = list(range(11))
    fd = _central_fd(lambda pp: float((oracle.render2d(pp, H, W, truncated=False, cov2d=1) * g).sum()), p,
                     range(len(p)), cols)
    err = np.abs(an[:, cols] - fd)
    tol = 2e-6 * np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max(axis=0, keepdims=True))
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-300)).max()


def test_cholesky_footprint_covers_the_cutoff_ellipse():
    """The Cholesky footprint rule's extents and tile test lose no pixel of the binary32 cutoff
    test, down to elongated primitives, and its L reproduces the binary64 Sigma^-1."""
    H, W = 112, 128
    p = synth.scene2d_cholesky(1200, H, W, 27, (0.5, 32.0))
    inside, outside, rect, dropped = oracle.cutoff_coverage(2, p, H, W, cov2d=1)
    assert inside > 0 and outside == 0 and dropped == 0 and rect >= inside
    rec, _, valid = oracle.footprints(2, p[:200], H, W, cov2d=1)
    for i in np.nonzero(valid)[0]:
        L0 = np.array([[p[i, 2], 0.0], [p[i, 3], p[i, 4]]], np.float64)
        K = np.linalg.inv(L0 @ L0.T)
        L = np.array([[rec[i, 2], 0.0], [rec[i, 3], rec[i, 4]]], np.float64)
        np.testing.assert_allclose(L @ L.T, K, rtol=2e-5, atol=2e-5 * np.abs(K).max())


# ---------------------------------------------------------------------------------------------
# 3D projection (Sec. 3.1 EWA, Sec. 4.1 frequency), blending (Eq. 3 with W')
# ---------------------------------------------------------------------------------------------

def test_on_axis_projection_closed_form():
    """Sec. 3.1: on the optical axis with R = I, Sigma' = diag(fx^2 sx^2, fy^2 sy^2) / tz^2 + 0.3 I
    and mu' is the principal point."""
    H, W = 64, 80
    cam = cam_identity(H, W, fx=300.0, fy=250.0)
    p = rec3d((0, 0, 5.0), (0.1, 0.2, 0.3), (1, 0, 0, 0), (0, 0, 0), 0.0, 0.5, (1, 1, 1))
    r = oracle.project3d(p, cam, H, W)[0]
    assert r[0] == 1 and r[1] == pytest.approx(5.0)
    np.testing.assert_allclose(r[2:4], [W / 2, H / 2], atol=1e-12)
    np.testing.assert_allclose(r[4:7], [300.0 ** 2 * 0.01 / 25 + 0.3, 0.0, 250.0 ** 2 * 0.04 / 25 + 0.3],
                               rtol=1e-6, atol=1e-12)


def test_off_axis_isotropic_projection_closed_form():
    """Sec. 3.1 with the perspective Jacobian J = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]]:
    an isotropic 3D Gaussian of std sigma projects to sigma^2 J J^T + 0.3 I."""
    H, W = 200, 240
    cam = cam_identity(H, W, fx=300.0, fy=280.0)
    tx, ty, tz, sig = 0.7, -0.4, 4.0, 0.05
    p = rec3d((tx, ty, tz), (sig, sig, sig), (0.3, -0.2, 0.8, 0.1), (0, 0, 0), 0.0, 0.5, (1, 1, 1))
    r = oracle.project3d(p, cam, H, W)[0]
    fx, fy = 300.0, 280.0
    # the float32 record rounds tx, ty, tz, sigma
    tx, ty, tz, sig = (float(np.float32(v)) for v in (tx, ty, tz, sig))
    s2 = sig * sig / tz ** 2
    expect = [s2 * fx * fx * (1 + tx * tx / tz ** 2) + 0.3, s2 * fx * fy * tx * ty / tz ** 2,
              s2 * fy * fy * (1 + ty * ty / tz ** 2) + 0.3]
    np.testing.assert_allclose(r[4:7], expect, rtol=1e-6)
    np.testing.assert_allclose(r[2:4], [fx * tx / tz + W / 2, fy * ty / tz + H / 2], rtol=1e-6)


def test_look_at_camera_projects_centre():
    """Pinhole projection with the OpenCV look-at camera: a camera at (0, -5, 0) looking at the
    origin with up +z sees world (x, 0, z) at pixel (fx x / 5 + cx, -fy z / 5 + cy)."""
    H, W = 100, 120
    cam = synth.camera(synth.look_at((0.0, -5.0, 0.0)), H, W, 50.0)
    p = np.concatenate([rec3d((0.3, 0.0, -0.2), (0.01,) * 3, (1, 0, 0, 0), (0, 0, 0), 0, 0.5, (1, 1, 1)),
                        rec3d((-0.5, 0.0, 0.4), (0.01,) * 3, (1, 0, 0, 0), (0, 0, 0), 0, 0.5, (1, 1, 1))])
    r = oracle.project3d(p, cam, H, W)
    fx = float(cam[12])
    np.testing.assert_allclose(r[0, 2:4], [fx * 0.3 / 5 + W / 2, -fx * -0.2 / 5 + H / 2], rtol=1e-6)
    np.testing.assert_allclose(r[1, 2:4], [fx * -0.5 / 5 + W / 2, -fx * 0.4 / 5 + H / 2], rtol=1e-6)
    np.testing.assert_allclose(r[:, 1], [5.0, 5.0], rtol=1e-6)


@pytest.mark.parametrize("axis", [0, 1])
def test_projected_frequency_of_a_facing_disc(axis):
    """Sec. 4.1 (reading: f' is the phase gradient on the fronto-parallel plane through the centre).
    A flat disc facing the camera at depth tz with f along camera x (or y) shows, along the image
    row (column) through its centre, alpha = o (1 + cos(2 pi f tz / fx du + phi)) / 2 exp(-du^2 / 2 s'^2)
    with s'^2 = (fx sigma / tz)^2 + 0.3."""
    H, W = 65, 65
    fx = 200.0
    cam = cam_identity(H, W, fx=fx)
    cam[14] = cam[15] = 32.5  # principal point on a pixel centre
    tz, sig, f0, phi, o = 3.0, 0.05, 3.0, 0.7, 0.6
    f = [0.0, 0.0, 0.0]
    f[axis] = f0
    p = rec3d((0, 0, tz), (sig, sig, 1e-5), (1, 0, 0, 0), f, phi, o, (1, 1, 1))
    C, T, nc, amb = oracle.render3d(p, cam, H, W, OPTS_EXACT, truncated=False)
    du = np.arange(W) + 0.5 - 32.5
    line = C[32, :, 0] if axis == 0 else C[:, 32, 0]
    tzf, sigf, f0f, phif, of = (float(np.float32(v)) for v in (tz, sig, f0, phi, o))
    s2 = (fx * sigf / tzf) ** 2 + 0.3
    expect = of * 0.5 * (1 + np.cos(2 * math.pi * f0f * tzf / fx * du + phif)) * np.exp(-0.5 * du ** 2 / s2)
    np.testing.assert_allclose(line, expect, rtol=1e-5, atol=1e-9)


def test_frequency_along_view_axis_is_dropped():
    """Sec. 4.1: the projected frequency keeps (f_x, f_y) only; a frequency along the viewing axis
    leaves the splat a plain Gaussian modulated by the constant (1 + cos phi) / 2."""
    H, W = 33, 33
    cam = cam_identity(H, W, fx=150.0)
    a = rec3d((0, 0, 2.0), (0.04, 0.06, 0.03), (0.9, 0.1, -0.2, 0.3), (0, 0, 0), 0.9, 0.5, (1, 1, 1))
    b = a.copy()
    b[0, 12] = 25.0
    Ca = oracle.render3d(a, cam, H, W, OPTS_EXACT, truncated=False)[0]
    Cb = oracle.render3d(b, cam, H, W, OPTS_EXACT, truncated=False)[0]
    np.testing.assert_allclose(Ca, Cb, rtol=1e-12, atol=1e-15)


def test_front_to_back_two_layers():
    """Eq. 3 with W': two primitives on the optical axis, the nearer one first:
    C = c1 a1 + c2 a2 (1 - a1) + (1 - a1)(1 - a2) bg with a = o (1 + cos phi) / 2 at the centre."""
    H, W = 33, 33
    cam = cam_identity(H, W, fx=100.0)
    cam[14] = cam[15] = 16.5
    near = rec3d((0, 0, 2.0), (0.05, 0.05, 0.05), (1, 0, 0, 0), (0, 0, 0), 0.8, 0.7, (1.0, 0.2, 0.1))
    far = rec3d((0, 0, 3.0), (0.2, 0.2, 0.2), (1, 0, 0, 0), (0, 0, 0), 2.0, 0.9, (0.1, 0.3, 1.0))
    opts = np.array([3.0, 1 / 255, 0.99, 1e-4, 0.3, 0.25, 0.5, 0.75], np.float32)
    for p in (np.concatenate([near, far]), np.concatenate([far, near])):
        C, T, nc, amb = oracle.render3d(p, cam, H, W, opts, pixels=[[16, 16]])
        a1 = float(np.float32(0.7)) * 0.5 * (1 + math.cos(float(np.float32(0.8))))
        a2 = float(np.float32(0.9)) * 0.5 * (1 + math.cos(float(np.float32(2.0))))
        c1, c2 = near[0, 15:18].astype(np.float64), far[0, 15:18].astype(np.float64)
        bg = opts[5:8].astype(np.float64)
        expect = c1 * a1 + c2 * a2 * (1 - a1) + (1 - a1) * (1 - a2) * bg
        np.testing.assert_allclose(C[0], expect, rtol=1e-12)
        assert T[0] == pytest.approx((1 - a1) * (1 - a2), rel=1e-12)
        assert nc[0] == 2


def test_transmittance_floor_stops_blending():
    """Blending stops before a primitive that would take T below T_min: with alpha = 0.95 per
    layer T goes 0.05, 2.5e-3, 1.25e-4, and the fourth layer (6.25e-6 < 1e-4) is not added."""
    H, W = 17, 17
    cam = cam_identity(H, W, fx=100.0)
    cam[14] = cam[15] = 8.5
    layers = [rec3d((0, 0, 2.0 + k), (0.1, 0.1, 0.1), (1, 0, 0, 0), (0, 0, 0), 0.0, 0.95, (1, 1, 1)) for k in range(6)]
    p = np.concatenate(layers)
    C, T, nc, amb = oracle.render3d(p, cam, H, W, pixels=[[8, 8]])
    a = float(np.float32(0.95))
    assert nc[0] == 3
    assert T[0] == pytest.approx((1 - a) ** 3, rel=1e-12)
    assert C[0, 0] == pytest.approx(a + a * (1 - a) + a * (1 - a) ** 2, rel=1e-12)


def test_alpha_floor_and_ceiling():
    """alpha below 1/255 is skipped; o W' above alpha_max is clamped to 0.99."""
    H, W = 17, 17
    cam = cam_identity(H, W, fx=100.0)
    cam[14] = cam[15] = 8.5
    faint = rec3d((0, 0, 2.0), (0.1,) * 3, (1, 0, 0, 0), (0, 0, 0), 0.0, 0.003, (1, 1, 1))
    solid = rec3d((0, 0, 3.0), (0.1,) * 3, (1, 0, 0, 0), (0, 0, 0), 0.0, 1.0, (0.5, 0.5, 0.5))
    C, T, nc, amb = oracle.render3d(np.concatenate([faint, solid]), cam, H, W, pixels=[[8, 8]])
    assert nc[0] == 1
    amax = float(np.float32(0.99))
    assert C[0, 0] == pytest.approx(0.5 * amax, rel=1e-12)
    assert T[0] == pytest.approx(1 - amax, rel=1e-12)


def test_blend_first_order_is_summed_field():
    """With every alpha small the front-to-back blend equals the summed field of c alpha up to
    second order: |C - sum c a| <= max|c| (sum a)^2 / 2."""
    H, W = 40, 40
    p = synth.scene3d(80, 31)
    p[:, 14] = 0.01
    cam = synth.sphere_cameras(1, H, W, 32)[0]
    C = oracle.render3d(p, cam, H, W, OPTS_EXACT, truncated=False)[0]
    # the same scene with every opacity scaled to 1e-8: pure first order
    q = p.copy()
    q[:, 14] = 1e-8
    lin = oracle.render3d(q, cam, H, W, OPTS_EXACT, truncated=False)[0] * (0.01 / 1e-8)
    asum = lin.max(axis=2)  # colours are <= 1, so sum a >= the largest channel of sum c a
    # bound with the exact alpha sum per pixel from a white copy
    w = q.copy()
    w[:, 15:18] = 1.0
    asum = oracle.render3d(w, cam, H, W, OPTS_EXACT, truncated=False)[0][..., 0] * (0.01 / 1e-8)
    assert np.all(np.abs(C - lin) <= 0.5 * asum[..., None] ** 2 + 1e-12)
    assert np.abs(C - lin).max() > 0


def test_grad3d_matches_central_differences():
    """Analytic gradient through blending, projection (J, Sigma', mu', f') and the quaternion
    against central differences of the binary64 forward (no thresholds)."""
    H, W = 28, 32
    p = synth.scene3d(6, 41, scale_range=(0.03, 0.08), max_freq=6.0, extent=0.3)
    p[:, 14] = np.linspace(0.3, 0.8, 6)
    cam = synth.camera(synth.look_at((0.4, -2.2, 0.9)), H, W, 50.0)
    g = synth.upstream_grad(H, W, 42)
    an = oracle.grad3d(p, cam, H, W, g, OPTS_EXACT, truncated=False)
    cols = list(range(18))
    floor = [0.3] * 3 + [0.03] * 3 + [0.5] * 4 + [1.0] * 3 + [1.0] + [0.3] + [0.3] * 3

    def L(pp):
        return float((oracle.render3d(pp, cam, H, W, OPTS_EXACT, truncated=False)[0] * g).sum())

    fd = _central_fd(L, p, range(len(p)), cols, floor=floor)
    ref = an[:, cols]
    err = np.abs(ref - fd)
    tol = 1e-5 * np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max(axis=0, keepdims=True))
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-300)).max()


# ---------------------------------------------------------------------------------------------
# literal frequency projection (opt-in reading of Sec. 4.1): f' = J W f
# ---------------------------------------------------------------------------------------------

OPTS_LITERAL = np.array([3.0, 1.0 / 255.0, 0.99, 1e-4, 0.3, 0.0, 0.0, 0.0, 1.0], np.float32)


def test_literal_frequency_projection_closed_forms():
    """Putting f through the covariance's map J (Sec. 4.1 read literally): on the optical axis a
    frequency facing the camera becomes (fx f_x / tz, fy f_y / tz), where the default reading
    gives (f_x tz / fx, f_y tz / fy); off axis a frequency along the view axis becomes
    f_z (-fx tx / tz^2, -fy ty / tz^2), the third column of J, where the default drops it."""
    H, W = 200, 240
    fx, fy = 300.0, 280.0
    cam = cam_identity(H, W, fx=fx, fy=fy)
    p = rec3d((0, 0, 5.0), (0.1, 0.1, 0.1), (1, 0, 0, 0), (0.25, -0.5, 0.0), 0.0, 0.5, (1, 1, 1))
    np.testing.assert_allclose(oracle.project3d(p, cam, H, W, OPTS_LITERAL)[0, 7:9], [fx * 0.25 / 5, -fy * 0.5 / 5],
                               rtol=1e-12)
    np.testing.assert_allclose(oracle.project3d(p, cam, H, W)[0, 7:9], [0.25 * 5 / fx, -0.5 * 5 / fy], rtol=1e-12)
    tx, ty, tz, fz = 0.7, -0.4, 4.0, 0.3
    p = rec3d((tx, ty, tz), (0.05,) * 3, (1, 0, 0, 0), (0.0, 0.0, fz), 0.0, 0.5, (1, 1, 1))
    tx, ty, tz, fz = (float(np.float32(v)) for v in (tx, ty, tz, fz))
    np.testing.assert_allclose(oracle.project3d(p, cam, H, W, OPTS_LITERAL)[0, 7:9],
                               [-fx * tx / tz ** 2 * fz, -fy * ty / tz ** 2 * fz], rtol=1e-12)
    np.testing.assert_allclose(oracle.project3d(p, cam, H, W)[0, 7:9], [0.0, 0.0], atol=1e-15)


def test_literal_frequency_grad_matches_central_differences():
    """The gradient with f' = J W f (through J's dependence on the centre, and W^T J^T to f)
    against central differences of the binary64 forward (no thresholds)."""
    H, W = 28, 32
    p = synth.scene3d(6, 43, scale_range=(0.03, 0.08), max_freq=0.05, extent=0.3)
    p[:, 14] = np.linspace(0.3, 0.8, 6)
    cam = synth.camera(synth.look_at((0.4, -2.2, 0.9)), H, W, 50.0)
    g = synth.upstream_grad(H, W, 44)
    opts = OPTS_EXACT.copy()
    opts = np.concatenate([opts, [1.0]]).astype(np.float32)
    an = oracle.grad3d(p, cam, H, W, g, opts, truncated=False)
    cols = list(range(18))
    floor = [0.3] * 3 + [0.03] * 3 + [0.5] * 4 + [0.05] * 3 + [1.0] + [0.3] + [0.3] * 3

    def L(pp):
        return float((oracle.render3d(pp, cam, H, W, opts, truncated=False)[0] * g).sum())

    fd = _central_fd(L, p, range(len(p)), cols, floor=floor)
    err = np.abs(an[:, cols] - fd)
    tol = 1e-5 * np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max(axis=0, keepdims=True))
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-300)).max()
    # the mode matters: the default reading gives a different frequency gradient here
    an0 = oracle.grad3d(p, cam, H, W, g, OPTS_EXACT, truncated=False)
    assert np.abs(an0[:, 10:13] - an[:, 10:13]).max() > 1e-3 * np.abs(an[:, 10:13]).max()


# ---------------------------------------------------------------------------------------------
# frequency map 2 (opt-in reading of Sec. 4.1): the oscillation integrated along the viewing ray,
# with the damping factor the integral over z brings
# ---------------------------------------------------------------------------------------------

OPTS_RAY = np.array([3.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0], np.float32)  # exact, no dilation


def _camera_frame(p, cam):
    """Camera-frame centre t, covariance Sigma_c and frequency fc of a 3D record (scipy's rotation,
    numpy products), and the pixel Jacobian J of the pinhole map at t."""
    from scipy.spatial.transform import Rotation

    V = cam[:12].reshape(3, 4).astype(np.float64)
    fx, fy = float(cam[12]), float(cam[13])
    r = p.astype(np.float64)
    t = V[:, :3] @ r[0:3] + V[:, 3]
    q = r[6:10] / np.linalg.norm(r[6:10])
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = V[:, :3] @ R @ np.diag(r[3:6] ** 2) @ R.T @ V[:, :3].T
    fc = V[:, :3] @ r[10:13]
    J = np.array([[fx / t[2], 0.0, -fx * t[0] / t[2] ** 2], [0.0, fy / t[2], -fy * t[1] / t[2] ** 2]])
    return t, Sig, fc, J


def _ray_integral(p, cam, a):
    """W'(a) of one primitive at image-plane offset a (pixels from the projected centre): the 3D
    wavelet integrated numerically along the line of camera-frame offsets y with J y = a (the
    viewing ray of the affine ray space), over the Gaussian integrated along the line through the
    centre.  The line comes from J's pseudo-inverse and null space (SVD); trapezoid rule over
    +-16 of the largest scale, far finer than the oscillation."""
    t, Sig, fc, J = _camera_frame(p, cam)
    Sinv = np.linalg.inv(Sig)
    n = np.linalg.svd(J)[2][2]  # unit direction with J n = 0
    smax = float(np.max(p[3:6]))
    phi = float(p[13])

    def line(y0, cosine):
        zc = -float(n @ y0)
        z = np.linspace(zc - 16 * smax, zc + 16 * smax, 40001)
        y = y0[None, :] + z[:, None] * n[None, :]
        G = np.exp(-0.5 * np.einsum("ki,ij,kj->k", y, Sinv, y))
        f = 0.5 * (np.cos(2 * math.pi * (y @ fc) + phi) + 1.0) * G if cosine else G
        return np.trapezoid(f, z)

    y0 = np.linalg.pinv(J) @ np.asarray(a, np.float64)
    return line(y0, True) / line(np.zeros(3), False)


def test_ray_integrated_frequency_matches_quadrature_along_the_ray():
    """Sec. 4.1 integrates the 3D wavelet over z.  In the EWA ray space (the same affine map as the
    covariance projection) the oracle's closed form (f' and the damping kappa from completing the
    square, with the marginal Gaussian of Sigma') must equal numerical quadrature of the 3D
    wavelet along the viewing line, for rotated anisotropic primitives off the optical axis under
    a rotated camera, at pixels across the footprint.  A dropped damping, a wrong sign of the
    correction term, the conditional taken along the optical axis instead of the ray, or Sigma in
    place of its inverse fails here."""
    H, W = 120, 160
    cam = synth.camera(synth.look_at((0.6, -2.5, 0.8)), H, W, 50.0)
    rng = np.random.default_rng(71)
    checked = 0
    kaps = []
    for trial in range(4):
        mu = rng.uniform(-0.25, 0.25, 3)
        s = np.exp(rng.uniform(np.log(0.03), np.log(0.08), 3))
        q = rng.standard_normal(4)
        p = rec3d(mu, s, q / np.linalg.norm(q), (0, 0, 0), rng.uniform(0, 2 * math.pi), 0.5, (1, 1, 1))
        # a frequency with a component of 3 cycles/unit along the viewing ray and 2 across it
        t = _camera_frame(p[0], cam)[0]
        V = cam[:12].reshape(3, 4).astype(np.float64)[:, :3]
        fcam = 3.0 * t / np.linalg.norm(t) + 2.0 * rng.standard_normal(3) / math.sqrt(3.0)
        p[0, 10:13] = V.T @ fcam
        proj = oracle.project3d(p, cam, H, W, OPTS_RAY)[0]
        kaps.append(proj[14])
        mx, my = proj[2], proj[3]
        Sd = np.array([[proj[4], proj[5]], [proj[5], proj[6]]])
        pix = []
        for _ in range(12):
            d = rng.multivariate_normal([0, 0], Sd)
            u, v = int(np.floor(mx + d[0])), int(np.floor(my + d[1]))
            if 0 <= u < W and 0 <= v < H:
                pix.append((u, v))
        C = oracle.render3d(p, cam, H, W, OPTS_RAY, truncated=False, pixels=pix)[0]
        for (u, v), c in zip(pix, C[:, 0]):
            ref = _ray_integral(p[0], cam, (u + 0.5 - mx, v + 0.5 - my))
            assert abs(c / float(np.float32(0.5)) - ref) <= 1e-9, (trial, u, v, c, ref)
            checked += 1
    assert checked >= 30
    assert max(kaps) < 0.99 and min(kaps) < 0.7, kaps  # dampings that matter


def test_ray_integrated_frequency_across_the_ray_is_the_plane_gradient():
    """A frequency perpendicular to the viewing ray (fc . n = 0) is not damped by the integral and
    its projection is the phase gradient on the fronto-parallel plane (frequency map 0)."""
    H, W = 120, 160
    cam = synth.camera(synth.look_at((0.6, -2.5, 0.8)), H, W, 50.0)
    mu = np.array([0.1, -0.05, 0.2])
    p = rec3d(mu, (0.05, 0.08, 0.03), (0.7, 0.2, -0.4, 0.5), (0, 0, 0), 0.4, 0.5, (1, 1, 1))
    t, Sig, fc, J = _camera_frame(p[0], cam)
    n = t / t[2]  # the viewing direction through the centre (unclamped)
    V = cam[:12].reshape(3, 4).astype(np.float64)[:, :3]
    fcam = np.cross(n, [0.3, 1.0, -0.2])
    fcam *= 5.0 / np.linalg.norm(fcam)
    p[0, 10:13] = V.T @ fcam
    p32 = p.astype(np.float32)
    t, Sig, fc, J = _camera_frame(p32[0], cam)
    assert abs(fc @ (t / t[2])) < 1e-6 * np.linalg.norm(fc)
    r2 = oracle.project3d(p32, cam, H, W, OPTS_RAY)[0]
    r0 = oracle.project3d(p32, cam, H, W, OPTS_EXACT)[0]
    np.testing.assert_allclose(r2[7:9], r0[7:9], rtol=1e-5, atol=1e-12)
    assert abs(r2[14] - 1.0) < 1e-9


def test_ray_integrated_damping_on_axis_isotropic_closed_form():
    """On the optical axis with an isotropic Gaussian of std sigma the viewing ray is the z axis and
    the z integral of cos(2 pi f_z z) exp(-z^2 / 2 sigma^2) over that of the Gaussian is the
    Gaussian's Fourier transform exp(-2 pi^2 f_z^2 sigma^2); the in-plane frequency keeps the map-0
    value (f_x tz / fx, f_y tz / fy)."""
    H, W = 64, 80
    fx, fy = 300.0, 250.0
    cam = cam_identity(H, W, fx=fx, fy=fy)
    for sig, f in [(0.05, (1.0, -2.0, 4.0)), (0.1, (0.0, 0.5, 2.5)), (0.02, (3.0, 0.0, -9.0))]:
        p = rec3d((0, 0, 5.0), (sig,) * 3, (0.6, -0.3, 0.2, 0.7), f, 0.0, 0.5, (1, 1, 1))
        r = oracle.project3d(p, cam, H, W, OPTS_RAY)[0]
        sg, fz, f0, f1 = (float(np.float32(v)) for v in (sig, f[2], f[0], f[1]))
        assert r[14] == pytest.approx(math.exp(-2 * math.pi ** 2 * fz ** 2 * sg ** 2), rel=1e-6)
        np.testing.assert_allclose(r[7:9], [f0 * 5.0 / fx, f1 * 5.0 / fy], rtol=1e-6, atol=1e-14)


def test_ray_integrated_frequency_grad_matches_central_differences():
    """The gradient under frequency map 2 (f' and kappa through the centre, the scales, the
    rotation and the frequency) against central differences of the binary64 forward."""
    H, W = 28, 32
    p = synth.scene3d(6, 47, scale_range=(0.03, 0.08), max_freq=6.0, extent=0.3)
    p[:, 14] = np.linspace(0.3, 0.8, 6)
    cam = synth.camera(synth.look_at((0.4, -2.2, 0.9)), H, W, 50.0)
    g = synth.upstream_grad(H, W, 48)
    opts = OPTS_EXACT.copy()
    opts = np.concatenate([opts, [2.0]]).astype(np.float32)
    kap = oracle.project3d(p, cam, H, W, opts)[:, 14]
    assert kap.min() < 0.9  # the damping takes part
    an = oracle.grad3d(p, cam, H, W, g, opts, truncated=False)
    cols = list(range(18))
    floor = [0.3] * 3 + [0.03] * 3 + [0.5] * 4 + [1.0] * 3 + [1.0] + [0.3] + [0.3] * 3

    def L(pp):
        return float((oracle.render3d(pp, cam, H, W, opts, truncated=False)[0] * g).sum())

    fd = _central_fd(L, p, range(len(p)), cols, floor=floor)
    err = np.abs(an[:, cols] - fd)
    tol = 1e-5 * np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max(axis=0, keepdims=True))
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-300)).max()
    # the map matters: map 0 gives a different gradient here
    an0 = oracle.grad3d(p, cam, H, W, g, OPTS_EXACT, truncated=False)
    assert np.abs(an0[:, 10:13] - an[:, 10:13]).max() > 1e-2 * np.abs(an[:, 10:13]).max()


# ---------------------------------------------------------------------------------------------
# spherical-harmonic colour (the view-dependent colour of 3DGS, Sec. 3.1)
# ---------------------------------------------------------------------------------------------

OPTS_SH3 = np.array([3.0, 0.0, 1.0, 0.0, 0.3, 0.0, 0.0, 0.0, 0.0, 3.0], np.float32)  # exact, SH degree 3


def test_sh_basis_is_orthonormal_on_the_sphere():
    """Gauss-Legendre in cos(theta) times uniform azimuth integrates products of degree <= 3
    harmonics exactly: the 16 functions are orthonormal."""
    ct, wt = np.polynomial.legendre.leggauss(8)
    ph = np.arange(16) * (2 * math.pi / 16)
    st = np.sqrt(1 - ct * ct)
    d = np.stack([np.outer(st, np.cos(ph)).ravel(), np.outer(st, np.sin(ph)).ravel(), np.repeat(ct, 16)], 1)
    w = np.repeat(wt, 16) * (2 * math.pi / 16)
    Y = oracle.sh_basis(d)
    np.testing.assert_allclose((Y * w[:, None]).T @ Y, np.eye(16), atol=1e-12)


def test_sh_basis_matches_scipy_real_harmonics():
    """The basis is scipy's complex spherical harmonics (with the Condon-Shortley phase) made real:
    sqrt(2) Im Y_l^|m| for m < 0, Y_l^0, sqrt(2) Re Y_l^m for m > 0, ordered m = -l..l."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    polar, az = np.arccos(d[:, 2]), np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.sh_basis(d)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            c = sp.sph_harm_y(l, abs(m), polar, az)
            ref = c.real if m == 0 else math.sqrt(2) * (c.imag if m < 0 else c.real)
            np.testing.assert_allclose(Y[:, k], ref, atol=1e-12)
            k += 1


def test_sh_record_with_only_the_constant_term_renders_the_rgb_record():
    """Degree-0 coefficients (c - 1/2) / Y_0^0 and nothing else reproduce the plain colour c."""
    H, W = 40, 44
    p = synth.scene3d(300, 51)
    q = np.zeros((len(p), synth.P3D_SH), np.float32)
    q[:, :20] = p
    q[:, 15:18] = (p[:, 15:18].astype(np.float64) - 0.5) / (0.5 / math.sqrt(math.pi))
    cam = synth.sphere_cameras(1, H, W, 52)[0]
    a = oracle.render3d(p, cam, H, W, OPTS_EXACT, truncated=False)[0]
    b = oracle.render3d(q, cam, H, W, OPTS_SH3, truncated=False)[0]
    assert np.abs(a - b).max() <= 1e-6


def test_sh_colour_is_taken_in_the_direction_from_the_camera_to_the_centre():
    """A camera at (0, -5, 0) looking at a primitive at the origin sees it in direction +y: with a
    single degree-1 coefficient s on the basis function of index 1, the centre pixel shows
    1/2 + Y_1(0, 1, 0) s (times opacity, the primitive's peak)."""
    H, W = 41, 41
    cam = synth.camera(synth.look_at((0.0, -5.0, 0.0)), H, W, 50.0)
    q = np.zeros((1, synth.P3D_SH), np.float32)
    q[0, :18] = [0, 0, 0, 0.05, 0.05, 0.05, 1, 0, 0, 0, 0, 0, 0, 0, 0.5, 0, 0, 0]
    q[0, 15:18] = 0.0
    q[0, 20:23] = 0.3  # band 1, m = -1
    C = oracle.render3d(q, cam, H, W, OPTS_SH3, truncated=False)[0]
    y1 = oracle.sh_basis(np.array([[0.0, 1.0, 0.0]]))[0, 1]
    # the centre pixel sits on mu' (q = 0, W' = 1): alpha = opacity 0.5, C = 0.5 c
    np.testing.assert_allclose(C[20, 20], 0.5 * (0.5 + y1 * np.float32(0.3)), rtol=1e-9)


def test_sh_grad_matches_central_differences():
    """Gradient of the SH colour (coefficients, and the centre through the view direction) against
    central differences of the binary64 forward."""
    H, W = 26, 30
    p = synth.scene3d_sh(5, 53, scale_range=(0.03, 0.08), max_freq=6.0, extent=0.3)
    p[:, 14] = np.linspace(0.3, 0.8, 5)
    cam = synth.camera(synth.look_at((0.4, -2.2, 0.9)), H, W, 50.0)
    g = synth.upstream_grad(H, W, 54)
    an = oracle.grad3d(p, cam, H, W, g, OPTS_SH3, truncated=False)
    cols = [0, 1, 2, 15, 16, 17] + list(range(20, 65))
    floor = [0.3] * synth.P3D_SH

    def L(pp):
        return float((oracle.render3d(pp, cam, H, W, OPTS_SH3, truncated=False)[0] * g).sum())

    fd = _central_fd(L, p, range(len(p)), cols, floor=floor)
    err = np.abs(an[:, cols] - fd)
    tol = 1e-5 * np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max(axis=0, keepdims=True))
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-300)).max()


# ---------------------------------------------------------------------------------------------
# binary32 footprint rule and tile lists (the 3DGS-style pipeline the paper follows, Sec. 4.1)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dims,scale", [(2, (1.0, 16.0)), (2, (0.5, 32.0)), (3, None)])
def test_cutoff_ellipse_inside_covered_range(dims, scale):
    """Tile culling loses nothing: every pixel that passes the binary32 3-sigma test lies inside the
    primitive's covered pixel range and in a tile (and a one-pixel rectangle) that the ellipse test
    accepts, including very elongated primitives (scale ratio up to 64)."""
    if dims == 2:
        H, W = 128, 160
        p = synth.scene2d(1500, H, W, 7, scale)
        inside, outside, rect, dropped = oracle.cutoff_coverage(2, p, H, W)
    else:
        H, W = 96, 112
        p = synth.scene3d(2500, 8)
        cam = synth.sphere_cameras(1, H, W, 9)[0]
        inside, outside, rect, dropped = oracle.cutoff_coverage(3, p, H, W, cam)
    assert inside > 0 and outside == 0 and dropped == 0 and rect >= inside


@pytest.mark.parametrize("dims", [2, 3])
def test_footprint_matches_binary64_projection(dims):
    """The binary32 Cholesky factor L of the inverse covariance reproduces the binary64 Sigma'^-1:
    L L^T = Sigma'^-1 to single-precision accuracy, and the centre matches mu'."""
    if dims == 2:
        H, W = 64, 64
        p = synth.scene2d(300, H, W, 13, (0.5, 32.0))
        rec, rect, valid = oracle.footprints(2, p, H, W)
        for i in range(len(p)):
            c, s = math.cos(p[i, 4]), math.sin(p[i, 4])
            R = np.array([[c, -s], [s, c]])
            K = np.linalg.inv(R @ np.diag(p[i, 2:4].astype(np.float64) ** 2) @ R.T)
            L = np.array([[rec[i, 2], 0.0], [rec[i, 3], rec[i, 4]]], np.float64)
            np.testing.assert_allclose(L @ L.T, K, rtol=2e-5, atol=2e-5 * np.abs(K).max())
            np.testing.assert_allclose(rec[i, :2], p[i, :2])
    else:
        H, W = 120, 100
        p = synth.scene3d(400, 14)
        cam = synth.sphere_cameras(1, H, W, 15)[0]
        rec, rect, valid = oracle.footprints(3, p, H, W, cam)
        pr = oracle.project3d(p, cam, H, W)
        assert np.array_equal(valid.astype(bool), pr[:, 0].astype(bool))
        for i in np.nonzero(valid)[0]:
            S = np.array([[pr[i, 4], pr[i, 5]], [pr[i, 5], pr[i, 6]]])
            K = np.linalg.inv(S)
            L = np.array([[rec[i, 2], 0.0], [rec[i, 3], rec[i, 4]]], np.float64)
            np.testing.assert_allclose(L @ L.T, K, rtol=1e-4, atol=1e-4 * np.abs(K).max())
            np.testing.assert_allclose(rec[i, :2], pr[i, 2:4], rtol=1e-5)
            assert rec[i, 7] == pytest.approx(pr[i, 1], rel=1e-6)


@pytest.mark.parametrize("dims", [2, 3])
def test_tile_lists_enumerate_covered_tiles_in_order(dims):
    """The sorted lists are ordered by tile, then camera depth (3D), then primitive index; every
    listed tile lies in the primitive's covered pixel range, and every tile holding a pixel well
    inside the cutoff ellipse (binary64 q <= 9 (1 - 1e-4)) is listed."""
    H, W = 72, 88
    if dims == 2:
        p = synth.scene2d(120, H, W, 17, (1.0, 12.0))
        cam = None
    else:
        p = synth.scene3d(600, 18)
        cam = synth.sphere_cameras(1, H, W, 19)[0]
    rec, rect, valid = oracle.footprints(dims, p, H, W, cam)
    tiles, prims = oracle.tile_lists(dims, p, H, W, cam)
    ntx = (W + 15) // 16
    depth = rec[:, 7].view(np.uint32) if dims == 3 else np.zeros(len(p), np.uint32)
    keys = [(int(t), int(depth[i]), int(i)) for t, i in zip(tiles, prims)]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    listed = set((int(t), int(i)) for t, i in zip(tiles, prims))
    for t, i in listed:
        u0, v0, u1, v1 = rect[i]
        assert valid[i] and u0 // 16 <= t % ntx <= u1 // 16 and v0 // 16 <= t // ntx <= v1 // 16
    # binary64 inverse covariance per primitive
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    if dims == 3:
        pr = oracle.project3d(p, cam, H, W)
    must = 0
    for i in range(len(p)):
        if not valid[i]:
            continue
        if dims == 2:
            c, sn = math.cos(p[i, 4]), math.sin(p[i, 4])
            R = np.array([[c, -sn], [sn, c]])
            K = np.linalg.inv(R @ np.diag(p[i, 2:4].astype(np.float64) ** 2) @ R.T)
            mu = p[i, :2].astype(np.float64)
        else:
            K = np.linalg.inv(np.array([[pr[i, 4], pr[i, 5]], [pr[i, 5], pr[i, 6]]]))
            mu = pr[i, 2:4]
        dx, dy = xx - mu[0], yy - mu[1]
        q = K[0, 0] * dx * dx + 2 * K[0, 1] * dx * dy + K[1, 1] * dy * dy
        vv, uu = np.nonzero(q <= 9.0 * (1 - 1e-4))
        for t in set((vv // 16) * ntx + uu // 16):
            must += 1
            assert (int(t), i) in listed
    assert must > 0 and len(listed) >= must


# ---------------------------------------------------------------------------------------------
# 6D: linear time model (reading of the deformation of Sec. 4.3)
# ---------------------------------------------------------------------------------------------

def test_deform6d_identity_at_time_zero_and_rates():
    p = synth.scene6d(50, 3)
    d0 = oracle.deform6d(p, 0.0)
    np.testing.assert_array_equal(d0, p[:, :20].astype(np.float64))
    d1 = oracle.deform6d(p, 0.5)
    q = p.astype(np.float64)
    np.testing.assert_allclose(d1[:, 0:3], q[:, 0:3] + 0.5 * q[:, 20:23])
    np.testing.assert_allclose(d1[:, 3:6], q[:, 3:6] * np.exp(0.5 * q[:, 27:30]))
    np.testing.assert_allclose(d1[:, 13], q[:, 13] + 0.5 * q[:, 26])


def test_deform6d_grad_matches_central_differences():
    p = synth.scene6d(4, 5)
    t = 0.37
    g3 = np.random.default_rng(6).standard_normal((4, 20))
    an = oracle.deform6d_grad(p, t, g3)

    def L(pp):
        return float((oracle.deform6d(pp, t) * g3).sum())

    fd = _central_fd(L, p, range(4), range(30), floor=[1.0] * 20 + [0.05] * 10)
    np.testing.assert_allclose(an[:, :30], fd, rtol=1e-6, atol=1e-8)


def _f32_fma(a, b, c):
    """binary32 fused multiply-add: the product of two binary32 values is exact in binary64, so
    one rounding of the binary64 sum to binary32 emulates it (up to a double rounding that is far
    below the bounds checked here)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _decision_pairs(seed, fmode):
    """(primitive, pixel) pairs inside the cutoff of a dense 3D view, with the oracle's decision values."""
    H, W = 96, 96
    p = synth.scene3d(20000, seed)
    cam = synth.sphere_cameras(1, H, W, seed + 1)[0]
    opts = np.array([3.0, 1.0 / 255.0, 0.99, 1e-4, 0.3, 0.0, 0.0, 0.0, float(fmode)], np.float32)
    if fmode == 1:
        p[:, 10:13] *= 0.02  # the literal map scales f by about fx / tz
    rec, _, valid = oracle.footprints(3, p, H, W, cam)
    rng = np.random.default_rng(seed)
    prims = np.nonzero(valid)[0]
    pairs = []
    for i in rng.choice(prims, 3000):
        u = int(rng.integers(0, W)); v = int(rng.integers(0, H))
        # a pixel near the centre, so that most pairs fall inside the cutoff
        u = int(np.clip(round(rec[i, 0] - 0.5 + rng.normal(0, rec[i, 5] / 3.0)), 0, W - 1))
        v = int(np.clip(round(rec[i, 1] - 0.5 + rng.normal(0, rec[i, 6] / 3.0)), 0, H - 1))
        pairs.append((i, u, v))
    pairs = np.array(pairs, np.int32)
    r10, out = oracle.alpha_decisions(p, cam, H, W, pairs, opts)
    k2 = np.float32(9.0)
    # keep the pairs inside the binary32 cutoff (the decision is only taken there)
    m = r10[pairs[:, 0]]
    dx = (pairs[:, 1].astype(np.float32) + np.float32(0.5)) - m[:, 0]
    dy = (pairs[:, 2].astype(np.float32) + np.float32(0.5)) - m[:, 1]
    a = _f32_fma(m[:, 2], dx, m[:, 3] * dy)
    b = m[:, 4] * dy
    q = _f32_fma(a, a, b * b)
    inside = q <= k2
    return pairs[inside], m[inside], out[inside], dx[inside], dy[inside], q[inside]


@pytest.mark.parametrize("fmode", [0, 1, 2])
def test_threshold_decision_alpha_bound_covers_binary32_evaluation(fmode):
    """Eq. 3's threshold decisions (alpha_min skip, alpha_max clamp, T_min stop) are taken from the
    binary32 projected record; the oracle's per-pair bound must cover the error of evaluating alpha
    in binary32 along the kernels' sequence of operations.  Emulated here in float32 with
    correctly rounded exp2 and cos (their approximate hardware forms are covered by the bound's
    documented instruction errors on top)."""
    pairs, m, out, dx, dy, q = _decision_pairs(301, fmode)
    assert len(pairs) > 1500
    f32 = np.float32
    e = q * f32(-0.7213475204444817)
    G = np.exp2(e.astype(np.float64)).astype(f32)
    t = _f32_fma(m[:, 5], dx, _f32_fma(m[:, 6], dy, m[:, 7]))
    r = (t + f32(12582912.0)) - f32(12582912.0)
    ang = (t - r) * f32(6.283185307179586)
    c = np.cos(ang.astype(np.float64)).astype(f32)
    # map 2: hk = kappa / 2 = ex2(kx) / 2 (correctly rounded here), else 1/2
    hk = (np.exp2(m[:, 9].astype(np.float64)).astype(f32) * f32(0.5)) if fmode == 2 else np.full_like(c, 0.5)
    M = _f32_fma(hk, c, np.full_like(c, 0.5))
    raw = m[:, 8] * (M * G)
    err = np.abs(raw.astype(np.float64) - out[:, 0])
    # the bound carries a safety factor of 1.5 over its first-order terms; the emulation must fit
    # within the terms themselves
    assert np.all(err <= out[:, 1] / 1.5), (err.max(), out[np.argmax(err / out[:, 1]), :])
    # and the bound is a few binary32 roundings of the pair's scale, not a blanket margin
    assert np.median(out[:, 1]) < 1e-6


@pytest.mark.parametrize("fmode", [0, 1, 2])
def test_threshold_decision_alpha_matches_binary64_projection(fmode):
    """The record the decisions read (centre, Cholesky factor, frequency under the chosen map,
    phase in cycles, opacity) is the binary32 rounding of the projection of Sec. 3.1 / Sec. 4.1:
    its alpha agrees with the binary64 projection's alpha to the rounding of the record.  A record
    built from a dropped phase, the other frequency map or a wrong opacity fails this."""
    pairs, m, out, dx, dy, q = _decision_pairs(302, fmode)
    diff = np.abs(out[:, 0] - out[:, 2])
    assert np.max(diff) < 2e-4, np.max(diff)
    assert np.median(diff) < 2e-6


def _ulps32(a, b):
    """Distance in binary32 units in the last place between same-shaped float32 arrays."""
    def ordered(x):
        i = np.ascontiguousarray(x, np.float32).view(np.int32).astype(np.int64)
        return np.where(i < 0, -(i & 0x7FFFFFFF), i)
    return np.abs(ordered(a) - ordered(b))


def test_footprint_rule_cos_sin_is_the_rounded_cosine_and_sine():
    """The 2D footprint rule's rotation (Sec. 3.1, Sigma = R S S^T R^T) takes cos and sin of the
    record's binary32 angle from a fixed sequence of IEEE operations (no library transcendental):
    binary32 with fused multiply-adds up to |theta| = 2^16, binary64 rounded once beyond.  Against
    numpy's binary64 cosine and sine of the same angles, rounded to binary32: every result of the
    binary32 branch within one ulp and most of them equal, every result of the binary64 branch
    equal; the symmetry under theta -> -theta holds bit for bit; special angles."""
    rng = np.random.default_rng(5)
    th = np.concatenate([np.linspace(0.0, math.pi, 100001), np.linspace(-60.0, 60.0, 100001),
                         rng.uniform(-65536.0, 65536.0, 100000)]).astype(np.float32)
    r = oracle.rule_cos_sin(th)
    t64 = th.astype(np.float64)
    for col, ref in ((0, np.cos(t64)), (1, np.sin(t64))):
        d = _ulps32(r[:, col], ref.astype(np.float32))
        assert d.max() <= 1, d.max()
        assert np.mean(d == 0) >= 0.8, np.mean(d == 0)
    # beyond 2^16: the binary64 branch, correctly rounded (k times the first two parts of pi/2 is
    # exact up to 2^20 quarter turns)
    wide = np.concatenate([rng.uniform(65537.0, 1.6e6, 20000), -rng.uniform(65537.0, 1.6e6, 20000)]).astype(np.float32)
    rw = oracle.rule_cos_sin(wide)
    w64 = wide.astype(np.float64)
    assert np.array_equal(rw[:, 0], np.cos(w64).astype(np.float32))
    assert np.array_equal(rw[:, 1], np.sin(w64).astype(np.float32))
    # cos is even and sin odd, bit for bit, in both branches
    both = np.concatenate([th, wide])
    pos, neg = oracle.rule_cos_sin(both), oracle.rule_cos_sin(-both)
    assert np.array_equal(neg[:, 0], pos[:, 0]) and np.array_equal(neg[:, 1], -pos[:, 1])
    # special angles
    sp = oracle.rule_cos_sin(np.array([0.0, math.pi / 2, math.pi, -math.pi / 2]))
    np.testing.assert_array_equal(sp[0], [1.0, 0.0])
    assert sp[1, 1] == 1.0 and abs(sp[1, 0]) < 1e-7
    assert sp[2, 0] == -1.0 and abs(sp[2, 1]) < 1e-7
    assert sp[3, 1] == -1.0
    # non-finite or absurd angles make the primitive invalid
    assert np.isnan(oracle.rule_cos_sin(np.array([np.inf, np.nan, 1e16, -1e16]))).all()

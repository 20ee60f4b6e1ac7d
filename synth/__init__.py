"""Seeded synthetic inputs for the WIPES rasterizer: scenes, cameras, targets and upstream gradients.

This module is shared by the tests, the benchmark and the serving driver.  It holds no part of
the rasterizer's arithmetic: it only draws parameters from the distributions that stand in for
the paper's workloads and lays them out in the record formats the library consumes.  Both the
oracle and the CUDA path receive exactly the arrays produced here.

Workload stand-ins (the paper's datasets and trained scenes are not available):
  * 2D image fitting, Section 5.1 (Kodak 768x512, DIV2K): ``scene2d`` with a photo-shaped
    target from ``target_noise_edges`` or ``target_gabor``.
  * 5D static novel view synthesis, Section 5.2 (Mip-NeRF360, Tanks&Temples, DeepBlending):
    ``scene3d`` viewed by ``sphere_cameras``.
  * 6D dynamic novel view synthesis, Section 5.3 (D-NeRF, NeRF-DS): ``scene6d`` with per-primitive
    linear time rates sampled at ``time_stamps``.

Record layouts (float32, row-major):
  2D  [N,16]: mu_x, mu_y, s_x, s_y, theta, f_x, f_y, phi, c_r, c_g, c_b, 0, 0, 0, 0, 0
              (pixels; frequency in cycles per pixel; phase in radians)
  3D  [N,20]: mu(3), s(3), q(w,x,y,z), f(3), phi, opacity, c(3), 0, 0
              (world units; frequency in cycles per unit)
  6D  [N,32]: the 3D record followed by v(3), df(3), dphi, dlog_s(3), 0, 0
  camera [17]: viewmat 3x4 row-major world->camera (OpenCV axes), fx, fy, cx, cy, near_z
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

P2D = 16
P3D = 20
P6D = 32
CAM_FLOATS = 17


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed)))


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def scene2d(n: int, H: int, W: int, seed: int, scale_range=(1.0, 16.0), max_freq=0.5) -> np.ndarray:
    """2D wavelet primitives: centres uniform over the image, log-uniform independent scales,
    rotation uniform in [0, pi), frequency magnitude uniform in [0, max_freq] cycles/px with a
    uniform direction, phase uniform in [0, 2 pi), colours uniform in [0, 1]."""
    rng = _rng(seed)
    p = np.zeros((n, P2D), dtype=np.float32)
    p[:, 0] = rng.uniform(0.0, W, n)
    p[:, 1] = rng.uniform(0.0, H, n)
    p[:, 2] = _log_uniform(rng, scale_range[0], scale_range[1], n)
    p[:, 3] = _log_uniform(rng, scale_range[0], scale_range[1], n)
    p[:, 4] = rng.uniform(0.0, math.pi, n)
    fm = rng.uniform(0.0, max_freq, n)
    fd = rng.uniform(0.0, 2.0 * math.pi, n)
    p[:, 5] = fm * np.cos(fd)
    p[:, 6] = fm * np.sin(fd)
    p[:, 7] = rng.uniform(0.0, 2.0 * math.pi, n)
    p[:, 8:11] = rng.uniform(0.0, 1.0, (n, 3))
    return p


def scene2d_cholesky(n: int, H: int, W: int, seed: int, scale_range=(1.0, 16.0), max_freq=0.5) -> np.ndarray:
    """2D wavelet primitives in the Cholesky record (mu, l1, l2, l3, f, phi, c): centres, frequency,
    phase and colours drawn as in scene2d; the diagonal entries l1, l3 log-uniform over the scale
    range with a random sign, the off-diagonal l2 uniform in [-l, l] with l log-uniform over the
    same range."""
    rng = _rng(seed)
    p = np.zeros((n, P2D), dtype=np.float32)
    p[:, 0] = rng.uniform(0.0, W, n)
    p[:, 1] = rng.uniform(0.0, H, n)
    p[:, 2] = _log_uniform(rng, scale_range[0], scale_range[1], n) * rng.choice([-1.0, 1.0], n)
    p[:, 3] = rng.uniform(-1.0, 1.0, n) * _log_uniform(rng, scale_range[0], scale_range[1], n)
    p[:, 4] = _log_uniform(rng, scale_range[0], scale_range[1], n) * rng.choice([-1.0, 1.0], n)
    fm = rng.uniform(0.0, max_freq, n)
    fd = rng.uniform(0.0, 2.0 * math.pi, n)
    p[:, 5] = fm * np.cos(fd)
    p[:, 6] = fm * np.sin(fd)
    p[:, 7] = rng.uniform(0.0, 2.0 * math.pi, n)
    p[:, 8:11] = rng.uniform(0.0, 1.0, (n, 3))
    return p


def target_gabor(H: int, W: int, seed: int, n_patches: int = 50) -> np.ndarray:
    """Target image [H,W,3]: 0.5 plus a sum of isotropic Gabor patches (Gaussian window times a
    signed cosine carrier) with random centre, width, wave vector, phase and colour amplitude."""
    rng = _rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64) + 0.5
    img = np.full((H, W, 3), 0.5)
    for _ in range(n_patches):
        x0, y0 = rng.uniform(0, W), rng.uniform(0, H)
        sig = rng.uniform(4.0, 24.0)
        k = rng.uniform(0.0, 0.25)
        ang = rng.uniform(0, 2 * math.pi)
        psi = rng.uniform(0, 2 * math.pi)
        amp = rng.uniform(-0.3, 0.3, 3)
        env = np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / (2 * sig * sig))
        car = np.cos(2 * math.pi * k * ((xx - x0) * math.cos(ang) + (yy - y0) * math.sin(ang)) + psi)
        img += (env * car)[..., None] * amp
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def target_noise_edges(H: int, W: int, seed: int, n_edges: int = 200) -> np.ndarray:
    """Photo-shaped target image [H,W,3]: per-channel noise with a 1/f amplitude spectrum plus
    random straight step edges of random colour contrast."""
    rng = _rng(seed)
    ky = np.fft.fftfreq(H)[:, None]
    kx = np.fft.fftfreq(W)[None, :]
    kk = np.sqrt(kx * kx + ky * ky)
    kk[0, 0] = 1.0
    img = np.zeros((H, W, 3))
    for ch in range(3):
        spec = (rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))) / kk
        spec[0, 0] = 0.0
        f = np.real(np.fft.ifft2(spec))
        img[..., ch] = f / (np.abs(f).max() + 1e-12) * 0.25
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64) + 0.5
    for _ in range(n_edges):
        x0, y0 = rng.uniform(0, W), rng.uniform(0, H)
        ang = rng.uniform(0, 2 * math.pi)
        side = (xx - x0) * math.cos(ang) + (yy - y0) * math.sin(ang) > 0
        img += side[..., None] * rng.uniform(-0.04, 0.04, 3)
    img += 0.5
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def scene3d(n: int, seed: int, scale_range=(0.002, 0.05), max_freq=40.0, extent=0.5) -> np.ndarray:
    """3D wavelet primitives: centres uniform in [-extent, extent]^3, anisotropic log-uniform
    scales, rotation quaternions normalize(N(0, I4)), frequency magnitude uniform in
    [0, max_freq] cycles/unit with a direction uniform on the sphere, phase uniform in
    [0, 2 pi), opacity sigmoid(N(0,1)), colours uniform in [0, 1]."""
    rng = _rng(seed)
    p = np.zeros((n, P3D), dtype=np.float32)
    p[:, 0:3] = rng.uniform(-extent, extent, (n, 3))
    p[:, 3:6] = _log_uniform(rng, scale_range[0], scale_range[1], (n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    p[:, 6:10] = q
    fm = rng.uniform(0.0, max_freq, n)
    fd = rng.standard_normal((n, 3))
    fd /= np.linalg.norm(fd, axis=1, keepdims=True)
    p[:, 10:13] = fm[:, None] * fd
    p[:, 13] = rng.uniform(0.0, 2.0 * math.pi, n)
    p[:, 14] = 1.0 / (1.0 + np.exp(-rng.standard_normal(n)))
    p[:, 15:18] = rng.uniform(0.0, 1.0, (n, 3))
    return p


P3D_SH = 68  # 3D record followed by the 15 higher spherical-harmonic coefficients per channel


def scene3d_sh(n: int, seed: int, degree: int = 3, sh_sigma: float = 0.15, **kw) -> np.ndarray:
    """3D primitives with spherical-harmonic colour: the scene3d record (its colour c serves as the
    degree-0 coefficients, drawn so that the constant part of the colour is uniform in [0, 1])
    followed by the coefficients of degrees 1..degree, N(0, sh_sigma) each (zero above degree)."""
    base = scene3d(n, seed, **kw)
    rng = _rng(seed + 7919)
    p = np.zeros((n, P3D_SH), dtype=np.float32)
    p[:, :P3D] = base
    y00 = 0.5 / math.sqrt(math.pi)
    p[:, 15:18] = (base[:, 15:18] - 0.5) / y00
    nk = (degree + 1) ** 2 - 1
    p[:, 20:20 + 3 * nk] = rng.normal(0.0, sh_sigma, (n, 3 * nk))
    return p


# layer shapes (out, in) of the deformation network (positional encoding of the centre with 10
# frequencies and of time with 6, 76 inputs zero-padded to 80; 8 layers of 256 with the encoding
# concatenated again at layer 5; 13 outputs)
MLP_SHAPES = [(256, 80)] + [(256, 256)] * 4 + [(256, 336)] + [(256, 256)] * 2 + [(13, 256)]


def deform_mlp_theta(seed: int, head_scale: float = 0.1) -> np.ndarray:
    """Packed float32 parameters of the deformation network: per layer W (out x in, row-major)
    then b, drawn U(-1/sqrt(in), 1/sqrt(in)) (the usual default of a linear layer); the output
    layer scaled by head_scale so that the deformations start small."""
    rng = _rng(seed)
    parts = []
    for li, (o, i) in enumerate(MLP_SHAPES):
        lim = 1.0 / math.sqrt(i)
        sc = head_scale if li == len(MLP_SHAPES) - 1 else 1.0
        parts.append(rng.uniform(-lim, lim, o * i) * sc)
        parts.append(rng.uniform(-lim, lim, o) * sc)
    return np.concatenate(parts).astype(np.float32)


def scene6d(n: int, seed: int, rate_sigma=0.05, **kw) -> np.ndarray:
    """6D primitives: a 3D scene plus per-primitive linear rates over a unit time span for the
    centre (v), frequency (df), phase (dphi) and log-scale (dlog_s), each N(0, rate_sigma)."""
    base = scene3d(n, seed, **kw)
    rng = _rng(seed + 7919)
    p = np.zeros((n, P6D), dtype=np.float32)
    p[:, :P3D] = base
    p[:, 20:30] = rng.normal(0.0, rate_sigma, (n, 10))
    return p


def time_stamps(n_stamps: int = 300) -> np.ndarray:
    return np.linspace(0.0, 1.0, n_stamps, dtype=np.float32)


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera [R|t] (3x4) for a camera at ``eye`` looking at ``target`` with OpenCV axes
    (x right, y down, z forward)."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    if np.linalg.norm(right) < 1e-6:
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ eye
    return np.concatenate([R, t[:, None]], axis=1)


def camera(viewmat34, H: int, W: int, fov_deg: float = 50.0, near: float = 0.2) -> np.ndarray:
    """Pack a pinhole camera [17] with a horizontal field of view ``fov_deg`` and the principal
    point at the image centre."""
    fx = 0.5 * W / math.tan(math.radians(fov_deg) * 0.5)
    cam = np.zeros(CAM_FLOATS, dtype=np.float32)
    cam[:12] = np.asarray(viewmat34, dtype=np.float64).reshape(12)
    cam[12] = fx
    cam[13] = fx
    cam[14] = 0.5 * W
    cam[15] = 0.5 * H
    cam[16] = near
    return cam


def sphere_cameras(k: int, H: int, W: int, seed: int, radius: float = 4.0, fov_deg: float = 50.0) -> np.ndarray:
    """``k`` cameras at seeded positions uniform on a sphere of ``radius`` around the origin,
    looking at the origin with world up +z.  Returns [k,17]."""
    rng = _rng(seed)
    cams = []
    for _ in range(k):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        cams.append(camera(look_at(radius * d), H, W, fov_deg))
    return np.stack(cams)


def upstream_grad(H: int, W: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded dL/dimage [H,W,3] for backward parity (standard normal times ``scale``)."""
    return (_rng(seed).standard_normal((H, W, 3)) * scale).astype(np.float32)


@dataclass(frozen=True)
class Config:
    name: str
    H: int
    W: int
    n: int
    seed: int


# The five workloads (one seed each: 1234 + index).
CFG0_2D_SMALL = Config("2d_256x256_n2000", 256, 256, 2000, 1234)
CFG1_2D_KODAK = Config("2d_768x512_n70000", 512, 768, 70000, 1235)
CFG2_5D = Config("5d_800x800_n300000", 800, 800, 300000, 1236)
CFG3_6D = Config("6d_1352x1014_n200000", 1014, 1352, 200000, 1237)


def cfg0_inputs():
    c = CFG0_2D_SMALL
    return scene2d(c.n, c.H, c.W, c.seed, (1.0, 16.0)), target_gabor(c.H, c.W, c.seed + 100)


def cfg1_inputs():
    c = CFG1_2D_KODAK
    return scene2d(c.n, c.H, c.W, c.seed, (0.5, 32.0)), target_noise_edges(c.H, c.W, c.seed + 100)


def cfg2_inputs(n_cams: int = 16):
    c = CFG2_5D
    return scene3d(c.n, c.seed), sphere_cameras(n_cams, c.H, c.W, c.seed + 100)


def cfg3_inputs(n_cams: int = 16):
    c = CFG3_6D
    return scene6d(c.n, c.seed), sphere_cameras(n_cams, c.H, c.W, c.seed + 100), time_stamps(300)


# ------------------------------------------------------------------------------------------------
# serving workload
# ------------------------------------------------------------------------------------------------

SERVING_SIZES = ((256, 256), (512, 512), (800, 800), (1080, 1920))  # (H, W)


@dataclass
class ServingScene:
    dims: int
    n: int
    seed: int
    params: dict      # size index -> [N,16] (2D, generated at that size) or the single [N,20] under key 0 (3D)
    cameras: dict     # size index -> [16,17] (3D only)


def serving_workload(n_scenes: int = 64, rate: float = 2000.0, seconds: float = 10.0, seed: int = 1238,
                     n_range=(10_000, 500_000), n_cams: int = 16):
    """Resident scenes and a Poisson request trace for the serving benchmark.

    Scenes: N log-uniform in n_range, 2D and 3D alternating (1:1); a 2D scene is drawn as the
    768x512 image-fitting scene (scales 0.5-32 px) at each serving size from one seed, a 3D scene
    as the 800x800 static scene with n_cams seeded cameras on the radius-4 sphere per size.
    Requests: Poisson arrivals at `rate` per second for `seconds`; each picks a scene, an image
    size uniformly from SERVING_SIZES and (3D) a camera.  Returns (scenes, requests) with requests
    an int/float array [R, 4]: arrival time (s), scene, size index, camera index."""
    rng = _rng(seed)
    scenes = []
    for k in range(n_scenes):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        s = seed * 1000 + k
        if k % 2 == 0:
            params = {i: scene2d(n, H, W, s, (0.5, 32.0)) for i, (H, W) in enumerate(SERVING_SIZES)}
            scenes.append(ServingScene(2, n, s, params, {}))
        else:
            cams = {i: sphere_cameras(n_cams, H, W, s + 1) for i, (H, W) in enumerate(SERVING_SIZES)}
            scenes.append(ServingScene(3, n, s, {0: scene3d(n, s)}, cams))
    gaps = rng.exponential(1.0 / rate, size=int(rate * seconds * 1.5) + 16)
    t = np.cumsum(gaps)
    t = t[t < seconds]
    m = len(t)
    req = np.zeros((m, 4), np.float64)
    req[:, 0] = t
    req[:, 1] = rng.integers(0, n_scenes, m)
    req[:, 2] = rng.integers(0, len(SERVING_SIZES), m)
    req[:, 3] = rng.integers(0, n_cams, m)
    return scenes, req

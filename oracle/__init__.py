"""Python access to the WIPES oracle (``wipes_oracle.c``): a brute-force binary64 CPU reference.

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU-baseline leg use
it; the product package never imports it.  It shares no code with the CUDA path: inputs come from
``synth`` (seeded generators) and results are compared against the library's outputs.

Every function takes numpy arrays in the record layouts documented in ``synth`` and returns
numpy arrays.  ``truncated=True`` applies the same per-pixel cutoff decision as the kernels
(binary32 footprint rule); ``truncated=False`` evaluates every primitive at every pixel.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wipes_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# opts vector layout shared by the 3D calls: cutoff, alpha_min, alpha_max, T_min, dilation, bg(3),
# frequency projection mode (0: phase gradient on the fronto-parallel plane, 1: literal J W f,
# 2: the oscillation integrated along the viewing ray, damped by kappa),
# spherical-harmonic colour degree (0: the record's RGB; 1..3: records of P3D_SH floats)
DEFAULT_OPTS_3D = np.array([3.0, 1.0 / 255.0, 0.99, 1e-4, 0.3, 0.0, 0.0, 0.0, 0.0, 0.0], dtype=np.float32)
P3D_SH = 68


def _opts3(opts):
    """The 10-entry options vector (shorter vectors get mode 0 and RGB colour)."""
    o = _f32(DEFAULT_OPTS_3D if opts is None else opts).ravel()
    return o if o.size == 10 else np.concatenate([o, np.zeros(10 - o.size, np.float32)])


def _stride3(opts):
    return P3D_SH if _opts3(opts)[9] else 20


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fused multiply-add contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                   "-fno-fast-math", "-o", _LIB + ".tmp", _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, f32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double
        lib.wo_footprints.argtypes = [i32, P, i64, P, i32, i32, f32, f32, P, P, P]
        lib.wo_tile_lists.argtypes = [i32, P, i64, P, i32, i32, f32, f32, P, P, i64]
        lib.wo_tile_lists.restype = i64
        lib.wo_render2d.argtypes = [P, i64, i32, i32, f32, i32, P, i64, i32, P]
        lib.wo_grad2d.argtypes = [P, i64, i32, i32, f32, i32, P, i32, P, P]
        lib.wo_render3d.argtypes = [P, i64, P, i32, i32, P, i32, P, i64, P, P, P, P]
        lib.wo_grad3d.argtypes = [P, i64, P, i32, i32, P, i32, P, P, P]
        lib.wo_project3d.argtypes = [P, i64, P, i32, i32, P, P]
        lib.wo_deform6d.argtypes = [P, i64, f64, P]
        lib.wo_deform6d_grad.argtypes = [P, i64, f64, P, P]
        lib.wo_cutoff_coverage.argtypes = [i32, P, i64, P, i32, i32, f32, f32, P]
        lib.wo_sh_basis.argtypes = [P, i64, P]
        lib.wo_alpha_decisions.argtypes = [P, i64, P, i32, i32, P, P, i64, P, P]
        lib.wo_rule_cos_sin.argtypes = [P, i64, P]
        _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _kind(dims, cov2d=0, sh=0):
    """Record kind of the C functions: 2 = 2D (RS), 3 = 3D, 4 = 2D with a Cholesky covariance,
    5 = 3D with spherical-harmonic colour (P3D_SH floats per record)."""
    if dims == 2:
        return 4 if cov2d else 2
    return 5 if sh else 3


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def footprints(dims, params, H, W, cam=None, cutoff=3.0, dilation=0.3, cov2d=0, sh=0):
    """binary32 footprint rule: (rec[N,8] = mx,my,l11,l21,l22,ex,ey,depth, rect[N,4] = u0,v0,u1,v1, valid[N]).
    cov2d=1: 2D records carry the Cholesky factor (l1, l2, l3) of Sigma instead of (s_x, s_y, theta)."""
    params = _f32(params)
    n = params.shape[0]
    rec = np.zeros((n, 8), np.float32)
    rect = np.zeros((n, 4), np.int32)
    valid = np.zeros(n, np.int32)
    camv = _f32(cam) if cam is not None else None
    _load().wo_footprints(_kind(dims, cov2d, sh), _ptr(params), n, _ptr(camv), H, W, cutoff, dilation, _ptr(rec), _ptr(rect),
                          _ptr(valid))
    return rec, rect, valid


def tile_lists(dims, params, H, W, cam=None, cutoff=3.0, dilation=0.3, cov2d=0, sh=0):
    """Sorted (tile, primitive) pairs: by tile, then camera depth (3D), then primitive index."""
    params = _f32(params)
    n = params.shape[0]
    camv = _f32(cam) if cam is not None else None
    lib = _load()
    kind = _kind(dims, cov2d, sh)
    total = lib.wo_tile_lists(kind, _ptr(params), n, _ptr(camv), H, W, cutoff, dilation, None, None, 0)
    tiles = np.zeros(max(total, 1), np.uint32)
    prims = np.zeros(max(total, 1), np.uint32)
    lib.wo_tile_lists(kind, _ptr(params), n, _ptr(camv), H, W, cutoff, dilation, _ptr(tiles), _ptr(prims), total)
    return tiles[:total], prims[:total]


def _pix(pixels):
    if pixels is None:
        return None, 0
    p = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    return p, p.shape[0]


def render2d(params, H, W, cutoff=3.0, truncated=True, pixels=None, cov2d=0):
    """Summed wavelet field, [H,W,3] (or [npix,3] at the given (u, v) pixels).  cov2d as in footprints."""
    params = _f32(params)
    pix, npix = _pix(pixels)
    out = np.zeros((npix if pix is not None else H * W, 3), np.float64)
    _load().wo_render2d(_ptr(params), params.shape[0], H, W, cutoff, int(truncated), _ptr(pix), npix, int(cov2d),
                        _ptr(out))
    return out if pix is not None else out.reshape(H, W, 3)


def grad2d(params, H, W, dldimg, cutoff=3.0, truncated=True, with_abs=False, cov2d=0):
    """dL/dparams [N,16] for L = sum(dldimg * C).  with_abs=True also returns, per parameter, the
    sum over pixels of |that pixel's contribution| (the scale of a summed gradient's rounding)."""
    params = _f32(params)
    g = _f32(dldimg)
    out = np.zeros((params.shape[0], 16), np.float64)
    gabs = np.zeros((params.shape[0], 16), np.float64) if with_abs else None
    _load().wo_grad2d(_ptr(params), params.shape[0], H, W, cutoff, int(truncated), _ptr(g), int(cov2d), _ptr(out),
                      _ptr(gabs))
    return (out, gabs) if with_abs else out


AMB_ALPHA_MIN, AMB_T_MIN, AMB_ALPHA_MAX = 1, 2, 4


def render3d(params, cam, H, W, opts=None, truncated=True, pixels=None):
    """Front-to-back blend.  Returns (C, T_final, n_contrib, ambiguous).  The threshold decisions
    are taken from the kernels' binary32 projected record (see alpha_decisions); ambiguous holds the
    AMB_* bits of decisions that lie within the kernels' error bound of their threshold: bits 0-1
    (alpha_min skip, T_min stop) can change the image, bit 2 (alpha_max clamp) only the gradient."""
    params = _f32(params)
    camv = _f32(cam)
    o = _opts3(opts)
    pix, npix = _pix(pixels)
    m = npix if pix is not None else H * W
    out = np.zeros((m, 3), np.float64)
    T = np.zeros(m, np.float64)
    nc = np.zeros(m, np.int32)
    amb = np.zeros(m, np.uint8)
    _load().wo_render3d(_ptr(params), params.shape[0], _ptr(camv), H, W, _ptr(o), int(truncated), _ptr(pix), npix,
                        _ptr(out), _ptr(T), _ptr(nc), _ptr(amb))
    if pix is None:
        return out.reshape(H, W, 3), T.reshape(H, W), nc.reshape(H, W), amb.reshape(H, W)
    return out, T, nc, amb


def grad3d(params, cam, H, W, dldimg, opts=None, truncated=True, with_abs=False):
    """dL/dparams [N,20] for L = sum(dldimg * C) (with_abs as in grad2d)."""
    params = _f32(params)
    camv = _f32(cam)
    o = _opts3(opts)
    g = _f32(dldimg)
    P = _stride3(opts)
    out = np.zeros((params.shape[0], P), np.float64)
    gabs = np.zeros((params.shape[0], P), np.float64) if with_abs else None
    _load().wo_grad3d(_ptr(params), params.shape[0], _ptr(camv), H, W, _ptr(o), int(truncated), _ptr(g), _ptr(out),
                      _ptr(gabs))
    return (out, gabs) if with_abs else out


def rule_cos_sin(theta):
    """The footprint rule's binary32 (cos, sin) of 2D rotation angles, taken as binary32 (the
    record's type): a fixed sequence of IEEE operations (Cody-Waite reduction, Taylor series; in
    binary32 up to |theta| = 2^16, in binary64 rounded once beyond).  Returns [n,2] float32."""
    th = np.ascontiguousarray(theta, dtype=np.float32).ravel()
    out = np.zeros((th.size, 2), np.float32)
    _load().wo_rule_cos_sin(_ptr(th), th.size, _ptr(out))
    return out


def alpha_decisions(params, cam, H, W, pairs, opts=None):
    """Threshold-decision values (Eq. 3's alpha_min skip, alpha_max clamp and T_min stop are taken
    from the kernels' binary32 projected record).  pairs[n,3] = (primitive, u, v).  Returns
    (rec[N,10] = mx, my, l11, l21, l22, f'x, f'y, phase in cycles, opacity and, under frequency map 2,
     the damping exponent kx (kappa = 2^kx; 0 otherwise) as binary32,
     out[n,3] = record alpha before the clamp (binary64), its kernel error bound, binary64-projection alpha)."""
    params = _f32(params)
    camv = _f32(cam)
    o = _opts3(opts)
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    rec = np.zeros((params.shape[0], 10), np.float32)
    out = np.zeros((pr.shape[0], 3), np.float64)
    _load().wo_alpha_decisions(_ptr(params), params.shape[0], _ptr(camv), H, W, _ptr(o), _ptr(pr), pr.shape[0],
                               _ptr(rec), _ptr(out))
    return rec, out


def project3d(params, cam, H, W, opts=None):
    """[N,16]: valid, tz, mu'x, mu'y, Sigma'00, Sigma'01, Sigma'11, f'x, f'y, phi, opacity, c(3), kappa, 0
    (kappa: the damping of the oscillation, 1 except under frequency map 2)."""
    params = _f32(params)
    camv = _f32(cam)
    o = _opts3(opts)
    out = np.zeros((params.shape[0], 16), np.float64)
    _load().wo_project3d(_ptr(params), params.shape[0], _ptr(camv), H, W, _ptr(o), _ptr(out))
    return out


def deform6d(params6, t):
    """Deformed 3D records [N,20] (binary64) at time t."""
    p = _f32(params6)
    out = np.zeros((p.shape[0], 20), np.float64)
    _load().wo_deform6d(_ptr(p), p.shape[0], float(t), _ptr(out))
    return out


def deform6d_grad(params6, t, g3):
    """dL/d(record6) [N,32] from dL/d(deformed record) [N,20]."""
    p = _f32(params6)
    g = np.ascontiguousarray(g3, dtype=np.float64)
    out = np.zeros((p.shape[0], 32), np.float64)
    _load().wo_deform6d_grad(_ptr(p), p.shape[0], float(t), _ptr(g), _ptr(out))
    return out


def sort_pairs(keys, vals, key_bits):
    """The sort of the path (Sec. 1: the GPU sort that orders the tile lists, and the 3D depth
    sort): (key, value) pairs of 32-bit words ordered stably by the low key_bits bits of the key,
    pairs with equal low bits in input order.  Returns the sorted (keys, vals) as uint32."""
    k = np.ascontiguousarray(keys).view(np.uint32).ravel()
    v = np.ascontiguousarray(vals).view(np.uint32).ravel()
    mask = np.uint32(0xFFFFFFFF) if key_bits >= 32 else np.uint32((1 << key_bits) - 1)
    order = np.argsort(k & mask, kind="stable")
    return k[order], v[order]


def sh_basis(dirs):
    """Real spherical harmonics up to degree 3 (16 per direction) at unit vectors dirs[n,3]."""
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((d.shape[0], 16), np.float64)
    _load().wo_sh_basis(_ptr(d), d.shape[0], _ptr(out))
    return out


def cutoff_coverage(dims, params, H, W, cam=None, cutoff=3.0, dilation=0.3, cov2d=0, sh=0):
    """(pairs inside the cutoff, of those outside the covered pixel range, pixels in the ranges,
    cutoff pairs that the tile ellipse test would drop)."""
    params = _f32(params)
    camv = _f32(cam) if cam is not None else None
    counts = np.zeros(4, np.int64)
    _load().wo_cutoff_coverage(_kind(dims, cov2d, sh), _ptr(params), params.shape[0], _ptr(camv), H, W, cutoff, dilation,
                               _ptr(counts))
    return int(counts[0]), int(counts[1]), int(counts[2]), int(counts[3])

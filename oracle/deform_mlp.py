"""Oracle of the 6D deformation field (Sec. 4.3): (dx, df, dSigma) = F_theta(gamma(x), gamma(t)).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): used by the tests, the smoke check and the
benchmark's CPU-baseline leg; the product package never imports it and shares no code with it.

The paper defines the deformation only through an MLP F_theta with positional encoding gamma
(Sec. 4.3) and keeps everything else as in Deformable 3D Gaussians.  The network read here:
  gamma(p) = (p, sin(2^k p), cos(2^k p) for k = 0..L-1) per coordinate, L = 10 for the centre x,
             L = 6 for the time t: 3 + 60 + 1 + 12 = 76 inputs (zero-padded to 80);
  h_0 = relu(W_0 gamma + b_0), h_l = relu(W_l h_{l-1} + b_l) for l = 1..7, except that layer 5
  takes the concatenation (gamma, h_4) (the skip connection), width 256;
  d = W_8 h_7 + b_8: 13 outputs, dx (3), dq (4), dlog s (3), df (3).
The deformed 3D record: mu + dx, q + dq, s * exp(dlog s), f + df; phase, opacity, colour kept.

Precision.  The device path runs the products in bfloat16 with fp32 accumulation.  ``bf16=True``
reproduces its roundings: every matrix-product operand (encoding, weights, hidden activations,
upstream gradients) is rounded to bfloat16 where the device rounds it; biases, the outputs and the
encoding's gradient (the skip layer's and layer 0's products summed unrounded) are not rounded,
and everything else is binary64.  ``bf16=False`` is the exact binary64 network, against which central differences pin
the gradient.  theta is the packed float32 parameter vector: for each layer W (out x in,
row-major) then b (out).
"""
from __future__ import annotations

import numpy as np

L_X, L_T = 10, 6
IN = 3 * (1 + 2 * L_X) + 1 * (1 + 2 * L_T)  # 76
IN_PAD = 80
WIDTH = 256
N_HIDDEN = 8
SKIP = 5  # layer 5 takes (gamma, h_4)
OUT = 13
# (out, in) of every linear layer, in order
SHAPES = [(WIDTH, IN_PAD)] + [(WIDTH, WIDTH)] * 4 + [(WIDTH, IN_PAD + WIDTH)] + [(WIDTH, WIDTH)] * 2 + [(OUT, WIDTH)]
# relative margin of the ReLU decisions: fp32 accumulation of K <= 336 products rounds by a few
# 2^-24 of the sum of |terms| in practice (the worst case is K 2^-24 = 2e-5)
AMB_REL = 4e-6


def theta_size() -> int:
    return sum(o * i + o for o, i in SHAPES)


def unpack(theta):
    """[(W, b)] per layer, binary64 views of the packed float32 vector."""
    t = np.asarray(theta, np.float32).astype(np.float64)
    out, k = [], 0
    for o, i in SHAPES:
        W = t[k:k + o * i].reshape(o, i)
        k += o * i
        b = t[k:k + o]
        k += o
        out.append((W, b))
    assert k == t.size
    return out


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), through float32, returned as float64."""
    f = np.ascontiguousarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return np.where(np.isfinite(f), out, f).astype(np.float64)


def encode(mu, t):
    """gamma(x) and gamma(t) per primitive: [N, IN_PAD], binary64."""
    mu = np.asarray(mu, np.float32).astype(np.float64)
    n = mu.shape[0]
    g = np.zeros((n, IN_PAD))
    g[:, 0:3] = mu
    for k in range(L_X):
        g[:, 3 + 6 * k: 6 + 6 * k] = np.sin(2.0 ** k * mu)
        g[:, 6 + 6 * k: 9 + 6 * k] = np.cos(2.0 ** k * mu)
    base = 3 + 6 * L_X
    tt = float(np.float32(t))
    g[:, base] = tt
    for k in range(L_T):
        g[:, base + 1 + 2 * k] = np.sin(2.0 ** k * tt)
        g[:, base + 2 + 2 * k] = np.cos(2.0 ** k * tt)
    return g


def forward(mu, t, theta, bf16_ops=True):
    """Network outputs d [N,13] and the cache the backward needs."""
    R = bf16 if bf16_ops else (lambda a: a)
    layers = unpack(theta)
    g = R(encode(mu, t))
    hs, x = [], g
    amb = np.zeros(g.shape[0], bool)
    for l in range(N_HIDDEN):
        W, b = layers[l]
        if l == SKIP:
            x = np.concatenate([g, hs[4]], axis=1)
        z = x @ R(W).T + b
        # a pre-activation this close to 0 (relative to the magnitude of its terms) can take the
        # ReLU either way under a different summation order
        amb |= (np.abs(z) <= AMB_REL * (np.abs(x) @ np.abs(R(W)).T + np.abs(b))).any(axis=1)
        h = R(np.maximum(z, 0.0))
        hs.append(h)
        x = h
    W, b = layers[N_HIDDEN]
    d = x @ R(W).T + b
    return d, {"g": g, "hs": hs, "layers": layers, "R": R, "amb_rows": amb}


def apply(params3, d):
    """The deformed 3D records [N,20] from canonical records and network outputs (binary64)."""
    p = np.asarray(params3, np.float32).astype(np.float64).copy()
    p[:, 0:3] += d[:, 0:3]
    p[:, 6:10] += d[:, 3:7]
    p[:, 3:6] *= np.exp(d[:, 7:10])
    p[:, 10:13] += d[:, 10:13]
    return p


def apply_backward(params3, d, g_out):
    """(dL/dd [N,13], dL/dparams3 through the direct terms) given dL/d(deformed record) [N,20]."""
    p = np.asarray(params3, np.float32).astype(np.float64)
    g = np.asarray(g_out, np.float64)
    es = np.exp(d[:, 7:10])
    gd = np.zeros((p.shape[0], OUT))
    gd[:, 0:3] = g[:, 0:3]
    gd[:, 3:7] = g[:, 6:10]
    gd[:, 7:10] = g[:, 3:6] * p[:, 3:6] * es
    gd[:, 10:13] = g[:, 10:13]
    gp = g.copy()
    gp[:, 3:6] = g[:, 3:6] * es
    return gd, gp


def _max_row_term(a, x, chunk=64):
    """max over rows r of |a[r, u]| |x[r, i]| for every (u, i): the largest single-row term."""
    out = np.zeros((a.shape[1], x.shape[1]))
    aa, xx = np.abs(a), np.abs(x)
    for r0 in range(0, a.shape[0], chunk):
        out = np.maximum(out, (aa[r0:r0 + chunk, :, None] * xx[r0:r0 + chunk, None, :]).max(axis=0))
    return out


def backward(mu, cache, gd, with_abs=False):
    """(dL/dtheta packed [P], dL/dmu [N,3]) of L given dL/dd [N,13], for the cache of forward().
    with_abs: also the packed sums of |products| (|dz|^T |x| and sum |dz|), the scale of each entry,
    and the packed largest single-row term (max over rows of |dh| |x| and |dh|, dh taken before the
    ReLU mask): the most one row can change an entry when its ReLU decision goes the other way."""
    R, layers, hs, g = cache["R"], cache["layers"], cache["hs"], cache["g"]
    grads = [None] * len(layers)
    absg = [None] * len(layers)
    maxg = [None] * len(layers)
    dy = R(gd)
    W, _ = layers[N_HIDDEN]
    grads[N_HIDDEN] = (dy.T @ hs[-1], dy.sum(0))
    absg[N_HIDDEN] = (np.abs(dy).T @ np.abs(hs[-1]), np.abs(dy).sum(0))
    if with_abs:
        maxg[N_HIDDEN] = (_max_row_term(dy, hs[-1]), np.abs(dy).max(0))
    dh = R(dy @ R(W))
    dg = np.zeros_like(g)
    for l in range(N_HIDDEN - 1, -1, -1):
        W, _ = layers[l]
        dz = np.where(hs[l] > 0.0, dh, 0.0)
        x = np.concatenate([g, hs[4]], axis=1) if l == SKIP else (g if l == 0 else hs[l - 1])
        grads[l] = (dz.T @ x, dz.sum(0))
        absg[l] = (np.abs(dz).T @ np.abs(x), np.abs(dz).sum(0))
        if with_abs:
            maxg[l] = (_max_row_term(dh, x), np.abs(dh).max(0))
        dx = dz @ R(W)
        if l == SKIP:
            dg += dx[:, :IN_PAD]
            dh = R(dx[:, IN_PAD:])
        elif l == 0:
            dg += dx
        else:
            dh = R(dx)
    # gamma(x): d/dx of (x, sin(2^k x), cos(2^k x))
    m = np.asarray(mu, np.float32).astype(np.float64)
    dmu = dg[:, 0:3].copy()
    for k in range(L_X):
        f = 2.0 ** k
        dmu += dg[:, 3 + 6 * k: 6 + 6 * k] * f * np.cos(f * m)
        dmu -= dg[:, 6 + 6 * k: 9 + 6 * k] * f * np.sin(f * m)
    packed = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    if with_abs:
        pack = lambda parts: np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in parts])  # noqa: E731
        return packed, dmu, pack(absg), pack(maxg)
    return packed, dmu


def deform(params3, t, theta, bf16_ops=True):
    """Deformed records [N,20] and the network outputs."""
    d, _ = forward(np.asarray(params3)[:, 0:3], t, theta, bf16_ops)
    return apply(params3, d), d


def deform_grad(params3, t, theta, g_out, bf16_ops=True):
    """(dL/dtheta, dL/dparams3 [N,20]) of L = sum(g_out * deformed record)."""
    p = np.asarray(params3, np.float32)
    d, cache = forward(p[:, 0:3], t, theta, bf16_ops)
    gd, gp = apply_backward(p, d, g_out)
    dtheta, dmu = backward(p[:, 0:3], cache, gd)
    gp[:, 0:3] += dmu
    return dtheta, gp

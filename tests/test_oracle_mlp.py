"""Pins of the deformation-network oracle (Sec. 4.3: (dx, df, dSigma) = F_theta(gamma(x), gamma(t)))
against facts that do not come from the oracle itself."""
import math

import numpy as np
import pytest

import synth
from oracle import deform_mlp as M


def test_layer_shapes_and_parameter_count():
    assert [tuple(s) for s in synth.MLP_SHAPES] == [tuple(s) for s in M.SHAPES]
    assert M.IN == 76 and synth.deform_mlp_theta(1).size == M.theta_size()


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=10000) * 10.0 ** rng.integers(-8, 8, 10000), [0.0, -0.0, 1.0, 3.0e38]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), ref)


def test_positional_encoding_invariants():
    """gamma keeps the input, pairs (sin, cos) lie on the unit circle, and consecutive bands double
    the frequency: sin(2^(k+1) x) = 2 sin(2^k x) cos(2^k x)."""
    rng = np.random.default_rng(2)
    mu = rng.uniform(-0.5, 0.5, (40, 3)).astype(np.float32)
    t = 0.37
    g = M.encode(mu, t)
    np.testing.assert_array_equal(g[:, 0:3], mu.astype(np.float64))
    assert g[0, 63] == pytest.approx(np.float32(t))
    assert np.all(g[:, 76:] == 0)
    for k in range(M.L_X):
        s, c = g[:, 3 + 6 * k: 6 + 6 * k], g[:, 6 + 6 * k: 9 + 6 * k]
        np.testing.assert_allclose(s * s + c * c, 1.0, atol=1e-14)
        if k + 1 < M.L_X:
            np.testing.assert_allclose(g[:, 9 + 6 * k: 12 + 6 * k], 2 * s * c, atol=1e-13)
    for k in range(M.L_T):
        s, c = g[:, 64 + 2 * k], g[:, 65 + 2 * k]
        np.testing.assert_allclose(s * s + c * c, 1.0, atol=1e-14)
        if k + 1 < M.L_T:
            np.testing.assert_allclose(g[:, 66 + 2 * k], 2 * s * c, atol=1e-13)
    assert g[0, 65] == pytest.approx(math.cos(np.float32(t)))


def test_zero_weights_give_the_output_bias():
    theta = np.zeros(M.theta_size(), np.float32)
    theta[-13:] = np.arange(13, dtype=np.float32) * 0.25
    mu = np.random.default_rng(3).uniform(-1, 1, (7, 3)).astype(np.float32)
    for exact in (True, False):
        d, _ = M.forward(mu, 0.5, theta, bf16_ops=not exact)
        np.testing.assert_array_equal(d, np.broadcast_to(np.arange(13) * 0.25, (7, 13)))


def test_skip_connection_takes_the_encoding_first():
    """With layers 0..4 zero, layer 5 sees (gamma, h_4 = 0): a unit of layer 5 that reads the first
    encoding channel (the centre's x), passed on unchanged by layers 6, 7 and the head, outputs x
    for x > 0."""
    theta = np.zeros(M.theta_size(), np.float32)
    offs, k = [], 0
    for o, i in M.SHAPES:
        offs.append(k)
        k += o * i + o
    theta[offs[5] + 0 * 336 + 0] = 1.0      # layer 5, unit 0 <- input channel 0 (gamma first)
    theta[offs[6] + 0 * 256 + 0] = 1.0      # layer 6, unit 0 <- unit 0
    theta[offs[7] + 0 * 256 + 0] = 1.0
    theta[offs[8] + 0 * 256 + 0] = 1.0      # output 0 <- unit 0
    mu = np.array([[0.25, -0.1, 0.3], [0.5, 0.2, -0.4], [-0.3, 0.1, 0.1]], np.float32)
    d, _ = M.forward(mu, 0.0, theta, bf16_ops=False)
    np.testing.assert_allclose(d[:, 0], np.maximum(mu[:, 0], 0.0), rtol=1e-15)
    assert np.all(d[:, 1:] == 0)


def test_deform_apply_closed_form():
    p = synth.scene3d(5, 4)
    d = np.random.default_rng(5).normal(0, 0.1, (5, 13))
    q = M.apply(p, d)
    pp = p.astype(np.float64)
    np.testing.assert_allclose(q[:, 0:3], pp[:, 0:3] + d[:, 0:3])
    np.testing.assert_allclose(q[:, 3:6], pp[:, 3:6] * np.exp(d[:, 7:10]))
    np.testing.assert_allclose(q[:, 6:10], pp[:, 6:10] + d[:, 3:7])
    np.testing.assert_allclose(q[:, 10:13], pp[:, 10:13] + d[:, 10:13])
    np.testing.assert_array_equal(q[:, 13:], pp[:, 13:])


def _fd(f, x0, h):
    """Central difference of f at the float32 value x0 with float32-representable steps, and
    whether the two one-sided differences agree (no ReLU kink inside the step)."""
    xp, xm = np.float32(x0 + h), np.float32(x0 - h)
    fp, f0, fm = f(xp), f(np.float32(x0)), f(xm)
    central = (fp - fm) / (float(xp) - float(xm))
    right = (fp - f0) / (float(xp) - float(x0))
    left = (f0 - fm) / (float(x0) - float(xm))
    return central, abs(right - left) <= 1e-3 * max(abs(central), 1e-2)


def test_network_gradient_matches_central_differences():
    """dL/dtheta (sampled entries of every layer) and dL/dparams3 of L = sum(g * deformed record),
    exact binary64 network, against central differences.  The network is piecewise smooth (ReLU):
    an entry whose step straddles a kink (the one-sided differences disagree) is not compared, and
    most entries must be."""
    rng = np.random.default_rng(6)
    p = synth.scene3d(6, 7, extent=0.4)
    theta = synth.deform_mlp_theta(8, head_scale=0.5)
    g = rng.normal(size=(6, 20))
    t = 0.3

    def L(th, pp):
        q, _ = M.deform(pp, t, th, bf16_ops=False)
        return float((q * g).sum())

    dth, dp = M.deform_grad(p, t, theta, g, bf16_ops=False)
    offs, k = [], 0
    for o, i in M.SHAPES:
        offs.append(k)
        k += o * i + o
    idx = []
    for li, (o, i) in enumerate(M.SHAPES):
        idx += list(rng.integers(offs[li], offs[li] + o * i + o, 6))
    checked = 0
    for j in idx:
        def f(v, j=j):
            th = theta.copy()
            th[j] = v
            return L(th, p)

        fd, smooth = _fd(f, theta[j], max(abs(float(theta[j])), 0.05) * 2.0 ** -16)
        if not smooth:
            continue
        checked += 1
        assert abs(dth[j] - fd) <= 2e-4 * abs(fd) + 1e-6 * np.abs(dth).max(), (j, dth[j], fd)
    assert checked >= 0.8 * len(idx)
    checked = total = 0
    for i in range(6):
        for c in [0, 1, 2, 3, 4, 5, 6, 9, 10, 12, 13, 14, 15]:
            def f(v, i=i, c=c):
                pp = p.copy()
                pp[i, c] = v
                return L(theta, pp)

            total += 1
            fd, smooth = _fd(f, p[i, c], max(abs(float(p[i, c])), 0.05) * 2.0 ** -18)
            if not smooth:
                continue
            checked += 1
            assert abs(dp[i, c] - fd) <= 2e-4 * abs(fd) + 1e-6 * np.abs(dp).max(), (i, c, dp[i, c], fd)
    assert checked >= 0.8 * total


def test_bf16_network_stays_near_the_exact_one():
    """The roundings of the device's bfloat16 products move the outputs by a small fraction of
    their scale (the bound the device parity test builds on)."""
    p = synth.scene3d(2000, 9)
    theta = synth.deform_mlp_theta(10)
    d64, _ = M.forward(p[:, 0:3], 0.6, theta, bf16_ops=False)
    d16, _ = M.forward(p[:, 0:3], 0.6, theta, bf16_ops=True)
    scale = np.abs(d64).max(axis=0)
    assert np.all(np.abs(d16 - d64).max(axis=0) <= 0.05 * scale)

"""Device parity of the 6D deformation network (Sec. 4.3, F_theta(gamma(x), gamma(t))) against the
oracle with the device's bfloat16 operand roundings emulated.

Tolerance.  Both sides round the same operands to bfloat16 at the same points; they differ by the
accumulation (fp32 in the tensor cores, binary64 in the oracle, ~1e-6 relative) and, where an fp32
value falls within that distance of a bfloat16 rounding boundary, by one bfloat16 unit (2^-8
relative) of that activation, which propagates.  Measured on the device: output errors stay below
0.22 2^-8 A (A the sum of |terms| of the output layer, median 1e-4 2^-8 A), so outputs are checked
at 2^-9 A; parameter-gradient errors exceed 2^-10 of their |products| sum for at most 0.2 % of
the entries, so every entry is checked at 2^-8 of that sum (plus the single-row term below) and
99.9 % of them without the single-row term.

A ReLU decision close to 0 can go either way: under the accumulation difference directly, or
after a bfloat16 flip upstream has moved its pre-activation by a unit of that flip.  It then moves
a whole row's term of the gradient (|dh| |x| before the mask, not a rounding of it).  The oracle
flags the rows with a pre-activation within the accumulation error of 0, and the backward checks
give them a zero upstream gradient; the rare decisions moved by upstream flips are covered by
adding twice the largest single-row term (measured at most 0.7 of it) to the parameter
gradients' tolerance, and by requiring the centre gradient of at least 99.5 % of the rows to
agree within 2^-10 of its scale.
"""
import numpy as np
import pytest

import synth
from helpers import lib_ready, torch_cuda
from oracle import deform_mlp as M

pytestmark = pytest.mark.gpu


def _setup(N, seed, t):
    torch = torch_cuda()
    w = lib_ready()
    p = synth.scene3d(N, seed)
    theta = synth.deform_mlp_theta(seed + 1, head_scale=0.2)
    P = torch.from_numpy(p).cuda()
    TH = torch.from_numpy(theta).cuda()
    st = w.State(w.Context.get(0))
    out = w.deform_mlp(P, t, TH, state=st)
    torch.cuda.synchronize()
    return torch, w, p, theta, P, TH, st, out


def _deltas(p, q):
    """Network outputs recovered from canonical and deformed records."""
    p = p.astype(np.float64)
    q = q.astype(np.float64)
    d = np.zeros((p.shape[0], 13))
    d[:, 0:3] = q[:, 0:3] - p[:, 0:3]
    d[:, 3:7] = q[:, 6:10] - p[:, 6:10]
    d[:, 7:10] = np.log(q[:, 3:6] / p[:, 3:6])
    d[:, 10:13] = q[:, 10:13] - p[:, 10:13]
    return d


@pytest.mark.parametrize("N,seed,t", [(3000, 61, 0.37), (777, 62, 0.9), (1, 63, 0.0)])
def test_deform_mlp_forward_matches_oracle(N, seed, t):
    torch, w, p, theta, P, TH, st, out = _setup(N, seed, t)
    q = out.cpu().numpy()
    d_ref, cache = M.forward(p[:, 0:3], t, theta)
    W8, b8 = cache["layers"][-1]
    A = np.abs(cache["hs"][-1]) @ np.abs(M.bf16(W8)).T + np.abs(b8)
    d_dev = _deltas(p, q)
    # recovering d from fp32 records costs up to an ulp of the record entries
    rec_ulp = np.zeros_like(d_dev)
    rec_ulp[:, 0:3] = np.spacing(np.abs(q[:, 0:3]).astype(np.float32))
    rec_ulp[:, 3:7] = np.spacing(np.abs(q[:, 6:10]).astype(np.float32))
    rec_ulp[:, 7:10] = 2e-7
    rec_ulp[:, 10:13] = np.spacing(np.abs(q[:, 10:13]).astype(np.float32))
    tol = 2.0 ** -9 * A + 1e-6 + 2 * rec_ulp
    err = np.abs(d_dev - d_ref)
    assert np.all(err <= tol), (err / tol).max()
    # the fields the network does not touch are copied
    np.testing.assert_array_equal(q[:, 13:], p[:, 13:])
    # the deformation is not trivially small
    assert np.abs(d_ref).max() > 1e-3


@pytest.mark.parametrize("N,seed,t", [(2500, 64, 0.42), (300, 65, 0.05)])
def test_deform_mlp_backward_matches_oracle(N, seed, t):
    torch, w, p, theta, P, TH, st, out = _setup(N, seed, t)
    g = np.random.default_rng(seed).normal(size=(N, 20)).astype(np.float32)
    d, cache = M.forward(p[:, 0:3], t, theta)
    assert cache["amb_rows"].mean() < 0.1
    g[cache["amb_rows"]] = 0.0
    gth, gp = w.deform_mlp_backward(st, P, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    gd, gp_ref = M.apply_backward(p, d, g)
    gth_ref, dmu, gabs, gmax = M.backward(p[:, 0:3], cache, gd, with_abs=True)
    gp_ref[:, 0:3] += dmu
    err = np.abs(gth.cpu().numpy() - gth_ref)
    tol = 2.0 ** -8 * gabs + 2.0 * gmax + 1e-6 * np.abs(gth_ref).max()
    assert np.all(err <= tol), (err / tol).max()
    # the same bound without the single-row term holds for nearly every entry
    assert np.mean(err > 2.0 ** -8 * gabs + 1e-6 * np.abs(gth_ref).max()) < 1e-3
    gp_dev = gp.cpu().numpy()
    # direct terms: rotation, frequency, phase, opacity and colour pass dL/d(deformed) through
    cols = list(range(6, 20))
    np.testing.assert_allclose(gp_dev[:, cols], gp_ref[:, cols], rtol=1e-6, atol=1e-7)
    # the scale's is dL/ds' exp(dlog s): exp of a network output, within the forward bound
    W8, b8 = cache["layers"][-1]
    A = np.abs(cache["hs"][-1]) @ np.abs(M.bf16(W8)).T + np.abs(b8)
    tol_s = np.abs(gp_ref[:, 3:6]) * (2.0 ** -9 * A[:, 7:10] + 1e-6) + 1e-7
    assert np.all(np.abs(gp_dev[:, 3:6] - gp_ref[:, 3:6]) <= tol_s)
    # the centre: the direct term plus the network's gradient through gamma(x)
    scale = np.abs(gp_ref[:, 0:3]).max(axis=0)
    rows_ok = np.all(np.abs(gp_dev[:, 0:3] - gp_ref[:, 0:3]) <= 2.0 ** -10 * scale, axis=1)
    assert rows_ok.mean() >= 0.995


def test_deform_mlp_backward_accumulates():
    torch, w, p, theta, P, TH, st, out = _setup(500, 66, 0.3)
    g = torch.from_numpy(np.random.default_rng(7).normal(size=(500, 20)).astype(np.float32)).cuda()
    a_th, a_p = w.deform_mlp_backward(st, P, g)
    b_th, b_p = w.deform_mlp_backward(st, P, g, grad_theta=a_th.clone(), grad_params3=a_p.clone(), accumulate=True)
    torch.cuda.synchronize()
    np.testing.assert_allclose(b_th.cpu().numpy(), 2 * a_th.cpu().numpy(), rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(b_p.cpu().numpy(), 2 * a_p.cpu().numpy(), rtol=1e-6, atol=1e-7)


def test_deform_field_autograd_through_render():
    """render3d(deform_field(params3, theta, t)) backpropagates through both Functions to the same
    gradients as the direct calls."""
    torch, w, p, theta, P, TH, st, out = _setup(800, 67, 0.6)
    H, W = 48, 64
    cam = synth.sphere_cameras(1, H, W, 68)[0]
    Pg = P.clone().requires_grad_(True)
    THg = TH.clone().requires_grad_(True)
    img = w.render3d(w.deform_field(Pg, THg, 0.6), cam, H, W)
    gimg = torch.from_numpy(synth.upstream_grad(H, W, 69)).cuda()
    (img * gimg).sum().backward()
    st2 = w.State(w.Context.get(0))
    q = w.deform_mlp(P, 0.6, TH, state=st2)
    st3 = w.State(w.Context.get(0))
    img2 = w.forward3d(q, cam, H, W, state=st3)
    g3 = w.backward(st3, q, gimg)
    gth, gp = w.deform_mlp_backward(st2, P, g3)
    torch.cuda.synchronize()
    assert torch.equal(img, img2)
    np.testing.assert_allclose(THg.grad.cpu().numpy(), gth.cpu().numpy(), rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(Pg.grad.cpu().numpy(), gp.cpu().numpy(), rtol=1e-4, atol=1e-6)

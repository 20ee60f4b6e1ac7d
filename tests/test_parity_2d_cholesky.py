"""Device parity of the 2D path with the Cholesky covariance record (GaussianImage's second
construction, Sec. 5.1: Sigma = L L^T) against the binary64 oracle: tile lists bit-exact, forward
within 1e-4, gradients within 1e-3 relative (with the summation-scale term)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import FWD_ATOL, grad_close, lib_ready, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    # (N, H, W, scale range, seed): several tiles with ragged edges, elongated primitives, one tile
    (400, 70, 100, (1.0, 16.0), 31),
    (1500, 200, 232, (0.5, 32.0), 32),
    (64, 16, 16, (0.5, 8.0), 33),
]


def _render(w, torch, p, H, W):
    params = torch.from_numpy(p).cuda()
    st = w.Context.get(0).acquire_state()
    img = w.forward2d(params, H, W, opts=w.make_opts(2, cov2d=1), state=st)
    torch.cuda.synchronize()
    return params, st, img


@pytest.mark.parametrize("N,H,W,scale,seed", CASES)
def test_cholesky_tile_lists_bit_exact(N, H, W, scale, seed):
    torch = torch_cuda()
    w = lib_ready()
    p = synth.scene2d_cholesky(N, H, W, seed, scale)
    _, st, _ = _render(w, torch, p, H, W)
    tiles, prims, _ = st.lists()
    ot, op = oracle.tile_lists(2, p, H, W, cov2d=1)
    assert np.array_equal(tiles.cpu().numpy().view(np.uint32), ot)
    assert np.array_equal(prims.cpu().numpy().view(np.uint32), op)


@pytest.mark.parametrize("N,H,W,scale,seed", CASES)
def test_cholesky_forward_matches_oracle(N, H, W, scale, seed):
    torch = torch_cuda()
    w = lib_ready()
    p = synth.scene2d_cholesky(N, H, W, seed, scale)
    _, _, img = _render(w, torch, p, H, W)
    ref = oracle.render2d(p, H, W, cov2d=1)
    err = np.abs(img.cpu().numpy().astype(np.float64) - ref)
    assert err.max() <= FWD_ATOL, (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("N,H,W,scale,seed", CASES)
def test_cholesky_backward_matches_oracle(N, H, W, scale, seed):
    torch = torch_cuda()
    w = lib_ready()
    p = synth.scene2d_cholesky(N, H, W, seed, scale)
    g = synth.upstream_grad(H, W, seed + 77)
    params, st, _ = _render(w, torch, p, H, W)
    grad = w.backward(st, params, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    ref, gabs = oracle.grad2d(p, H, W, g, with_abs=True, cov2d=1)
    ok, worst, idx = grad_close(grad.cpu().numpy(), ref, gabs, cols=list(range(11)))
    assert ok, (worst, idx)
    assert np.all(grad.cpu().numpy()[:, 11:] == 0)


def test_cholesky_option_is_validated():
    torch = torch_cuda()
    w = lib_ready()
    from paper_2508_12615_gb300 import _abi

    p = torch.from_numpy(synth.scene2d_cholesky(10, 16, 16, 34)).cuda()
    with pytest.raises(_abi.WipesError) as e:
        w.forward2d(p, 16, 16, opts=w.make_opts(2, cov2d=2))
    assert e.value.status == 1

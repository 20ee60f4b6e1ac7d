"""Device parity of the 2D path (summed wavelet field, Eq. 4 with the wavelet of Eq. 5) against the
binary64 oracle: tile lists bit-exact, forward within 1e-4, gradients within 1e-3 relative."""
import numpy as np
import pytest

import oracle
import synth
from helpers import FWD_ATOL, grad_close, lib_ready, sample_pixels, torch_cuda

pytestmark = pytest.mark.gpu


def _gpu_forward(w, torch, p, H, W):
    params = torch.from_numpy(p).cuda()
    st = w.Context.get(0).acquire_state()
    img = w.forward2d(params, H, W, state=st)
    torch.cuda.synchronize()
    return params, st, img


CASES = [
    # (N, H, W, scale range, seed): several tiles and ragged right/bottom edges
    (300, 70, 100, (1.0, 16.0), 1),
    (2000, 256, 256, (1.0, 16.0), 1234),  # the 256x256 workload
    (500, 37, 129, (0.5, 32.0), 3),
    (64, 16, 16, (0.5, 8.0), 4),           # a single tile
    (200, 1, 300, (0.5, 4.0), 5),          # one row
    (200, 300, 1, (0.5, 4.0), 6),          # one column
]


@pytest.mark.parametrize("N,H,W,scale,seed", CASES)
def test_tile_lists_bit_exact(N, H, W, scale, seed):
    torch = torch_cuda()
    w = lib_ready()
    p = synth.scene2d(N, H, W, seed, scale)
    _, st, _ = _gpu_forward(w, torch, p, H, W)
    tiles, prims, ranges = st.lists()
    ot, op = oracle.tile_lists(2, p, H, W)
    assert np.array_equal(tiles.cpu().numpy().view(np.uint32), ot)
    assert np.array_equal(prims.cpu().numpy().view(np.uint32), op)
    r = ranges.cpu().numpy()
    tx = (W + 15) // 16
    for t in range(r.shape[0]):
        sel = np.nonzero(ot == t)[0]
        if len(sel):
            assert (r[t, 0], r[t, 1]) == (sel[0], sel[-1] + 1)
        else:
            assert r[t, 0] == r[t, 1]
    assert tx * ((H + 15) // 16) == r.shape[0]


@pytest.mark.parametrize("N,H,W,scale,seed", CASES)
def test_forward_matches_oracle(N, H, W, scale, seed):
    torch = torch_cuda()
    w = lib_ready()
    p = synth.scene2d(N, H, W, seed, scale)
    _, _, img = _gpu_forward(w, torch, p, H, W)
    ref = oracle.render2d(p, H, W, truncated=True)
    err = np.abs(img.cpu().numpy().astype(np.float64) - ref)
    assert err.max() <= FWD_ATOL, (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("N,H,W,scale,seed", CASES)
def test_backward_matches_oracle(N, H, W, scale, seed):
    torch = torch_cuda()
    w = lib_ready()
    p = synth.scene2d(N, H, W, seed, scale)
    g = synth.upstream_grad(H, W, seed + 77)
    params, st, _ = _gpu_forward(w, torch, p, H, W)
    grad = w.backward(st, params, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    ref, gabs = oracle.grad2d(p, H, W, g, truncated=True, with_abs=True)
    ok, worst, idx = grad_close(grad.cpu().numpy(), ref, gabs, cols=list(range(11)))
    assert ok, (worst, idx)
    assert np.all(grad.cpu().numpy()[:, 11:] == 0)


def test_tile_lists_with_huge_and_offscreen_footprints():
    """Warps whose covered ranges differ by two orders of magnitude: huge footprints (hundreds of
    tiles each, so one primitive's range spans many of the 32-tile counting and emission rounds),
    primitives whose centre lies far outside the image (empty or partial ranges) and small ones,
    interleaved in index order.  Lists and ranges bit-exact; the image within the forward bound."""
    torch = torch_cuda()
    w = lib_ready()
    H, W = 200, 300
    rng = np.random.default_rng(41)
    p = synth.scene2d(1200, H, W, 41, (0.5, 6.0))
    huge = rng.random(p.shape[0]) < 0.04
    p[huge, 2:4] = rng.uniform(60.0, 200.0, (int(huge.sum()), 2)).astype(np.float32)
    off = rng.random(p.shape[0]) < 0.10
    p[off, 0] = rng.choice([-1.0, 1.0], int(off.sum())).astype(np.float32) * rng.uniform(310.0, 700.0, int(off.sum())).astype(np.float32)
    _, st, img = _gpu_forward(w, torch, p, H, W)
    tiles, prims, ranges = st.lists()
    ot, op = oracle.tile_lists(2, p, H, W)
    assert np.array_equal(tiles.cpu().numpy().view(np.uint32), ot)
    assert np.array_equal(prims.cpu().numpy().view(np.uint32), op)
    per_prim = np.bincount(op.astype(np.int64), minlength=p.shape[0])
    assert per_prim[huge].max() > 96  # some range spans more than three rounds
    r = ranges.cpu().numpy()
    for t in range(r.shape[0]):
        sel = np.nonzero(ot == t)[0]
        assert (r[t, 0], r[t, 1]) == ((sel[0], sel[-1] + 1) if len(sel) else (r[t, 0], r[t, 0]))
    ref = oracle.render2d(p, H, W, truncated=True)
    assert np.abs(img.cpu().numpy().astype(np.float64) - ref).max() <= FWD_ATOL


def test_rotation_angles_across_quadrants_bit_exact():
    """Rotation angles far outside [0, pi) (negative, many turns, and a third beyond 2^16, where
    the rule takes its binary64 branch): the footprint rule's cos and sin come from the same IEEE
    operation sequence on both sides, so the lists stay bit-exact and the image matches the
    oracle's binary64 rotation."""
    torch = torch_cuda()
    w = lib_ready()
    H, W = 96, 128
    p = synth.scene2d(1500, H, W, 21, (0.5, 24.0))
    rng = np.random.default_rng(22)
    th = rng.uniform(-200.0, 200.0, p.shape[0])
    wide = rng.random(p.shape[0]) < 1.0 / 3.0
    th[wide] = rng.choice([-1.0, 1.0], int(wide.sum())) * rng.uniform(7.0e4, 1.5e6, int(wide.sum()))
    p[:, 4] = th.astype(np.float32)
    _, st, img = _gpu_forward(w, torch, p, H, W)
    tiles, prims, _ = st.lists()
    ot, op = oracle.tile_lists(2, p, H, W)
    assert np.array_equal(tiles.cpu().numpy().view(np.uint32), ot)
    assert np.array_equal(prims.cpu().numpy().view(np.uint32), op)
    ref = oracle.render2d(p, H, W, truncated=True)
    assert np.abs(img.cpu().numpy().astype(np.float64) - ref).max() <= FWD_ATOL


def test_cutoff_boundary_pixels():
    """Axis-aligned primitives (theta = 0, s = (1, 2), so L = diag(1, 1/2) exactly) centred on pixel
    centres put pixel centres exactly on the cutoff ellipse (q = 9, inside by reading 6); centres
    moved by one binary32 step put the same pixels one step inside or outside.  The kernels fold
    the cutoff into the exponent, so these pixels check that the fold agrees with the q <= 9
    decision of the oracle's binary32 rule exactly."""
    torch = torch_cuda()
    w = lib_ready()
    H, W = 32, 48
    rng = np.random.default_rng(31)
    rows = []
    for k, (cx, cy) in enumerate([(8.5, 8.5), (24.5, 10.5), (40.5, 8.5), (10.5, 24.5), (26.5, 22.5), (38.5, 24.5)]):
        mx, my = np.float32(cx), np.float32(cy)
        if k % 3 == 1:  # one step towards -inf: pixels at dx = +3 fall outside, dx = -3 inside
            mx, my = np.nextafter(mx, np.float32(-np.inf)), np.nextafter(my, np.float32(-np.inf))
        elif k % 3 == 2:  # one step towards +inf: the reverse
            mx, my = np.nextafter(mx, np.float32(np.inf)), np.nextafter(my, np.float32(np.inf))
        f = rng.uniform(-0.3, 0.3, 2)
        rows.append([mx, my, 1.0, 2.0, 0.0, f[0], f[1], rng.uniform(0, 6.28), *rng.uniform(0.2, 1.0, 3)] + [0.0] * 5)
    p = np.array(rows, dtype=np.float32)
    rec, _, _ = oracle.footprints(2, p, H, W)
    assert np.all(rec[:, 2] == 1.0) and np.all(rec[:, 3] == 0.0) and np.all(rec[:, 4] == 0.5)
    # the boundary pixels of the centred primitive 0: q = 9 exactly at dx = +-3 and dy = +-6
    assert (np.float32(8.5 + 3.0) - p[0, 0]) ** 2 == np.float32(9.0)
    params, st, img = _gpu_forward(w, torch, p, H, W)
    tiles, prims, _ = st.lists()
    ot, op = oracle.tile_lists(2, p, H, W)
    assert np.array_equal(tiles.cpu().numpy().view(np.uint32), ot)
    assert np.array_equal(prims.cpu().numpy().view(np.uint32), op)
    ref = oracle.render2d(p, H, W, truncated=True)
    err = np.abs(img.cpu().numpy().astype(np.float64) - ref)
    assert err.max() <= FWD_ATOL, (err.max(), np.unravel_index(err.argmax(), err.shape))
    g = synth.upstream_grad(H, W, 32)
    grad = w.backward(st, params, torch.from_numpy(g).cuda()).cpu().numpy()
    ref_g, gabs = oracle.grad2d(p, H, W, g, truncated=True, with_abs=True)
    ok, worst, idx = grad_close(grad, ref_g, gabs, cols=list(range(11)))
    assert ok, (worst, idx)


def test_cutoff_outside_supported_range_is_refused():
    """The cutoff's power-of-two scale in the exponent is exact for cutoffs in [2^-10, 2^10]; other
    values are refused on the host with WIPES_ERR_INVALID before any device work."""
    torch = torch_cuda()
    w = lib_ready()
    from paper_2508_12615_gb300 import _abi

    params = torch.from_numpy(synth.scene2d(10, 16, 16, 3)).cuda()
    for bad in (2.0 ** -11, 2.0 ** 11, 0.0, float("inf"), float("nan")):
        with pytest.raises(_abi.WipesError) as e:
            w.forward2d(params, 16, 16, opts=w.make_opts(2, cutoff_sigma=bad))
        assert e.value.status == 1
    for ok in (2.0 ** -10, 2.0 ** 10):
        w.forward2d(params, 16, 16, opts=w.make_opts(2, cutoff_sigma=ok))
    torch.cuda.synchronize()


def test_autograd_function_matches_direct_calls():
    torch = torch_cuda()
    w = lib_ready()
    H, W = 48, 80
    p = synth.scene2d(150, H, W, 9)
    target = torch.from_numpy(synth.target_gabor(H, W, 10)).cuda()
    params = torch.from_numpy(p).cuda().requires_grad_(True)
    img = w.render2d(params, H, W)
    loss = ((img - target) ** 2).mean()
    loss.backward()
    # the same through the ABI calls, with the library's own loss kernel
    st = w.Context.get(0).acquire_state()
    img2 = w.forward2d(params.detach(), H, W, state=st)
    l2, gimg = w.l2_loss(img2, target)
    g2 = w.backward(st, params.detach(), gimg)
    torch.cuda.synchronize()
    assert torch.equal(img.detach(), img2)
    assert abs(float(l2) - float(loss)) <= 1e-6 * abs(float(loss))
    np.testing.assert_allclose(params.grad.cpu().numpy(), g2.cpu().numpy(), rtol=1e-5, atol=1e-7)


def test_deterministic():
    torch = torch_cuda()
    w = lib_ready()
    H, W = 96, 112
    p = synth.scene2d(800, H, W, 11, (0.5, 32.0))
    g = torch.from_numpy(synth.upstream_grad(H, W, 12)).cuda()
    outs = []
    for _ in range(2):
        params, st, img = _gpu_forward(w, torch, p, H, W)
        outs.append((img.clone(), w.backward(st, params, g).clone()))
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_edge_cases():
    torch = torch_cuda()
    w = lib_ready()
    H, W = 40, 50
    # no primitives: zero image and an empty gradient
    params = torch.zeros(0, 16, device="cuda")
    st = w.Context.get(0).acquire_state()
    img = w.forward2d(params, H, W, state=st)
    g = w.backward(st, params, torch.ones(H, W, 3, device="cuda"))
    torch.cuda.synchronize()
    assert img.abs().max().item() == 0 and g.shape == (0, 16)
    # off-screen, degenerate (zero or negative scale, NaN) and screen-filling primitives
    p = synth.scene2d(12, H, W, 13)
    p[0, :2] = [-500.0, 20.0]
    p[1, :2] = [25.0, 1e6]
    p[2, 2] = 0.0
    p[3, 3] = -1.0
    p[4, 0] = np.nan
    p[5, 2:4] = [400.0, 300.0]
    p[6, 2:4] = [0.05, 40.0]  # very elongated
    params, st, img = _gpu_forward(w, torch, p, H, W)
    ref = oracle.render2d(p, H, W, truncated=True)
    assert np.abs(img.cpu().numpy() - ref).max() <= FWD_ATOL
    gd = synth.upstream_grad(H, W, 14)
    grad = w.backward(st, params, torch.from_numpy(gd).cuda()).cpu().numpy()
    assert np.all(grad[[0, 1, 2, 3, 4]] == 0)
    ref, gabs = oracle.grad2d(p, H, W, gd, with_abs=True)
    ok, worst, idx = grad_close(grad, ref, gabs, cols=list(range(11)))
    assert ok, (worst, idx)


def test_state_reused_for_a_frame_with_no_pairs():
    """A state that held tile lists is reused for primitives that all lie off-screen (primitives,
    but no (tile, primitive) pairs): every tile range comes back empty, the image and the gradient
    are zero."""
    torch = torch_cuda()
    w = lib_ready()
    H, W = 48, 64
    st = w.Context.get(0).acquire_state()
    p = synth.scene2d(300, H, W, 41)
    params = torch.from_numpy(p).cuda()
    w.forward2d(params, H, W, state=st)
    torch.cuda.synchronize()
    assert st.info()["n_instances"] > 0
    q = p.copy()
    q[:, 0] += 10_000.0  # every centre far to the right of the image
    params2 = torch.from_numpy(q).cuda()
    img = w.forward2d(params2, H, W, state=st)
    grad = w.backward(st, params2, torch.ones(H, W, 3, device="cuda"))
    torch.cuda.synchronize()
    assert st.info()["n_instances"] == 0
    _, _, ranges = st.lists()
    r = ranges.cpu().numpy()
    assert np.all(r[:, 0] == r[:, 1])
    assert img.abs().max().item() == 0 and grad.abs().max().item() == 0


def test_full_size_768x512_70k_sampled():
    """The 768x512, 70,000-primitive image-fitting workload, in the launch configuration the
    benchmark times: lists bit-exact, sampled pixels and sampled primitive gradients vs the oracle."""
    torch = torch_cuda()
    w = lib_ready()
    p, target = synth.cfg1_inputs()
    c = synth.CFG1_2D_KODAK
    H, W = c.H, c.W
    params, st, img = _gpu_forward(w, torch, p, H, W)
    tiles, prims, _ = st.lists()
    ot, op = oracle.tile_lists(2, p, H, W)
    assert np.array_equal(tiles.cpu().numpy().view(np.uint32), ot)
    assert np.array_equal(prims.cpu().numpy().view(np.uint32), op)
    pix = sample_pixels(H, W, 1500, 21)
    ref = oracle.render2d(p, H, W, pixels=pix)
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]]
    assert np.abs(got - ref).max() <= FWD_ATOL
    # gradients of a primitive depend only on that primitive and dL/dimage in the summed field
    g = synth.upstream_grad(H, W, 22, scale=1e-3)
    grad = w.backward(st, params, torch.from_numpy(g).cuda()).cpu().numpy()
    sel = np.random.default_rng(23).choice(p.shape[0], 300, replace=False)
    ref_g, gabs = oracle.grad2d(p[sel], H, W, g, with_abs=True)
    ok, worst, idx = grad_close(grad[sel], ref_g, gabs, cols=list(range(11)))
    assert ok, (worst, idx)

"""The allocation-free loss entry point (for callers that cannot call cudaMalloc, e.g. code whose
allocator owns all device memory, or hosts that forbid device allocation after start-up) matches
the regular loss entry point.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from helpers import lib_ready, torch_cuda

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_loss_matches_regular_loss_on_two_calls():
    torch = torch_cuda()
    w = lib_ready()
    from paper_2508_12615_gb300 import _abi

    lib = _abi.lib()
    ctx = w.Context.get(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(5)
    for n in (768 * 512 * 3, 1000003):  # two calls in a row, the second smaller and ragged
        img = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
        tgt = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
        loss_a = torch.empty((), device="cuda")
        loss_b = torch.empty((), device="cuda")
        grad_a = torch.empty_like(img)
        grad_b = torch.full_like(img, float("nan"))
        _abi.check(lib.wipes_l2_loss(ctx.handle, _p(img), _p(tgt), n, _p(loss_a), _p(grad_a), stream), "l2_loss")
        _abi.check(lib.wipes_l2_loss_noalloc(_p(img), _p(tgt), n, _p(loss_b), _p(grad_b), stream), "l2_loss_noalloc")
        torch.cuda.synchronize()
        assert torch.equal(grad_a, grad_b)
        ref = float(((img.double() - tgt.double()) ** 2).mean())
        assert abs(float(loss_b) - float(loss_a)) <= 1e-6 * abs(float(loss_a))
        assert abs(float(loss_b) - ref) <= 1e-6 * ref


def test_noalloc_loss_rejects_sizes_beyond_its_scratch():
    torch = torch_cuda()
    lib_ready()
    from paper_2508_12615_gb300 import _abi

    lib = _abi.lib()
    x = torch.zeros(4, device="cuda")
    st = lib.wipes_l2_loss_noalloc(_p(x), _p(x), 268435456 + 1, _p(x), _p(x), None)
    assert st == 1 and b"268,435,456" not in lib.wipes_last_error() and b"268435456" in lib.wipes_last_error()
    assert lib.wipes_l2_loss_noalloc(_p(x), _p(x), 0, _p(x), _p(x), None) == 1


def test_noalloc_loss_leaves_device_memory_untouched():
    """After a first call (which may load the library's kernels and its scratch array), further
    calls change neither the device's free memory nor torch's reserved pool."""
    torch = torch_cuda()
    lib_ready()
    from paper_2508_12615_gb300 import _abi

    lib = _abi.lib()
    n = 1 << 20
    img = torch.rand(n, device="cuda")
    tgt = torch.rand(n, device="cuda")
    loss = torch.empty((), device="cuda")
    grad = torch.empty_like(img)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _abi.check(lib.wipes_l2_loss_noalloc(_p(img), _p(tgt), n, _p(loss), _p(grad), stream), "warm-up")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        _abi.check(lib.wipes_l2_loss_noalloc(_p(img), _p(tgt), n, _p(loss), _p(grad), stream), "l2_loss_noalloc")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    ref = float(((img.double() - tgt.double()) ** 2).mean())
    assert abs(float(loss) - ref) <= 1e-6 * ref

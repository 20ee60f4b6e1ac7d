"""Failure detection without a GPU fault: a bounded device wait that runs out is reported as a
status the host reads, and the context stays usable afterwards.

The radix sort's decoupled look-back waits for earlier tiles to publish their digit counts; the
diagnostic entry point runs one pass whose predecessor tile never publishes (a flag that nothing
sets), so the wait must run out, set the device error word and return.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import FWD_ATOL, lib_ready, torch_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(120)]

TIMEOUT = 4  # WIPES_ERR_TIMEOUT


def test_sort_lookback_timeout_is_reported_once_and_context_survives():
    torch = torch_cuda()
    w = lib_ready()
    from paper_2508_12615_gb300 import _abi

    lib = _abi.lib()
    ctx = w.Context.get(0)
    assert lib.wipes_selftest_sort_timeout(ctx.handle, None) == TIMEOUT
    assert b"ran out" in lib.wipes_last_error()
    # reported once: the next check is clean
    assert lib.wipes_sync_status(ctx.handle, None) == 0
    # the context still renders correctly
    p = synth.scene2d(300, 64, 80, seed=5)
    img = w.forward2d(torch.from_numpy(p).cuda(), 64, 80)
    torch.cuda.synchronize()
    ref = oracle.render2d(p, 64, 80)
    assert np.abs(img.cpu().numpy() - ref).max() <= FWD_ATOL
    assert lib.wipes_sync_status(ctx.handle, None) == 0

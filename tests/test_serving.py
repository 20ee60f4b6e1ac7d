"""Serving: continuous batching over resident scenes gives every request the same image it gets
alone, and admission keeps device memory within the HBM budget."""
import numpy as np
import pytest

import synth
from helpers import lib_ready, torch_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]


def _workload():
    return synth.serving_workload(n_scenes=6, rate=2000.0, seconds=0.06, seed=77, n_range=(2000, 20000), n_cams=3)


def test_each_request_renders_the_same_alone_and_in_the_mix():
    torch = torch_cuda()
    lib_ready()
    from paper_2508_12615_gb300.serve import Server

    scenes, reqs = _workload()
    assert len(reqs) > 50
    srv = Server(scenes, hbm_budget=40e9, max_batch=16, n_streams=2)
    res = srv.run_batched(reqs, keep_outputs=True)
    assert res.batches > 1 and np.all(np.isfinite(res.complete))
    assert np.all(res.complete >= res.arrival - 1e-3)
    for i in range(len(reqs)):
        alone = srv.render_one(reqs[i])
        torch.cuda.synchronize()
        assert torch.equal(alone, res.outputs[i]), i
    plain = srv.run_plain(reqs, keep_outputs=True)
    for i in range(len(reqs)):
        assert torch.equal(plain.outputs[i], res.outputs[i]), i
    s = res.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["mpix_s"] > 0
    del srv
    _teardown_is_clean()


def _teardown_is_clean():
    """Dropping a server releases its states and context without leaving a CUDA error behind."""
    import gc

    from paper_2508_12615_gb300 import Context, _abi

    gc.collect()
    _abi.call("wipes_sync_status", Context.get(0).handle, None)


def test_admission_respects_the_budget_and_evicts_views():
    torch_cuda()
    lib_ready()
    from paper_2508_12615_gb300.serve import Server

    scenes, reqs = _workload()
    probe = Server(scenes, hbm_budget=1e12)
    budget = probe.resident_bytes + 150e6  # room for a few views and outputs only
    srv = Server(scenes, hbm_budget=budget, max_batch=8, n_streams=2)
    res = srv.run_batched(reqs)
    assert np.all(np.isfinite(res.complete))
    assert res.peak_bytes <= budget
    assert res.prepared > len(srv.views)  # views were evicted and prepared again
    # the library refuses workspace growth past the limit with WIPES_ERR_OOM, before allocating
    from paper_2508_12615_gb300 import _abi

    _abi.call("wipes_set_memory_limit", srv.ctx.handle, 1)
    with pytest.raises(_abi.WipesError) as e:
        srv._prepare(reqs[0], srv._spare.pop() if srv._spare else __import__("paper_2508_12615_gb300").State(srv.ctx),
                     srv.streams[0])
    assert e.value.status == 5
    del srv, probe
    _teardown_is_clean()

"""Continuous-batching render server over resident wavelet scenes.

Requests name a resident scene, an image size and (3D) a camera.  The server keeps scene
parameters and, per view, the prepared tile lists (projected records, sorted lists, tile ranges)
on the device, admits requests while an HBM budget allows, and renders every admitted request of
a round in one persistent batch launch (``wipes_blend_batch``).  Rounds run on several CUDA
streams, so requests that arrive while one round is on the GPU are admitted into the next and the
two overlap on the device.  The plain path renders one request at a time with the one-frame calls.

Latency is measured on the device clock: a request's completion is the time of the event recorded
after the launch that rendered it, relative to an event recorded when the run starts.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _abi
from .render import Context, State, _ptr, make_opts

SIZES = ((256, 256), (512, 512), (800, 800), (1080, 1920))  # (H, W)


@dataclass
class RunResult:
    arrival: np.ndarray          # seconds
    complete: np.ndarray         # seconds, device clock
    pixels: np.ndarray           # per request
    batches: int = 0
    prepared: int = 0            # views prepared (projection, binning, sort)
    peak_bytes: int = 0          # largest device bytes of scenes, workspaces and outputs
    outputs: dict = field(default_factory=dict)  # request index -> image (when kept)

    def summary(self) -> dict:
        lat = (self.complete - self.arrival) * 1e3
        span = float(self.complete.max() - self.arrival.min())
        return {"requests": int(len(lat)), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "mpix_s": float(self.pixels.sum() / span / 1e6), "makespan_s": span, "batches": self.batches,
                "views_prepared": self.prepared, "peak_gb": self.peak_bytes / 1e9}


class _View:
    __slots__ = ("state", "busy")

    def __init__(self, state: State, busy: int):
        self.state, self.busy = state, busy


class Server:
    """Resident scenes (``synth.ServingScene``) on one device, served under an HBM budget."""

    def __init__(self, scenes, device: int = 0, hbm_budget: float = 120e9, max_batch: int = 128,
                 n_streams: int = 2, cache_views: bool = True, max_prepares_per_round: int = 8):
        self.dev = torch.device("cuda", device)
        self.ctx = Context(device)  # own context: its workspace memory is the server's to budget
        self.budget = float(hbm_budget)
        self.max_batch = max_batch
        self.max_prepares = max_prepares_per_round  # bounds how long forming one round can take
        self.cache_views = cache_views
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_streams)]
        self.opts = {2: make_opts(2), 3: make_opts(3)}
        self.scenes = scenes
        self.params = []
        self.resident_bytes = 0
        for sc in scenes:
            d = {k: torch.from_numpy(v).to(self.dev) for k, v in sc.params.items()}
            self.params.append(d)
            self.resident_bytes += sum(t.numel() * 4 for t in d.values())
        self.views: "collections.OrderedDict[tuple, _View]" = collections.OrderedDict()
        self._spare: list[State] = []

    # -- views --------------------------------------------------------------------------------
    def _key(self, req) -> tuple:
        scene, size, cam = int(req[1]), int(req[2]), int(req[3])
        return (scene, size, cam if self.scenes[scene].dims == 3 else -1)

    def _prepare(self, req, state: State, stream: torch.cuda.Stream) -> None:
        scene, size, cam = int(req[1]), int(req[2]), int(req[3])
        sc = self.scenes[scene]
        H, W = SIZES[size]
        s = ctypes.c_void_p(stream.cuda_stream)
        if sc.dims == 2:
            p = self.params[scene][size]
            _abi.call("wipes_prepare2d", self.ctx.handle, state.handle, _ptr(p), p.shape[0], H, W,
                      ctypes.byref(self.opts[2]), s)
        else:
            p = self.params[scene][0]
            c = _abi.camera_struct(sc.cameras[size][cam].tolist())
            _abi.call("wipes_prepare3d", self.ctx.handle, state.handle, _ptr(p), p.shape[0], ctypes.byref(c), H, W,
                      ctypes.byref(self.opts[3]), s)

    def _reserved(self) -> int:
        b = ctypes.c_int64()
        _abi.call("wipes_get_memory_reserved", self.ctx.handle, ctypes.byref(b))
        return b.value

    def _free_one(self, keep: tuple | None) -> bool:
        """Release workspace memory: a spare state first, else the least recently used idle view."""
        if self._spare:
            self._spare.pop()  # destroying the state frees its buffers
            return True
        victim = next((k for k, v in self.views.items() if v.busy == 0 and k != keep), None)
        if victim is None:
            return False
        self.views.pop(victim)
        return True

    def _prepare_within_budget(self, req, key, stream, outputs: int) -> State | None:
        """Prepare a view with the workspace limited to what the budget leaves after the resident
        scenes and the output images; on a refusal free memory and retry.  None: cannot fit now.
        Every retry first destroys the refused state and then frees one spare state or one idle
        view, so the loop ends."""
        limit = int(self.budget - self.resident_bytes - outputs)
        if limit <= 0:
            return None
        _abi.call("wipes_set_memory_limit", self.ctx.handle, limit)
        while True:
            st = self._spare.pop() if self._spare else State(self.ctx)
            try:
                self._prepare(req, st, stream)
                return st
            except _abi.WipesError as e:
                if e.status != 5:  # not WIPES_ERR_OOM
                    raise
            del st  # destroys the refused state and its buffers
            if not self._free_one(keep=key):
                return None

    # -- batched path ---------------------------------------------------------------------------
    def run_batched(self, requests: np.ndarray, keep_outputs: bool = False) -> RunResult:
        R = len(requests)
        res = RunResult(requests[:, 0].copy(), np.full(R, np.nan), np.zeros(R))
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        pending: collections.deque = collections.deque()
        inflight = []  # (stream index, event, request indices, views, outputs, bytes)
        nxt = done = 0
        out_bytes = 0
        while done < R:
            now = time.perf_counter() - t0
            while nxt < R and requests[nxt, 0] <= now:
                pending.append(nxt)
                nxt += 1
            for b in [b for b in inflight if b[1].query()]:
                inflight.remove(b)
                t_done = start.elapsed_time(b[1]) / 1e3
                for i, v, o in zip(b[2], b[3], b[4]):
                    res.complete[i] = t_done
                    v.busy -= 1
                    if not self.cache_views:
                        self._spare.append(v.state)
                    if keep_outputs:
                        res.outputs[i] = o
                out_bytes -= b[5]
                done += len(b[2])
            busy = {b[0] for b in inflight}
            free = [k for k in range(len(self.streams)) if k not in busy]
            if not pending or not free:
                if nxt < R and not pending and not inflight:
                    time.sleep(max(0.0, min(requests[nxt, 0] - now, 1e-3)))
                continue
            k = free[0]
            stream = self.streams[k]
            reqs, views, outs, nbytes = [], [], [], 0
            prepares = 0
            with torch.cuda.stream(stream):
                while pending and len(reqs) < self.max_batch:
                    i = pending[0]
                    req = requests[i]
                    H, W = SIZES[int(req[2])]
                    key = self._key(req)
                    v = self.views.get(key) if self.cache_views else None
                    if v is None and prepares >= self.max_prepares and reqs:
                        break  # leave further new views to the next scheduling pass
                    prepares += v is None
                    out_need = out_bytes + nbytes + H * W * 12
                    while self.resident_bytes + out_need + self._reserved() > self.budget and self._free_one(key):
                        pass
                    if v is not None and self.resident_bytes + out_need + self._reserved() > self.budget:
                        if inflight or reqs:
                            break  # budget full: admit later, when rounds in flight release memory
                        raise RuntimeError("a single request does not fit the HBM budget")
                    if v is None:
                        st = self._prepare_within_budget(req, key, stream, out_need)
                        if st is None:
                            if inflight or reqs:
                                break  # budget full: admit later, when rounds in flight release memory
                            raise RuntimeError("a single request does not fit the HBM budget")
                        res.prepared += 1
                        v = _View(st, 0)
                        if self.cache_views:
                            self.views[key] = v
                    else:
                        self.views.move_to_end(key)
                    pending.popleft()
                    v.busy += 1
                    out = torch.empty(H, W, 3, device=self.dev)
                    reqs.append(i)
                    views.append(v)
                    outs.append(out)
                    nbytes += H * W * 12
                    res.pixels[i] = H * W
                    res.peak_bytes = max(res.peak_bytes, self.resident_bytes + self._reserved() + out_bytes + nbytes)
                if reqs:
                    st_arr = (ctypes.c_void_p * len(reqs))(*[v.state.handle.value for v in views])
                    out_arr = (ctypes.c_void_p * len(reqs))(*[o.data_ptr() for o in outs])
                    _abi.call("wipes_blend_batch", self.ctx.handle, st_arr, out_arr, len(reqs),
                              ctypes.c_void_p(stream.cuda_stream))
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(stream)
                    inflight.append((k, ev, reqs, views, outs, nbytes))
                    out_bytes += nbytes
                    res.batches += 1
        torch.cuda.synchronize(self.dev)
        return res

    # -- plain path over the view cache ----------------------------------------------------------
    def run_plain_cached(self, requests: np.ndarray, keep_outputs: bool = False) -> RunResult:
        """One request at a time, in arrival order, from the same view cache and HBM budget as the
        batched path: a view is prepared on first use and kept; each request is rendered by its own
        one-frame launch (wipes_blend_batch with one job) on one stream.  Against run_batched this
        leaves batching as the only difference."""
        R = len(requests)
        res = RunResult(requests[:, 0].copy(), np.full(R, np.nan), np.zeros(R))
        stream = self.streams[0]
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        events = []
        with torch.cuda.stream(stream):
            for i in range(R):
                while time.perf_counter() - t0 < requests[i, 0]:
                    pass
                req = requests[i]
                H, W = SIZES[int(req[2])]
                key = self._key(req)
                out = torch.empty(H, W, 3, device=self.dev)
                v = self.views.get(key) if self.cache_views else None
                if v is None:
                    st = self._prepare_within_budget(req, key, stream, H * W * 12)
                    if st is None:
                        raise RuntimeError("a single request does not fit the HBM budget")
                    res.prepared += 1
                    v = _View(st, 0)
                    if self.cache_views:
                        self.views[key] = v
                else:
                    self.views.move_to_end(key)
                _abi.call("wipes_blend_batch", self.ctx.handle, (ctypes.c_void_p * 1)(v.state.handle.value),
                          (ctypes.c_void_p * 1)(out.data_ptr()), 1, ctypes.c_void_p(stream.cuda_stream))
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                events.append(ev)
                res.pixels[i] = H * W
                res.peak_bytes = max(res.peak_bytes, self.resident_bytes + self._reserved() + H * W * 12)
                if keep_outputs:
                    res.outputs[i] = out
        torch.cuda.synchronize(self.dev)
        res.complete[:] = [start.elapsed_time(e) / 1e3 for e in events]
        res.batches = R
        return res

    # -- plain path -------------------------------------------------------------------------------
    def run_plain(self, requests: np.ndarray, keep_outputs: bool = False) -> RunResult:
        """One request at a time, in arrival order, with the one-frame calls (no batching, no view
        cache)."""
        R = len(requests)
        res = RunResult(requests[:, 0].copy(), np.full(R, np.nan), np.zeros(R))
        _abi.call("wipes_set_memory_limit", self.ctx.handle, 0)
        st = State(self.ctx)
        stream = self.streams[0]
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        events = []
        with torch.cuda.stream(stream):
            for i in range(R):
                while time.perf_counter() - t0 < requests[i, 0]:
                    pass
                out = self.render_one(requests[i], st, stream)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                events.append(ev)
                res.pixels[i] = out.shape[0] * out.shape[1]
                res.prepared += 1
                if keep_outputs:
                    res.outputs[i] = out
        torch.cuda.synchronize(self.dev)
        res.complete[:] = [start.elapsed_time(e) / 1e3 for e in events]
        res.batches = R
        return res

    def render_one(self, req, state: State | None = None, stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        """Render one request alone (wipes_render2d / wipes_render3d), outside the budget."""
        _abi.call("wipes_set_memory_limit", self.ctx.handle, 0)
        stream = stream or torch.cuda.current_stream(self.dev)
        state = state or State(self.ctx)
        scene, size, cam = int(req[1]), int(req[2]), int(req[3])
        sc = self.scenes[scene]
        H, W = SIZES[size]
        out = torch.empty(H, W, 3, device=self.dev)
        s = ctypes.c_void_p(stream.cuda_stream)
        if sc.dims == 2:
            p = self.params[scene][size]
            _abi.call("wipes_render2d", self.ctx.handle, state.handle, _ptr(p), p.shape[0], H, W,
                      ctypes.byref(self.opts[2]), _ptr(out), s)
        else:
            p = self.params[scene][0]
            c = _abi.camera_struct(sc.cameras[size][cam].tolist())
            _abi.call("wipes_render3d", self.ctx.handle, state.handle, _ptr(p), p.shape[0], ctypes.byref(c), H, W,
                      ctypes.byref(self.opts[3]), _ptr(out), s)
        return out

#!/usr/bin/env python
"""Benchmark of the WIPES wavelet rasterizer on one GB300 (or N replicas under torchrun).

Workload: 2D image fitting at 768x512 RGB with 70,000 wavelet primitives (seeded synthetic scene and
target standing in for a Kodak image).  One step = forward render, mean-squared-error loss and its
gradient, backward to all primitive parameters: every stage runs in libwipes.so kernels.

Prints one JSON line: value = whole-job fwd+bwd iterations/s; also forward-only Mpix/s, the
end-to-end rate with host buffers, per-stage times, the roofline of the dominant kernel and the
binary64 oracle timed on the host cores (a reported baseline, not a target).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import types
import subprocess
import sys
import tempfile
import time

import numpy as np

# the oracle's OpenMP threads sleep instead of spinning when idle, so that they take no host time
# from the measurements that follow them
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd Mpix/s and fwd+bwd iter/s (768×512, 70k prims); serving p50/p99 ms vs plain path"
WORKLOAD = "2d_image_fitting_768x512_n70000"
FP32_LANES_PER_SM = 128
SMS = 152
# Algorithmic FP32-pipe operations (an FMA counts as one) and MUFU operations per (pixel, primitive)
# pair inside the cutoff ellipse, counted from the method's arithmetic rather than from the kernels:
# the 2D forward 15 + 2 (offsets, quadratic form, phase reduction, exp2, cos, modulation, 3-channel
# accumulate), the 3D forward 6 more (alpha, clamp, transmittance update and tests), each backward
# 2.5 times its forward with one more MUFU (sin).
OPS_PER_PAIR = {"2d": {"blend": (15, 2), "bwd_raster": (37.5, 3)}, "3d": {"blend": (21, 2), "bwd_raster": (52.5, 3)}}
# DRAM bytes (read + write) per launch, per (workload, kernel), from the ncu captures summarised in
# profiles/ (dram__bytes_read.sum + dram__bytes_write.sum), for the kernel build measured there; an
# entry is removed when its kernel changes.
TRAFFIC_BYTES = {("2d", "k_backward2d"): 17_499_648 + 737_536, ("2d", "k_blend2d"): 9_069_824,
                 ("5d", "k_backward3d"): 23_489_536 + 3_840, ("5d", "k_blend3d"): 14_042_880 + 19_712}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["2d", "2dsmall", "2dchol", "5d", "5dsh", "6d", "6dmlp"], default="2d",
                    help="2d: the 768x512 / 70k image-fitting workload (default, the headline); 2dsmall: the "
                         "256x256 / 2k image-fitting workload; 2dchol: the "
                         "same with the Cholesky covariance record; 5d: 800x800 / 300k static scene; 5dsh: the "
                         "same with degree-3 spherical-harmonic colour; 6d: 1352x1014 / 200k dynamic scene, 4 "
                         "samples per step (linear time model); 6dmlp: the same scene deformed by the network")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="with the default workload, skip the other configurations (256x256 / 2k, 800x800 / 300k, "
                         "1352x1014 / 200k) that the line otherwise carries under 'configs'")
    ap.add_argument("--config-steps", type=int, default=20, help="timed steps of each of those configurations")
    ap.add_argument("--config-cpu-seconds", type=float, default=8.0,
                    help="CPU work budget of the oracle baseline of each of those configurations")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serving-seconds", type=float, default=10.0, help="length of the serving request trace")
    ap.add_argument("--saturation-seconds", type=float, default=0.5,
                    help="length of the serving trace at 20,000 requests/s (above the plain path's capacity)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="CPU work budget of the oracle baseline")
    ap.add_argument("--no-sort-bw", action="store_true", help="skip the radix-sort bandwidth measurement")
    ap.add_argument("--sort-n", type=int, default=1 << 25, help="pairs of the sort bandwidth measurement")
    ap.add_argument("--only-sort", action="store_true",
                    help="print only the sort bandwidth measurement (one JSON object) and exit")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.file = tempfile.NamedTemporaryFile(prefix="clocks_", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.close()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[0].isdigit() and int(parts[0]) == self.gpu:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][2]),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows), "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------------------------------------
# CPU oracle baseline
# ------------------------------------------------------------------------------------------------

def oracle_step_sample(p, target, H, W, budget_s: float):
    """Time the binary64 oracle on a bounded sample of one step (forward on a subset of rows,
    backward on a subset of primitives) and extrapolate to one full step.  Returns
    (seconds per full step, sample description)."""
    import numpy as np

    import oracle

    oracle.build()
    n = p.shape[0]
    # calibration on a tiny sample
    rows = max(1, H // 256)
    pix = np.stack(np.meshgrid(np.arange(W), np.arange(rows)), -1).reshape(-1, 2).astype(np.int32)
    t0 = time.perf_counter()
    oracle.render2d(p, H, W, pixels=pix)
    t_fwd_px = (time.perf_counter() - t0) / len(pix)
    g = np.zeros((H, W, 3), np.float32)
    sub = p[: max(1, n // 2000)]
    t0 = time.perf_counter()
    oracle.grad2d(sub, H, W, g)
    t_bwd_prim = (time.perf_counter() - t0) / len(sub)
    full = t_fwd_px * H * W + t_bwd_prim * n

    def sample(frac):
        n_rows = max(1, int(round(H * frac)))
        n_prims = max(1, int(round(n * frac)))
        pix = np.stack(np.meshgrid(np.arange(W), np.arange(n_rows)), -1).reshape(-1, 2).astype(np.int32)
        t0 = time.perf_counter()
        img_rows = oracle.render2d(p, H, W, pixels=pix)
        t_f = time.perf_counter() - t0
        # upstream gradient of the mean squared error on the sampled rows
        gimg = np.zeros((H, W, 3), np.float32)
        gimg[:n_rows] = (2.0 / (H * W * 3)) * (img_rows.reshape(n_rows, W, 3) - target[:n_rows])
        t0 = time.perf_counter()
        oracle.grad2d(p[:n_prims], H, W, gimg)
        t_b = time.perf_counter() - t0
        return n_rows, n_prims, t_f, t_b

    frac = min(1.0, budget_s / max(full, 1e-9))
    n_rows, n_prims, t_f, t_b = sample(frac)
    # the tiny calibration samples overstate the per-item cost (thread start-up, cold caches): when
    # the sample took well under the budget, size it again from its own measured rate
    if frac < 1.0 and t_f + t_b < 0.5 * budget_s:
        est = t_f * (H / n_rows) + t_b * (n / n_prims)
        n_rows, n_prims, t_f, t_b = sample(min(1.0, 0.9 * budget_s / max(est, 1e-9)))
    per_step = t_f * (H / n_rows) + t_b * (n / n_prims)
    desc = (f"forward on {n_rows} of {H} rows and backward for {n_prims} of {n} primitives "
            f"({t_f + t_b:.1f} s of CPU work), scaled to one full step")
    return per_step, desc


def cpu_cores() -> int:
    env = os.environ.get("OMP_NUM_THREADS")
    return int(env) if env and env.isdigit() else (os.cpu_count() or 1)


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time: every rank contributes its own, all receive the maximum."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, ms: float) -> float:
    """Steps per second of the whole job: each of the `world` replicas ran `steps` steps within
    the slowest rank's `ms`."""
    return world * steps / (ms / 1000.0)


# ------------------------------------------------------------------------------------------------
# arms
# ------------------------------------------------------------------------------------------------

def reference_arm(args, rank: int, world: int):
    import synth

    if rank != 0:
        return
    p, target = synth.cfg1_inputs()
    c = synth.CFG1_2D_KODAK
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    per_step = []
    desc = ""
    for i in range(args.warmup + args.steps):
        s, desc = oracle_step_sample(p, target, c.H, c.W, budget)
        if i >= args.warmup:
            per_step.append(s)
    ms = 1000.0 * statistics.mean(per_step)
    value = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": c.H, "W": c.W, "primitives": c.n, "seed": c.seed},
            "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": "each step: " + desc},
            "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Workload:
    """One benchmark workload: inputs resident on the device, a fwd+bwd step, a forward-only
    pass, and an end-to-end step from pinned host buffers."""

    def __init__(self, kind: str, dev):
        import torch

        import paper_2508_12615_gb300 as w
        import synth

        self.kind, self.dev, self.w = kind, dev, w
        ctx = w.Context.get(dev.index)
        self.ctx = ctx
        self.st = w.State(ctx)
        if kind == "2d":
            c = synth.CFG1_2D_KODAK
            p, target = synth.cfg1_inputs()
            self.name, self.H, self.W, self.seed = WORKLOAD, c.H, c.W, c.seed
            self.samples = [None]
            self.opts = w.make_opts(2)
        elif kind == "2dsmall":
            c = synth.CFG0_2D_SMALL
            p, target = synth.cfg0_inputs()
            self.name, self.H, self.W, self.seed = "2d_image_fitting_256x256_n2000", c.H, c.W, c.seed
            self.samples = [None]
            self.opts = w.make_opts(2)
        elif kind == "2dchol":
            c = synth.CFG1_2D_KODAK
            _, target = synth.cfg1_inputs()
            p = synth.scene2d_cholesky(c.n, c.H, c.W, c.seed, (0.5, 32.0))
            self.name, self.H, self.W, self.seed = "2d_cholesky_768x512_n70000", c.H, c.W, c.seed
            self.samples = [None]
            self.opts = w.make_opts(2, cov2d=1)
        elif kind in ("5d", "5dsh"):
            c = synth.CFG2_5D
            p, cams = synth.cfg2_inputs()
            if kind == "5dsh":
                p = synth.scene3d_sh(c.n, c.seed, degree=3)
            target = synth.target_noise_edges(c.H, c.W, c.seed + 200)
            self.name, self.H, self.W, self.seed = "5d_static_800x800_n300000", c.H, c.W, c.seed
            if kind == "5dsh":
                self.name = "5d_static_sh3_800x800_n300000"
            self.cams = cams
            self.samples = [(k, None) for k in range(len(cams))]
            self.opts = w.make_opts(3, sh_degree=3 if kind == "5dsh" else 0)
        else:
            c = synth.CFG3_6D
            p, cams, times = synth.cfg3_inputs()
            if kind == "6dmlp":  # canonical records and the deformation network's parameters
                p = np.ascontiguousarray(p[:, :20])
                self.theta = torch.from_numpy(synth.deform_mlp_theta(c.seed + 400)).to(dev)
                self.gtheta = torch.zeros_like(self.theta)
                self.st_mlp = w.State(ctx)
            target = synth.target_noise_edges(c.H, c.W, c.seed + 200)
            self.name, self.H, self.W, self.seed = "6d_dynamic_1352x1014_n200000_batch4", c.H, c.W, c.seed
            if kind == "6dmlp":
                self.name = "6d_dynamic_mlp_1352x1014_n200000_batch4"
            self.cams, self.times = cams, times
            rng = np.random.default_rng(c.seed + 300)
            self.samples = [(int(rng.integers(len(cams))), float(times[rng.integers(len(times))])) for _ in range(64)]
            self.opts = w.make_opts(3)
        self.p, self.target = p, target
        self.params = torch.from_numpy(p).to(dev)
        self.target_d = torch.from_numpy(target).to(dev)
        self.img = torch.empty(self.H, self.W, 3, device=dev)
        self.gimg = torch.empty_like(self.img)
        # the parameter gradient and the loss share one buffer, so that a step's results come back
        # to the host in one copy
        n_out = self.params.numel()
        self.out = torch.empty(n_out + 4, device=dev)
        self.grad = self.out[:n_out].view_as(self.params)
        self.loss = self.out[n_out]
        if kind in ("6d", "6dmlp"):
            self.p3 = torch.empty(p.shape[0], 20, device=dev)
            self.g3 = torch.empty_like(self.p3)
        self.batch = 4 if kind in ("6d", "6dmlp") else 1
        # 6D: the step's samples run concurrently, one stream each, every one with its own library
        # context (a context's loss buffer serves one call at a time), state and buffers; only
        # their accumulation into the shared parameter gradient follows the sample order
        self.lanes = []
        self.concurrent = True
        if kind in ("6d", "6dmlp"):
            for b in range(self.batch):
                first = b == 0
                lctx = ctx if first else w.Context(dev.index)
                lane = types.SimpleNamespace(
                    ctx=lctx, st=self.st if first else w.State(lctx), stream=torch.cuda.Stream(device=dev),
                    done=torch.cuda.Event(), img=self.img if first else torch.empty_like(self.img),
                    gimg=self.gimg if first else torch.empty_like(self.gimg),
                    p3=self.p3 if first else torch.empty_like(self.p3), g3=self.g3 if first else torch.empty_like(self.g3),
                    loss=self.out[n_out + b])
                if kind == "6dmlp":
                    lane.st_mlp = self.st_mlp if first else w.State(lctx)
                self.lanes.append(lane)
        self.k = 0
        self.pixels_per_step = self.H * self.W * self.batch

    def _sample(self):
        s = self.samples[self.k % len(self.samples)]
        self.k += 1
        return s

    def _one(self, params, target, accumulate=False, fwd_only=False):
        w = self.w
        if self.kind in ("2d", "2dsmall", "2dchol"):
            w.forward2d(params, self.H, self.W, self.opts, state=self.st, out=self.img)
            if fwd_only:
                return
            w.l2_loss(self.img, target, loss=self.loss, grad=self.gimg)
            w.backward(self.st, params, self.gimg, out=self.grad)
            return
        cam_i, t = self._sample()
        cam = self.cams[cam_i]
        if self.kind in ("5d", "5dsh"):
            w.forward3d(params, cam, self.H, self.W, self.opts, state=self.st, out=self.img)
            if fwd_only:
                return
            w.l2_loss(self.img, target, loss=self.loss, grad=self.gimg)
            w.backward(self.st, params, self.gimg, out=self.grad)
            return
        raise AssertionError("6D samples run through _one_6d")

    def _one_6d(self, lane, b, params, target, fwd_only, prev_done):
        """Sample b of a 6D step on its lane's stream (the current stream): the time model or the
        network, the render, the loss, the render backward, and, after sample b - 1's (prev_done),
        the accumulation into the parameter gradient."""
        import torch

        from paper_2508_12615_gb300 import _abi
        from paper_2508_12615_gb300.render import _ptr, _stream

        w = self.w
        cam_i, t = self._sample()
        cam = self.cams[cam_i]
        n = params.shape[0]
        if self.kind == "6dmlp":
            w.deform_mlp(params, t, self.theta, state=lane.st_mlp, out=lane.p3)
        else:
            _abi.call("wipes_deform6d", _ptr(params), n, t, _ptr(lane.p3), _stream(self.dev))
        w.forward3d(lane.p3, cam, self.H, self.W, self.opts, state=lane.st, out=lane.img)
        if fwd_only:
            return
        w.l2_loss(lane.img, target, loss=lane.loss, grad=lane.gimg, ctx=lane.ctx)
        w.backward(lane.st, lane.p3, lane.gimg, out=lane.g3)
        if prev_done is not None:
            torch.cuda.current_stream().wait_event(prev_done)
        if self.kind == "6dmlp":
            w.deform_mlp_backward(lane.st_mlp, params, lane.g3, grad_theta=self.gtheta, grad_params3=self.grad,
                                  accumulate=b > 0)
        else:
            _abi.call("wipes_deform6d_backward", _ptr(params), n, t, _ptr(lane.g3), _ptr(self.grad), int(b > 0),
                      _stream(self.dev))
        lane.done.record()

    def _lanes_run(self, params, target, fwd_only):
        import torch

        main = torch.cuda.current_stream()
        if not self.concurrent:  # one sample after another on the current stream
            for b, lane in enumerate(self.lanes):
                self._one_6d(lane, b, params, target, fwd_only, None)
            return
        prev = None
        for b, lane in enumerate(self.lanes):
            lane.stream.wait_stream(main)
            with torch.cuda.stream(lane.stream):
                self._one_6d(lane, b, params, target, fwd_only, prev)
            prev = lane.done
        for lane in self.lanes:
            main.wait_stream(lane.stream)

    def step(self, params=None, target=None):
        params = self.params if params is None else params
        target = self.target_d if target is None else target
        if self.lanes:
            self._lanes_run(params, target, fwd_only=False)
            return
        for b in range(self.batch):
            self._one(params, target, accumulate=b > 0)

    def forward(self):
        if self.lanes:
            self._lanes_run(self.params, self.target_d, fwd_only=True)
            return
        for b in range(self.batch):
            self._one(self.params, self.target_d, fwd_only=True)

    def count_pairs(self):
        import torch

        from paper_2508_12615_gb300 import _abi

        self.k = 0
        if self.lanes:
            self._one_6d(self.lanes[0], 0, self.params, self.target_d, True, None)
        else:
            self._one(self.params, self.target_d, fwd_only=True)
        visited, inside = ctypes.c_int64(), ctypes.c_int64()
        _abi.call("wipes_state_count_pairs", self.ctx.handle, self.st.handle, ctypes.byref(visited),
                  ctypes.byref(inside), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        return visited.value * self.batch, inside.value * self.batch, self.st.info()["n_instances"] * self.batch


def measure(wl, steps: int, warmup: int, flush, dist, world: int, dev, sample_clocks: bool) -> dict:
    """Time one workload: `steps` fwd+bwd steps (L2 flushed before each, each bracketed by CUDA
    events, max over ranks), the library's per-stage brackets in a separate pass, the forward alone,
    and the end-to-end step through the public API with pinned host buffers."""
    import torch

    from paper_2508_12615_gb300 import _abi

    lib = _abi.lib()
    ctx = wl.ctx

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(3, warmup)):
        wl.step()
    torch.cuda.synchronize()

    # fwd+bwd steps (no events between the stages here: the stage brackets come in a separate pass)
    launches0 = lib.wipes_kernel_launches()
    sampler = ClockSampler(torch.cuda.current_device()) if sample_clocks else None
    if sampler:
        sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record()
        wl.step()
        ev[k][1].record()
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop() if sampler else None
    launches = lib.wipes_kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # per-stage times: more steps with the library's CUDA-event brackets around each stage (the
    # samples of a 6D step one after another, so that each kernel is timed alone)
    lib.wipes_set_timing(ctx.handle, 1)
    lib.wipes_get_timing(ctx.handle, None, None, 1)
    wl.concurrent = False
    for _ in range(max(3, min(steps, 20))):
        flush.zero_()
        wl.step()
    torch.cuda.synchronize()
    wl.concurrent = True
    stage_ms = (ctypes.c_double * len(_abi.STAGES))()
    stage_n = (ctypes.c_int64 * len(_abi.STAGES))()
    lib.wipes_get_timing(ctx.handle, stage_ms, stage_n, 1)
    lib.wipes_set_timing(ctx.handle, 0)
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    stages = {name: {"ms_per_launch": (stage_ms[i] / stage_n[i]) if stage_n[i] else None, "launches": int(stage_n[i])}
              for i, name in enumerate(_abi.STAGES) if stage_n[i]}

    # forward only (Mpix/s)
    fwd_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        fwd_ev[k][0].record()
        wl.forward()
        fwd_ev[k][1].record()
    torch.cuda.synchronize()
    fwd_ms = statistics.mean(a.elapsed_time(b) for a, b in fwd_ev)

    # end to end through the public API with host buffers: a step's inputs (parameters, then
    # target) travel from pinned host memory in one copy, its results (gradient, then loss) back in
    # another, every step
    n_p = wl.params.numel()
    in_host = torch.empty(n_p + wl.target_d.numel(), dtype=torch.float32).pin_memory()
    in_host[:n_p].copy_(torch.from_numpy(wl.p).reshape(-1))
    in_host[n_p:].copy_(torch.from_numpy(wl.target).reshape(-1))
    out_host = torch.empty(wl.out.numel(), dtype=torch.float32).pin_memory()
    e2e_in = torch.empty(in_host.numel(), device=dev)
    e2e_params = e2e_in[:n_p].view_as(wl.params)     # offset 0: 16-byte aligned
    e2e_target = e2e_in[n_p:].view_as(wl.target_d)   # offset n_p * 4 bytes, a multiple of 64
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        e_ev[k][0].record()
        e2e_in.copy_(in_host, non_blocking=True)
        wl.step(e2e_params, e2e_target)
        out_host.copy_(wl.out, non_blocking=True)
        e_ev[k][1].record()
        torch.cuda.current_stream().synchronize()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e_ev), dist, dev)
    return {"value": whole_job_rate(world, steps, total_ms), "ms_per_step": total_ms / steps, "steps": steps,
            "fwd_ms": fwd_ms, "fwd_mpix_s": wl.pixels_per_step / (fwd_ms * 1e-3) / 1e6 * world,
            "e2e": {"value": whole_job_rate(world, steps, e2e_ms), "unit": "iter/s",
                    "h2d_bytes_per_step": int(wl.p.nbytes + wl.target.nbytes),
                    "d2h_bytes_per_step": int(out_host.numel() * 4)},
            "gpu_launches": int(launches), "stages": stages, "clocks": clocks, "wall_s_timed_region": t_wall}


def roofline_of(wl, stages: dict, pk: dict, pk_kind: str):
    """The dominant rasterizer kernel's algorithmic FP32 rate against the ALU peak, plus the work
    counts it rests on."""
    visited, inside, instances = wl.count_pairs()
    dom = max(("blend", "bwd_raster"), key=lambda s: stages[s]["ms_per_launch"])
    clock_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak_tops = SMS * FP32_LANES_PER_SM * clock_mhz * 1e6 / 1e12
    dims = "2d" if wl.kind in ("2d", "2dsmall", "2dchol") else "3d"
    fp32_ops, mufu_ops = OPS_PER_PAIR[dims][dom]
    launch_s = stages[dom]["ms_per_launch"] * 1e-3
    pairs_per_launch = inside / wl.batch
    achieved = pairs_per_launch * fp32_ops / launch_s / 1e12
    kernel = {"2d": {"blend": "k_blend2d", "bwd_raster": "k_backward2d"},
              "3d": {"blend": "k_blend3d", "bwd_raster": "k_backward3d"}}[dims][dom]
    traffic = TRAFFIC_BYTES.get((wl.kind, kernel))
    roofline = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                "frac": achieved / peak_tops, "traffic": traffic,
                "peak_source": f"152 SMs x 128 FP32 lanes x {clock_mhz:.0f} MHz ({pk_kind} max SM clock)",
                "work": f"{pairs_per_launch:.0f} pairs inside the cutoff per launch x {fp32_ops:g} FP32 + "
                        f"{mufu_ops} MUFU ops",
                "mufu_frac": pairs_per_launch * mufu_ops / launch_s / (SMS * 16 * clock_mhz * 1e6)}
    return roofline, {"visited": visited, "inside": inside, "instances": instances}


def oracle_3d_sample(wl, budget_s: float):
    """The binary64 oracle on a bounded sample of one 3D step: forward and backward of the pixels of
    bands of rows (one camera or (camera, time) sample), scaled to every row and every sample of a
    step.  Each oracle call also pays a cost independent of the band (projection and depth order of
    every primitive, per-thread gradient accumulators): two band heights separate it from the cost
    per row, and a full frame is counted as one such call plus every row.  Returns (seconds per full
    step, sample description)."""
    import oracle
    import synth

    oracle.build()
    cam_i, t = wl.samples[0]
    cam = wl.cams[cam_i]
    p = wl.p if t is None else oracle.deform6d(wl.p, t).astype(np.float32)
    H, W = wl.H, wl.W

    def sample(rows):
        r0 = (H - rows) // 2
        pix = np.stack(np.meshgrid(np.arange(W), np.arange(r0, r0 + rows)), -1).reshape(-1, 2).astype(np.int32)
        t0 = time.perf_counter()
        oracle.render3d(p, cam, H, W, pixels=pix)
        t_f = time.perf_counter() - t0
        g = np.zeros((H, W, 3), np.float32)
        g[r0:r0 + rows] = synth.upstream_grad(rows, W, 5)
        t0 = time.perf_counter()
        oracle.grad3d(p, cam, H, W, g)
        t_b = time.perf_counter() - t0
        return t_f + t_b

    r1 = 1
    t1 = sample(r1)
    r2 = 4
    t2 = sample(r2)
    per_row = max(1e-6, (t2 - t1) / (r2 - r1))
    fixed = max(0.0, t1 - per_row * r1)
    r3 = int(min(H, max(r2 + 1, (budget_s - t1 - t2) / per_row)))
    t3 = sample(r3)
    per_row = max(1e-6, (t3 - t1) / (r3 - r1))
    fixed = max(0.0, t1 - per_row * r1)
    per_frame = fixed + per_row * H
    what = "(camera, time) sample" if t is not None else "view"
    desc = (f"forward and backward of bands of {r1}, {r2} and {r3} of {H} rows of one {what} "
            f"({t1 + t2 + t3:.1f} s of CPU work): {fixed:.2f} s per pass independent of the band plus "
            f"{per_row:.3f} s per row, scaled to {wl.batch} full frame{'s' if wl.batch > 1 else ''} per step")
    return per_frame * wl.batch, desc


def our_arm(args, rank: int, world: int, local_rank: int):
    import torch

    import synth

    from paper_2508_12615_gb300 import build

    dist = None
    if world > 1:
        import torch.distributed as dist

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = Workload(args.workload, dev)
    ctx = wl.ctx
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB of L2
    m = measure(wl, args.steps, args.warmup, flush, dist, world, dev, sample_clocks=rank == 0)
    stages = m["stages"]

    # the other configurations of the workload family, each measured the same way (fewer steps)
    others = []
    if args.workload == "2d" and not args.no_configs:
        for kind in ("2dsmall", "5d", "6d"):
            o = Workload(kind, dev)
            mo = measure(o, args.config_steps, args.warmup, flush, dist, world, dev, sample_clocks=rank == 0)
            others.append((o, mo))

    if rank != 0:
        return

    pk, pk_kind = peaks()
    roofline, pairs = roofline_of(wl, stages, pk, pk_kind)

    # the deformation network is a dense contraction on the tensor cores: per row and layer
    # 2 x out x in flops forward and twice that backward (dh = dz W and dW = dz^T x), so
    # 6 x sum(out x in) flops per row for one forward and backward; bf16 operands, fp32
    # accumulation, against the measured sustained bf16 rate (the network runs inside a long step)
    roofline_mlp = None
    if wl.kind == "6dmlp" and "mlp_fwd" in stages:
        rows = wl.p.shape[0]
        macs = sum(o * i for o, i in synth.MLP_SHAPES) * rows
        t_f = stages["mlp_fwd"]["ms_per_launch"] * 1e-3
        t_b = stages["mlp_bwd"]["ms_per_launch"] * 1e-3
        peak_bf16 = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0)))
        ach = 6.0 * macs / (t_f + t_b) / 1e12
        roofline_mlp = {"bound": "tensor", "kernel": "deformation network (encode, 9 layers, apply; forward and backward)",
                        "achieved": ach, "peak": peak_bf16, "unit": "TFLOP/s", "frac": ach / peak_bf16, "traffic": None,
                        "peak_source": f"{pk_kind} sustained bf16 (cuBLAS)",
                        "work": f"6 x {macs // rows} multiply-adds per row x {rows} rows",
                        "fwd_tflops": 2.0 * macs / t_f / 1e12, "bwd_tflops": 4.0 * macs / t_b / 1e12}

    configs = {}
    for o, mo in others:
        rl, pr = roofline_of(o, mo["stages"], pk, pk_kind)
        configs[o.name] = {"value": mo["value"], "unit": "iter/s" if o.batch == 1 else "steps/s",
                           "ms_per_step": mo["ms_per_step"], "steps": mo["steps"],
                           "samples_per_step": o.batch, "H": o.H, "W": o.W, "primitives": int(o.p.shape[0]),
                           "seed": o.seed, "fwd_mpix_s": mo["fwd_mpix_s"], "fwd_ms": mo["fwd_ms"], "e2e": mo["e2e"],
                           "gpu_launches": mo["gpu_launches"],
                           "stages_ms": {k: v["ms_per_launch"] for k, v in mo["stages"].items()},
                           "pairs": pr, "roofline": rl, "clocks": mo["clocks"], "cpu_baseline": None}

    # serving first: its latencies are host-loop sensitive, and the CPU baselines below occupy
    # every host core
    serving = None
    if world == 1 and not args.no_serving and wl.kind == "2d":
        serving = serving_run(args, dev)

    cpu = None
    if world == 1 and not args.no_cpu_baseline and wl.kind in ("2d", "2dsmall"):
        per_step, desc = oracle_step_sample(wl.p, wl.target, wl.H, wl.W, args.cpu_seconds)
        cpu = {"value": 1.0 / per_step, "unit": "iter/s", "cores": cpu_cores(), "kind": "oracle", "sample": desc}
    if world == 1 and not args.no_cpu_baseline:
        for o, _ in others:
            if o.kind == "2dsmall":
                per_step, desc = oracle_step_sample(o.p, o.target, o.H, o.W, args.config_cpu_seconds)
            else:
                per_step, desc = oracle_3d_sample(o, args.config_cpu_seconds)
            configs[o.name]["cpu_baseline"] = {"value": 1.0 / per_step, "unit": configs[o.name]["unit"],
                                               "cores": cpu_cores(), "kind": "oracle", "sample": desc}

    # the path's sort: its share of the step on this workload, and its bandwidth on a large input
    hbm = float(pk.get("hbm_gbs", 6800.0))
    sort = {"peak_gbs": hbm, "peak_source": f"{pk_kind} HBM copy bandwidth"}
    if "tile_sort" in stages:
        passes = max(1, (ceil_log2(((wl.W + 15) // 16) * ((wl.H + 15) // 16)) + 7) // 8)
        n_inst = pairs["instances"] / wl.batch
        b = n_inst * (4 + 16 * passes + 8)
        t = stages["tile_sort"]["ms_per_launch"] * 1e-3
        sort["tile_sort"] = {"pairs": n_inst, "passes": passes, "ms": t * 1e3, "algorithmic_bytes": b,
                             "gbs": b / t / 1e9, "frac": b / t / 1e9 / hbm}
    if world == 1 and not args.no_sort_bw:
        sort["large"] = sort_bandwidth(args, dev, ctx, hbm)

    line = {
        "metric": METRIC, "value": m["value"], "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "H": wl.H, "W": wl.W, "primitives": int(wl.p.shape[0]), "seed": wl.seed,
                   "samples_per_step": wl.batch, "l2": "flushed before every timed step (512 MB write)",
                   "replicas": world},
        "fwd_mpix_s": m["fwd_mpix_s"],
        "fwd_ms": m["fwd_ms"],
        "e2e": m["e2e"],
        "gpu_launches": m["gpu_launches"],
        "stages_ms": {k: v["ms_per_launch"] for k, v in stages.items()},
        "pairs": pairs,
        "roofline": roofline,
        **({"roofline_mlp": roofline_mlp} if roofline_mlp else {}),
        "cpu_baseline": cpu,
        "serving": serving,
        "sort": sort,
        "configs": configs,
        "clocks": m["clocks"],
        "wall_s_timed_region": m["wall_s_timed_region"],
    }
    print(json.dumps(line), flush=True)


def ceil_log2(x: int) -> int:
    return max(0, (int(x) - 1).bit_length())


def sort_bandwidth(args, dev, ctx, hbm_gbs: float) -> dict:
    """wipes_sort_pairs on args.sort_n random 32-bit keys with 32-bit values (4 passes of 8 bits):
    algorithmic bytes per pair = 4 (the histogram reads every key once) + 16 per pass (read key and
    value, write both), over the mean CUDA-event time of the sort call.  Every sort starts from the
    same unsorted input, copied in before the timed call."""
    import torch

    from paper_2508_12615_gb300 import State, sort_pairs

    n = int(args.sort_n)
    g = torch.Generator(device=dev).manual_seed(1239)
    keys0 = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device=dev, generator=g)
    vals0 = torch.arange(n, dtype=torch.int32, device=dev)
    keys, vals = torch.empty_like(keys0), torch.empty_like(vals0)
    st = State(ctx)
    times = []
    for it in range(13):
        keys.copy_(keys0)
        vals.copy_(vals0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sort_pairs(keys, vals, 32, state=st)
        b.record()
        torch.cuda.synchronize()
        if it >= 3:
            times.append(a.elapsed_time(b))
    ms = statistics.mean(times)
    passes = 4
    byts = n * (4 + 16 * passes)
    del st, keys0, vals0, keys, vals
    return {"pairs": n, "key_bits": 32, "passes": passes, "ms": ms, "algorithmic_bytes": byts,
            "gbs": byts / (ms * 1e-3) / 1e9, "frac": byts / (ms * 1e-3) / 1e9 / hbm_gbs}


def serving_run(args, dev):
    """64 resident scenes (2D and 3D, 10k-500k primitives), image sizes uniform over 256^2, 512^2,
    800^2 and 1920x1080, HBM budget 120 GB.  At the offered load of 2000 requests/s: p50/p99 latency
    and Mpix/s of the continuous-batching server, of the plain one-request-at-a-time path (one-frame
    render calls, every request prepared), and of the plain path over the same view cache as the
    server (one one-frame launch per request), all on the same trace.  Then above saturation
    (20,000 requests/s): the server against the plain path over the view cache.  Each arm starts on
    a fresh server (empty view cache)."""
    import gc

    import torch

    import synth
    from paper_2508_12615_gb300.serve import Server

    t = time.perf_counter()
    scenes, reqs = synth.serving_workload(n_scenes=64, rate=2000.0, seconds=args.serving_seconds)
    gen_s = time.perf_counter() - t

    def fresh():
        gc.collect()
        torch.cuda.synchronize(dev)
        return Server(scenes, device=dev.index, hbm_budget=120e9, max_batch=128, n_streams=2)

    fresh().run_batched(reqs[: min(len(reqs), 200)])  # warm the allocator and the kernels
    batched = fresh().run_batched(reqs).summary()
    plain = fresh().run_plain(reqs).summary()
    plain_cached = fresh().run_plain_cached(reqs).summary()
    _, sat = synth.serving_workload(n_scenes=64, rate=20000.0, seconds=args.saturation_seconds, seed=1239)
    sat_batched = fresh().run_batched(sat).summary()
    sat_plain_cached = fresh().run_plain_cached(sat).summary()
    gc.collect()
    return {"workload": f"64 scenes 10k-500k prims (2D:3D 1:1), Poisson 2000 req/s for {args.serving_seconds:g} s, "
                        "sizes {256^2, 512^2, 800^2, 1920x1080}, HBM budget 120 GB",
            "requests": int(len(reqs)), "batched": batched, "plain": plain, "plain_cached": plain_cached,
            "saturated": {"workload": f"the same scenes, Poisson 20000 req/s for {args.saturation_seconds:g} s "
                                      "(seed 1239), each arm from an empty view cache",
                          "requests": int(len(sat)), "batched": sat_batched, "plain_cached": sat_plain_cached},
            "scene_generation_s": gen_s}


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.only_sort:
        import torch

        import paper_2508_12615_gb300 as w

        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        pk, pk_kind = peaks()
        print(json.dumps(sort_bandwidth(args, dev, w.Context.get(dev.index), float(pk.get("hbm_gbs", 6800.0)))),
              flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    our_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""PyTorch-facing API of the wavelet rasterizer.

PyTorch supplies device memory, the current CUDA stream and autograd; every step of rendering and
differentiation runs in ``libwipes.so`` (see ``include/wipes.h``).  Parameter records are float32
CUDA tensors in the layouts documented there ([N,16] in 2D, [N,20] in 3D, [N,32] in 6D).

    img = render2d(params, H, W)            # differentiable, Render2D
    img = render3d(params, camera, H, W)    # differentiable, Render3D
    p3 = deform6d(params6, t)               # differentiable 6D time model
"""
from __future__ import annotations

import ctypes
import threading
import weakref

import torch

from . import _abi

P2D, P3D, P6D, P3D_SH = 16, 20, 32, 68


class Context:
    """One library context per CUDA device (cached)."""

    _cache: dict[int, "Context"] = {}
    _lock = threading.Lock()

    def __init__(self, device: int):
        self.device = device
        h = ctypes.c_void_p()
        _abi.call("wipes_create", device, ctypes.byref(h))
        self.handle = h
        self._free_states: list[State] = []

    @classmethod
    def get(cls, device) -> "Context":
        dev = torch.device(device).index if not isinstance(device, int) else device
        dev = torch.cuda.current_device() if dev is None else dev
        with cls._lock:
            if dev not in cls._cache:
                cls._cache[dev] = Context(dev)
            return cls._cache[dev]

    def acquire_state(self) -> "State":
        with self._lock:
            if self._free_states:
                return self._free_states.pop()
        return State(self)

    def release_state(self, st: "State") -> None:
        with self._lock:
            self._free_states.append(st)

    def __del__(self):
        try:
            if self.handle:
                _abi.lib().wipes_destroy(self.handle)
        except Exception:
            pass


class State:
    """Workspace of one forward pass, kept for its backward (wipes_state)."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _abi.call("wipes_state_create", ctx.handle, ctypes.byref(h))
        self.handle = h

    def info(self) -> dict:
        i = _abi.StateInfo()
        _abi.call("wipes_state_get_info", self.handle, ctypes.byref(i))
        return {k: getattr(i, k) for k, _ in _abi.StateInfo._fields_}

    def lists(self):
        """Sorted (tile ids, primitive ids) and the [n_tiles, 2] tile ranges of the last forward pass."""
        info = self.info()
        dev = torch.device("cuda", self.ctx.device)
        n = info["n_instances"]
        tiles = torch.empty(n, dtype=torch.int32, device=dev)
        prims = torch.empty(n, dtype=torch.int32, device=dev)
        ranges = torch.empty(info["tiles_x"] * info["tiles_y"], 2, dtype=torch.int32, device=dev)
        _abi.call("wipes_state_copy_lists", self.handle, _ptr(tiles), _ptr(prims), _ptr(ranges), _stream(dev))
        return tiles, prims, ranges

    def pixel_state(self):
        """3D: final transmittance [H,W] and per-pixel last processed list position [H,W]."""
        info = self.info()
        dev = torch.device("cuda", self.ctx.device)
        T = torch.empty(info["H"], info["W"], dtype=torch.float32, device=dev)
        last = torch.empty(info["H"], info["W"], dtype=torch.int32, device=dev)
        _abi.call("wipes_state_copy_pixel_state", self.handle, _ptr(T), _ptr(last), _stream(dev))
        return T, last

    def __del__(self):
        try:
            if self.handle:
                _abi.lib().wipes_state_destroy(self.handle)
        except Exception:
            pass


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check(t: torch.Tensor, cols: int, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != cols:
        raise ValueError(f"{name} must be float32 [N,{cols}], got {tuple(t.shape)} {t.dtype}")
    return t.contiguous()


def make_opts(dims: int, **overrides) -> _abi.Opts:
    """Default options for dims 2 or 3, with keyword overrides (bg takes a 3-sequence)."""
    o = _abi.default_opts(dims)
    for k, v in overrides.items():
        if k == "bg":
            for i in range(3):
                o.bg[i] = float(v[i])
        else:
            setattr(o, k, v)
    return o


def forward2d(params: torch.Tensor, H: int, W: int, opts: _abi.Opts | None = None, state: State | None = None,
              out: torch.Tensor | None = None) -> torch.Tensor:
    """Summed wavelet field [H,W,3] (no autograd)."""
    params = _check(params, P2D, "params")
    ctx = state.ctx if state is not None else Context.get(params.device)
    state = state or ctx.acquire_state()
    opts = opts or make_opts(2)
    if out is None:
        out = torch.empty(H, W, 3, dtype=torch.float32, device=params.device)
    _abi.call("wipes_render2d", ctx.handle, state.handle, _ptr(params), params.shape[0], H, W, ctypes.byref(opts),
              _ptr(out), _stream(params.device))
    return out


def forward3d(params: torch.Tensor, camera, H: int, W: int, opts: _abi.Opts | None = None,
              state: State | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Front-to-back blended image [H,W,3] (no autograd).  camera: 17 floats.  params [N,20], or
    [N,68] with spherical-harmonic colour (opts.sh_degree > 0)."""
    opts = opts or make_opts(3)
    params = _check(params, P3D_SH if opts.sh_degree else P3D, "params")
    ctx = state.ctx if state is not None else Context.get(params.device)
    state = state or ctx.acquire_state()
    cam = _abi.camera_struct(camera.tolist() if hasattr(camera, "tolist") else camera)
    if out is None:
        out = torch.empty(H, W, 3, dtype=torch.float32, device=params.device)
    _abi.call("wipes_render3d", ctx.handle, state.handle, _ptr(params), params.shape[0], ctypes.byref(cam), H, W,
              ctypes.byref(opts), _ptr(out), _stream(params.device))
    return out


def backward(state: State, params: torch.Tensor, grad_out: torch.Tensor,
             out: torch.Tensor | None = None) -> torch.Tensor:
    """dL/dparams for the last forward pass on ``state`` given dL/dimage."""
    grad_out = grad_out.contiguous()
    if out is None:
        out = torch.empty_like(params)
    _abi.call("wipes_render_backward", state.ctx.handle, state.handle, _ptr(params), _ptr(grad_out), _ptr(out),
              _stream(params.device))
    return out


def l2_loss(img: torch.Tensor, target: torch.Tensor, loss: torch.Tensor | None = None,
            grad: torch.Tensor | None = None, ctx: Context | None = None):
    """(mean squared error as a device scalar, its gradient with respect to img).  The call uses
    a small reduction buffer of its context (the device's default one unless ``ctx`` is given):
    calls on one context must not overlap on the GPU."""
    img = img.contiguous()
    target = target.contiguous()
    ctx = ctx or Context.get(img.device)
    if loss is None:
        loss = torch.empty((), dtype=torch.float32, device=img.device)
    if grad is None:
        grad = torch.empty_like(img)
    _abi.call("wipes_l2_loss", ctx.handle, _ptr(img), _ptr(target), img.numel(), _ptr(loss), _ptr(grad),
              _stream(img.device))
    return loss, grad


class _Lease:
    """Holds a pooled State for one autograd node; returns it to the pool when released or freed."""

    def __init__(self, ctx: Context):
        self.state = ctx.acquire_state()
        self._fin = weakref.finalize(self, ctx.release_state, self.state)

    def release(self):
        self._fin()


class Render2D(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, H, W, opts):
        lease = _Lease(Context.get(params.device))
        img = forward2d(params, H, W, opts, lease.state)
        ctx.lease = lease
        ctx.save_for_backward(params)
        return img

    @staticmethod
    def backward(ctx, grad):
        (params,) = ctx.saved_tensors
        g = backward(ctx.lease.state, params.contiguous(), grad)
        ctx.lease.release()
        return g, None, None, None


class Render3D(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, camera, H, W, opts):
        lease = _Lease(Context.get(params.device))
        img = forward3d(params, camera, H, W, opts, lease.state)
        ctx.lease = lease
        ctx.save_for_backward(params)
        return img

    @staticmethod
    def backward(ctx, grad):
        (params,) = ctx.saved_tensors
        g = backward(ctx.lease.state, params.contiguous(), grad)
        ctx.lease.release()
        return g, None, None, None, None


class Deform6D(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params6, t):
        params6 = _check(params6, P6D, "params6")
        out = torch.empty(params6.shape[0], P3D, dtype=torch.float32, device=params6.device)
        _abi.call("wipes_deform6d", _ptr(params6), params6.shape[0], float(t), _ptr(out), _stream(params6.device))
        ctx.t = float(t)
        ctx.save_for_backward(params6)
        return out

    @staticmethod
    def backward(ctx, grad):
        (params6,) = ctx.saved_tensors
        g6 = torch.empty_like(params6)
        grad = grad.contiguous()
        _abi.call("wipes_deform6d_backward", _ptr(params6), params6.shape[0], ctx.t, _ptr(grad), _ptr(g6), 0,
                  _stream(params6.device))
        return g6, None


def sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32, state: State | None = None) -> None:
    """Sort (key, value) pairs of 32-bit words in place, stably by the low ``key_bits`` bits of the
    key, with the path's radix sort.  ``keys`` and ``vals``: contiguous int32 or uint32 device
    tensors of the same length (the bits are taken as unsigned)."""
    for name, t in (("keys", keys), ("vals", vals)):
        if t.dtype not in (torch.int32, torch.uint32) or not t.is_cuda or not t.is_contiguous() or t.dim() != 1:
            raise ValueError(f"{name} must be a contiguous 1-D int32/uint32 CUDA tensor")
    if keys.numel() != vals.numel():
        raise ValueError("keys and vals must have the same length")
    st = state if state is not None else State(Context.get(keys.device))
    _abi.call("wipes_sort_pairs", st.ctx.handle, st.handle, _ptr(keys), _ptr(vals), keys.numel(), int(key_bits),
              _stream(keys.device.index))


def deform_mlp_param_count() -> int:
    """Number of float32 parameters of the 6D deformation network."""
    return int(_abi.lib().wipes_deform_mlp_param_count())


def deform_mlp(params3: torch.Tensor, t: float, theta: torch.Tensor, state: State | None = None,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """Deformed [N,20] records at time t from canonical ones through the network with parameters
    theta (no autograd); the activations stay in ``state`` for deform_mlp_backward."""
    params3 = _check(params3, P3D, "params3")
    theta = theta.contiguous()
    if theta.dtype != torch.float32 or theta.numel() != deform_mlp_param_count():
        raise ValueError("theta must be float32 with deform_mlp_param_count() entries")
    ctx = state.ctx if state is not None else Context.get(params3.device)
    state = state or ctx.acquire_state()
    if out is None:
        out = torch.empty_like(params3)
    _abi.call("wipes_deform_mlp", ctx.handle, state.handle, _ptr(params3), params3.shape[0], float(t), _ptr(theta),
              _ptr(out), _stream(params3.device))
    return out


def deform_mlp_backward(state: State, params3: torch.Tensor, grad_out: torch.Tensor,
                        grad_theta: torch.Tensor | None = None, grad_params3: torch.Tensor | None = None,
                        accumulate: bool = False):
    """(dL/dtheta, dL/dparams3) of the last deform_mlp on ``state`` given dL/d(deformed records)."""
    grad_out = grad_out.contiguous()
    dev = params3.device
    if grad_theta is None:
        grad_theta = torch.zeros(deform_mlp_param_count(), dtype=torch.float32, device=dev)
    if grad_params3 is None:
        grad_params3 = torch.zeros_like(params3)
    _abi.call("wipes_deform_mlp_backward", state.ctx.handle, state.handle, _ptr(params3), _ptr(grad_out),
              _ptr(grad_theta), _ptr(grad_params3), int(accumulate), _stream(dev))
    return grad_theta, grad_params3


class DeformMLP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params3, theta, t):
        lease = _Lease(Context.get(params3.device))
        out = deform_mlp(params3.contiguous(), t, theta, lease.state)
        ctx.lease = lease
        ctx.save_for_backward(params3)
        return out

    @staticmethod
    def backward(ctx, grad):
        (params3,) = ctx.saved_tensors
        g_theta, g_params = deform_mlp_backward(ctx.lease.state, params3.contiguous(), grad)
        ctx.lease.release()
        return g_params, g_theta, None


def render2d(params: torch.Tensor, H: int, W: int, opts: _abi.Opts | None = None) -> torch.Tensor:
    """Differentiable 2D render: image [H,W,3] from [N,16] wavelet records."""
    return Render2D.apply(params, H, W, opts)


def render3d(params: torch.Tensor, camera, H: int, W: int, opts: _abi.Opts | None = None) -> torch.Tensor:
    """Differentiable 3D render: image [H,W,3] from [N,20] wavelet records seen by ``camera``."""
    return Render3D.apply(params, camera, H, W, opts)


def deform_field(params3: torch.Tensor, theta: torch.Tensor, t: float) -> torch.Tensor:
    """Differentiable 6D deformation by the network: [N,20] canonical records at time t -> [N,20]."""
    return DeformMLP.apply(params3, theta, t)


def deform6d(params6: torch.Tensor, t: float) -> torch.Tensor:
    """Differentiable 6D time model: [N,32] records at time t -> [N,20] 3D records."""
    return Deform6D.apply(params6, t)

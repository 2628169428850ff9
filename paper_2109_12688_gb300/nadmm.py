"""Thin ctypes binding of ``libnadmm.so`` (C ABI declared in include/nadmm.h).

Functions carry the C names and only marshal arguments: torch tensors (or raw
integer addresses) become pointers, torch streams become ``cudaStream_t``.
Every step of the registration runs in the library's CUDA kernels; if the
library is missing this module raises instead of computing anything.
"""
from __future__ import annotations

import ctypes
import math
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnadmm.so")

NADMM_OK = 0
NADMM_ERR_INVALID_ARG = 1
NADMM_ERR_UNSUPPORTED_SIZE = 2
NADMM_ERR_ALIGNMENT = 3
NADMM_ERR_NO_WORKSPACE = 4
NADMM_ERR_CUDA = 5
NADMM_ERR_NONFINITE = 6
NADMM_ERR_TIMEOUT = 7
NADMM_ERR_NO_SAVED_FORWARD = 8
NADMM_FLAG_NO_GRAPH = 1
NADMM_FLAG_SAVE_FOR_BACKWARD = 2
NADMM_FLAG_LANE_MASK = 0xFC
NADMM_FLAG_FUSED_PENCIL = 0x100
NADMM_FLAG_PIPELINED_PLANE = 0x200
NADMM_FLAG_FOUR_PASS = 0x400
NADMM_FLAG_SLAB_PATH = 0x800
NADMM_FLAG_OUTER_Z2 = 0x1000
NADMM_FLAG_OUTER_Z4 = 0x2000
NADMM_FLAG_OUTER_MASK = 0x3000
NADMM_FLAG_SLAB_PAIRS = 0x4000
# plan bits nadmm_autotune chooses
PLAN_FLAGS = 0xFC | 0x100 | 0x400 | 0x800 | 0x3000


def NADMM_FLAG_LANE8(axis):
    return 1 << (2 + 2 * axis)


def NADMM_FLAG_LANE16(axis):
    return 2 << (2 + 2 * axis)

KERNEL_CLASSES = ("plane_first", "plane_k1", "plane", "plane_final", "pencil", "warp", "grad",
                  "bound", "compose", "slab_first", "slab_k1", "slab", "slab_final", "zslab")


class NadmmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


class nadmm_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("order_n", ctypes.c_int32), ("lambda_", ctypes.c_float),
                ("theta", ctypes.c_float), ("outer_iters", ctypes.c_int32),
                ("inner_iters", ctypes.c_int32), ("data_term", ctypes.c_int32),
                ("eps", ctypes.c_float), ("bound_kappa", ctypes.c_float),
                ("bound_delta", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("admm_tol", ctypes.c_float), ("warp_tol", ctypes.c_float),
                ("restart_eta", ctypes.c_float)]


_lib = None
_P = ctypes.c_void_p
_SIGS = {
    "nadmm_config_init": (None, [ctypes.POINTER(nadmm_config), ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_int32]),
    "nadmm_create": (ctypes.c_int, [ctypes.POINTER(nadmm_config), ctypes.POINTER(_P)]),
    "nadmm_destroy": (None, [_P]),
    "nadmm_workspace_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "nadmm_set_workspace": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "nadmm_set_params": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float]),
    "nadmm_register": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "nadmm_register_host": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "nadmm_get_status": (ctypes.c_int, [_P, _P]),
    "nadmm_create_batched_configs": (ctypes.c_int, [ctypes.POINTER(nadmm_config), ctypes.c_int32,
                                                    ctypes.POINTER(_P)]),
    "nadmm_get_restarts": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "nadmm_last_error": (ctypes.c_char_p, []),
    "nadmm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "nadmm_spectral_solve": (ctypes.c_int, [_P, _P, _P, _P]),
    "nadmm_admm_run": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                      _P, _P, _P]),
    "nadmm_linearise": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "nadmm_bound_compose": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "nadmm_jacobian_det": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "nadmm_spectral_solve_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                                     ctypes.c_int32, ctypes.c_int32,
                                                     ctypes.c_float, ctypes.c_float, _P, _P, _P]),
    "nadmm_register_profiled": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_float),
                                               ctypes.POINTER(ctypes.c_int32)]),
    "nadmm_create_batched": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(_P)]),
    "nadmm_batch_set_lanes": (ctypes.c_int, [_P, ctypes.c_int32]),
    "nadmm_batch_get_lanes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "nadmm_register_batched": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                              ctypes.POINTER(_P), _P]),
    "nadmm_backward": (ctypes.c_int, [_P] * 9),
    "nadmm_selftest_wait_timeout": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "nadmm_create_pyramid": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_P)]),
    "nadmm_register_pyramid": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "nadmm_backward_batched": (ctypes.c_int, [_P] + [ctypes.POINTER(_P)] * 7 + [_P]),
    "nadmm_autotune_workspace_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "nadmm_autotune": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, ctypes.POINTER(ctypes.c_uint32),
                                      ctypes.POINTER(ctypes.c_float)]),
    "nadmm_batch_set_pair_plan": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32]),
    "nadmm_get_iterations": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]),
    "nadmm_ssd_after_warp": (ctypes.c_int, [_P] * 6),
    "nadmm_ssd_after_warp_backward": (ctypes.c_int, [_P] * 9),
}


def load(path: str | None = None):
    """Load libnadmm.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build(); "
                          "there is no fallback implementation")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != NADMM_OK:
        lib = load()
        raise NadmmError(status, lib.nadmm_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---------------------------------------------------------------- C names
def nadmm_config_init(nx, ny, nz):
    cfg = nadmm_config()
    load().nadmm_config_init(ctypes.byref(cfg), nx, ny, nz)
    return cfg


def nadmm_create(cfg):
    h = _P()
    _check(load().nadmm_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def nadmm_create_batched(base, dims_list):
    n = len(dims_list)
    arr = (ctypes.c_int32 * (3 * n))(*[int(v) for d in dims_list for v in d])
    h = _P()
    _check(load().nadmm_create_batched(ctypes.byref(base), n, arr, ctypes.byref(h)))
    return h


def nadmm_create_batched_configs(cfgs):
    arr = (nadmm_config * len(cfgs))(*cfgs)
    h = _P()
    _check(load().nadmm_create_batched_configs(arr, len(cfgs), ctypes.byref(h)))
    return h


def nadmm_batch_set_lanes(h, lanes):
    _check(load().nadmm_batch_set_lanes(h, lanes))


def nadmm_batch_get_lanes(h):
    n = ctypes.c_int32(0)
    _check(load().nadmm_batch_get_lanes(h, ctypes.byref(n)))
    return n.value


def nadmm_register_batched(h, fixed, moving, u_out, stream=None):
    n = len(fixed)
    if len(moving) != n or len(u_out) != n:
        raise ValueError("fixed, moving and u_out need one entry per pair")
    arr = lambda xs: (_P * n)(*[_ptr(x) for x in xs])
    _check(load().nadmm_register_batched(h, arr(fixed), arr(moving), arr(u_out), _stream(stream)))


def nadmm_backward(h, fixed, moving, grad_u, grad_fixed, grad_moving, grad_lambda=None,
                   grad_theta=None, stream=None):
    _check(load().nadmm_backward(h, _ptr(fixed), _ptr(moving), _ptr(grad_u), _ptr(grad_fixed),
                                 _ptr(grad_moving), _ptr(grad_lambda), _ptr(grad_theta),
                                 _stream(stream)))


def nadmm_ssd_after_warp(h, fixed, moving, u, loss, stream=None):
    _check(load().nadmm_ssd_after_warp(h, _ptr(fixed), _ptr(moving), _ptr(u), _ptr(loss),
                                       _stream(stream)))


def nadmm_ssd_after_warp_backward(h, fixed, moving, u, grad_loss, grad_fixed, grad_moving,
                                  grad_u, stream=None):
    _check(load().nadmm_ssd_after_warp_backward(h, _ptr(fixed), _ptr(moving), _ptr(u),
                                                _ptr(grad_loss), _ptr(grad_fixed),
                                                _ptr(grad_moving), _ptr(grad_u), _stream(stream)))


def nadmm_selftest_wait_timeout(h, attempts, stream=None):
    _check(load().nadmm_selftest_wait_timeout(h, attempts, _stream(stream)))


def nadmm_create_pyramid(finest, outer, inner):
    """outer, inner: per-level counts, coarsest first."""
    n = len(outer)
    if len(inner) != n:
        raise ValueError("outer and inner need one entry per level")
    o = (ctypes.c_int32 * n)(*outer)
    i = (ctypes.c_int32 * n)(*inner)
    h = _P()
    _check(load().nadmm_create_pyramid(ctypes.byref(finest), n, o, i, ctypes.byref(h)))
    return h


def nadmm_register_pyramid(h, fixed, moving, u_out, stream=None):
    _check(load().nadmm_register_pyramid(h, _ptr(fixed), _ptr(moving), _ptr(u_out),
                                         _stream(stream)))


def nadmm_backward_batched(h, fixed, moving, grad_u, grad_fixed, grad_moving, grad_lambda=None,
                           grad_theta=None, stream=None):
    n = len(fixed)
    arr = lambda xs: None if xs is None else (_P * n)(*[_ptr(x) for x in xs])
    _check(load().nadmm_backward_batched(h, arr(fixed), arr(moving), arr(grad_u), arr(grad_fixed),
                                         arr(grad_moving), arr(grad_lambda), arr(grad_theta),
                                         _stream(stream)))


def nadmm_autotune_workspace_size(cfg):
    n = ctypes.c_size_t()
    _check(load().nadmm_autotune_workspace_size(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def nadmm_autotune(cfg, workspace, nbytes, stream=None):
    """Returns (flags with the fastest plan bits, its ms per ADMM iteration)."""
    f = ctypes.c_uint32()
    ms = ctypes.c_float()
    _check(load().nadmm_autotune(ctypes.byref(cfg), _ptr(workspace), nbytes, _stream(stream),
                                 ctypes.byref(f), ctypes.byref(ms)))
    return f.value, ms.value


def nadmm_batch_set_pair_plan(h, pair, plan_flags):
    _check(load().nadmm_batch_set_pair_plan(h, pair, plan_flags))


def nadmm_get_iterations(h, stream=None):
    o = ctypes.c_int32()
    a = ctypes.c_int32()
    _check(load().nadmm_get_iterations(h, _stream(stream), ctypes.byref(o), ctypes.byref(a)))
    return o.value, a.value


def nadmm_destroy(h):
    load().nadmm_destroy(h)


def nadmm_workspace_size(h):
    n = ctypes.c_size_t()
    _check(load().nadmm_workspace_size(h, ctypes.byref(n)))
    return n.value


def nadmm_set_workspace(h, ws, nbytes):
    _check(load().nadmm_set_workspace(h, _ptr(ws), nbytes))


def nadmm_set_params(h, lam, theta):
    _check(load().nadmm_set_params(h, lam, theta))


def nadmm_register(h, fixed, moving, u_out, stream=None):
    _check(load().nadmm_register(h, _ptr(fixed), _ptr(moving), _ptr(u_out), _stream(stream)))


def nadmm_register_host(h, fixed_host, moving_host, u_out_host, stream=None):
    _check(load().nadmm_register_host(h, _ptr(fixed_host), _ptr(moving_host), _ptr(u_out_host),
                                      _stream(stream)))


def nadmm_register_profiled(h, fixed, moving, u_out, stream=None):
    ms = (ctypes.c_float * len(KERNEL_CLASSES))()
    n = (ctypes.c_int32 * len(KERNEL_CLASSES))()
    _check(load().nadmm_register_profiled(h, _ptr(fixed), _ptr(moving), _ptr(u_out),
                                          _stream(stream), ms, n))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}


def nadmm_get_status(h, stream=None):
    return load().nadmm_get_status(h, _stream(stream))


def nadmm_get_restarts(h, stream=None):
    n = ctypes.c_int32(0)
    _check(load().nadmm_get_restarts(h, _stream(stream), ctypes.byref(n)))
    return n.value


def nadmm_last_error():
    return load().nadmm_last_error().decode()


def nadmm_status_string(status):
    return load().nadmm_status_string(status).decode()


def nadmm_spectral_solve(h, y, w, stream=None):
    _check(load().nadmm_spectral_solve(h, _ptr(y), _ptr(w), _stream(stream)))


def nadmm_spectral_solve_noalloc(nx, ny, nz, order_n, lam, theta, y, w, stream=None):
    _check(load().nadmm_spectral_solve_noalloc(nx, ny, nz, order_n, lam, theta, _ptr(y), _ptr(w),
                                               _stream(stream)))


def nadmm_admm_run(h, J, c, w_km1, w_km2, b_km1, b_km2, k, steps, w_out, b_out, stream=None):
    _check(load().nadmm_admm_run(h, _ptr(J), _ptr(c), _ptr(w_km1), _ptr(w_km2), _ptr(b_km1),
                                 _ptr(b_km2), k, steps, _ptr(w_out), _ptr(b_out), _stream(stream)))


def nadmm_linearise(h, fixed, moving, u, J, c, I1w_out=None, stream=None):
    _check(load().nadmm_linearise(h, _ptr(fixed), _ptr(moving), _ptr(u), _ptr(J), _ptr(c),
                                  _ptr(I1w_out), _stream(stream)))


def nadmm_bound_compose(h, w, u_in, u_out, scale_out=None, stream=None):
    _check(load().nadmm_bound_compose(h, _ptr(w), _ptr(u_in), _ptr(u_out), _ptr(scale_out),
                                      _stream(stream)))


def nadmm_jacobian_det(h, u, det=None, nonpositive=None, stream=None):
    _check(load().nadmm_jacobian_det(h, _ptr(u), _ptr(det), _ptr(nonpositive), _stream(stream)))


# ---------------------------------------------------------------- convenience
def make_config(dims, order_n=2, lam=10.0, theta=0.1, outer=10, inner=10, data_term=2,
                eps=1e-6, kappa=0.5, delta=1.0, flags=0, admm_tol=0.0, warp_tol=0.0,
                restart_eta=-1.0):
    """nadmm_config for dims = (nx, ny, nz); kappa/delta may be math.inf."""
    nx, ny, nz = dims
    cfg = nadmm_config_init(nx, ny, nz)
    cfg.order_n = order_n
    cfg.lambda_ = lam
    cfg.theta = theta
    cfg.outer_iters = outer
    cfg.inner_iters = inner
    cfg.data_term = data_term
    cfg.eps = eps
    cfg.bound_kappa = kappa if math.isfinite(kappa) else float("inf")
    cfg.bound_delta = delta if math.isfinite(delta) else float("inf")
    cfg.flags = flags
    cfg.admm_tol = admm_tol
    cfg.warp_tol = warp_tol
    cfg.restart_eta = restart_eta
    return cfg


def _require(t, n, what):
    """The kernels read or write exactly n float32 values through a device
    pointer: reject anything else before it reaches them."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{what}: a CUDA tensor is expected")
    if t.dtype != torch.float32:
        raise TypeError(f"{what}: float32 expected, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{what}: {n} values expected, got {t.numel()}")


class Registration:
    """A handle plus a torch-allocated device workspace (PyTorch is used for
    device memory only)."""

    def __init__(self, dims, device="cuda", requires_grad=False, autotune_cache=None,
                 tune=False, **kw):
        import torch
        self.dims = tuple(dims)
        if requires_grad:
            kw["flags"] = kw.get("flags", 0) | NADMM_FLAG_SAVE_FOR_BACKWARD
        if tune or autotune_cache:
            kw["flags"] = (kw.get("flags", 0) & ~PLAN_FLAGS) | autotune(
                self.dims, device, autotune_cache)
        self.cfg = make_config(self.dims, **kw)
        self.serial = 0  # forward passes run on this handle
        self.handle = nadmm_create(self.cfg)
        nbytes = nadmm_workspace_size(self.handle)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        nadmm_set_workspace(self.handle, self._ws_ptr, nbytes)

    def register(self, fixed, moving, u_out=None, stream=None):
        import torch
        nx, ny, nz = self.dims
        V = nx * ny * nz
        _require(fixed, V, "fixed")
        _require(moving, V, "moving")
        if u_out is None:
            u_out = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=fixed.device)
        _require(u_out, 3 * V, "u_out")
        if stream is None:
            stream = torch.cuda.current_stream(fixed.device)
        nadmm_register(self.handle, fixed, moving, u_out, stream)
        self.serial += 1
        return u_out

    def set_params(self, lam, theta):
        if (lam, theta) != (self.cfg.lambda_, self.cfg.theta):
            nadmm_set_params(self.handle, lam, theta)
            self.cfg.lambda_ = lam
            self.cfg.theta = theta

    def backward(self, fixed, moving, grad_u, stream=None):
        """Gradients (I0, I1, lambda, theta) of <grad_u, u> through the last
        forward pass; lambda/theta as 0-dim device tensors."""
        import torch
        nx, ny, nz = self.dims
        V = nx * ny * nz
        _require(fixed, V, "fixed")
        _require(moving, V, "moving")
        _require(grad_u, 3 * V, "grad_u")
        if stream is None:
            stream = torch.cuda.current_stream(fixed.device)
        g0 = torch.empty_like(fixed)
        g1 = torch.empty_like(moving)
        par = torch.zeros(8, dtype=torch.float32, device=fixed.device)  # [0]: lambda, [4]: theta
        nadmm_backward(self.handle, fixed, moving, grad_u.contiguous(), g0, g1, par.data_ptr(),
                       par.data_ptr() + 16, stream)
        return g0, g1, par[0], par[4]

    def close(self):
        if self.handle:
            nadmm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(dims, device="cuda", cache=None, **kw):
    """Plan bits (NADMM_FLAG_LANE*) for a grid: nadmm_autotune's choice,
    remembered in the JSON file `cache` (if given) under the key
    "nx,ny,nz|<SM count>|<device name>" so that a grid is timed once per GPU
    type.  Extra keywords shape the config as in make_config."""
    import json
    import torch
    dev = torch.device(device)
    props = torch.cuda.get_device_properties(dev)
    key = "%d,%d,%d|%d|%s" % (tuple(dims) + (props.multi_processor_count, props.name))
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            table = json.load(fh)
    if key in table:
        return int(table[key]["plan_flags"])
    cfg = make_config(tuple(dims), **kw)
    nbytes = nadmm_autotune_workspace_size(cfg)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    ptr = (ws.data_ptr() + 255) // 256 * 256
    flags, ms = nadmm_autotune(cfg, ptr, nbytes, torch.cuda.current_stream(dev))
    plan = flags & PLAN_FLAGS
    if cache:
        table[key] = {"plan_flags": plan, "ms_per_iteration": ms}
        with open(cache, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
    return plan


PAPER_V1_OUTER = (10, 10, 5)   # warpings per level, coarsest first (Sec. 4, first version)
PAPER_V1_INNER = (10, 5, 5)    # ADMM iterations per level


class PyramidRegistration(Registration):
    """A pyramid handle (coarsest level first in outer/inner) plus its workspace."""

    def __init__(self, dims, outer=PAPER_V1_OUTER, inner=PAPER_V1_INNER, device="cuda", **kw):
        import torch
        self.dims = tuple(dims)
        self.cfg = make_config(self.dims, **kw)
        self.handle = nadmm_create_pyramid(self.cfg, outer, inner)
        self.serial = 0
        nbytes = nadmm_workspace_size(self.handle)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        nadmm_set_workspace(self.handle, self._ws_ptr, nbytes)

    def register(self, fixed, moving, u_out=None, stream=None):
        import torch
        nx, ny, nz = self.dims
        V = nx * ny * nz
        _require(fixed, V, "fixed")
        _require(moving, V, "moving")
        if u_out is None:
            u_out = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=fixed.device)
        _require(u_out, 3 * V, "u_out")
        if stream is None:
            stream = torch.cuda.current_stream(fixed.device)
        nadmm_register_pyramid(self.handle, fixed, moving, u_out, stream)
        return u_out


class BatchedRegistration(Registration):
    """A batched handle (pairs of different grid sizes) plus its workspace."""

    def __init__(self, dims_list, device="cuda", lanes=None, requires_grad=False,
                 autotune_cache=None, tune=False, per_pair=None, **kw):
        """per_pair: optional list of dicts of make_config arguments that
        override kw for each pair (e.g. a regulariser order per pair)."""
        import torch
        self.dims_list = [tuple(d) for d in dims_list]
        if requires_grad:
            kw["flags"] = kw.get("flags", 0) | NADMM_FLAG_SAVE_FOR_BACKWARD
        self.cfg = make_config(self.dims_list[0], **kw)
        if per_pair is None:
            self.handle = nadmm_create_batched(self.cfg, self.dims_list)
        else:
            cfgs = [make_config(d, **{**kw, **extra}) for d, extra in zip(self.dims_list, per_pair)]
            self.handle = nadmm_create_batched_configs(cfgs)
        if lanes is not None:
            nadmm_batch_set_lanes(self.handle, lanes)
        if tune or autotune_cache:
            plans = {}
            for i, d in enumerate(self.dims_list):
                if d not in plans:
                    plans[d] = autotune(d, device, autotune_cache)
                nadmm_batch_set_pair_plan(self.handle, i, plans[d])
        nbytes = nadmm_workspace_size(self.handle)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        nadmm_set_workspace(self.handle, self._ws_ptr, nbytes)

    def _require_pairs(self, **lists):
        n = len(self.dims_list)
        for what, ts in lists.items():
            if len(ts) != n:
                raise ValueError(f"{what}: {n} tensors expected, got {len(ts)}")
            per = 3 if what in ("u_out", "grad_u") else 1
            for i, ((nx, ny, nz), t) in enumerate(zip(self.dims_list, ts)):
                _require(t, per * nx * ny * nz, f"{what}[{i}]")

    def register(self, fixed, moving, u_out=None, stream=None):
        import torch
        self._require_pairs(fixed=fixed, moving=moving)
        if u_out is None:
            u_out = [torch.empty((3, nz, ny, nx), dtype=torch.float32, device=f.device)
                     for (nx, ny, nz), f in zip(self.dims_list, fixed)]
        self._require_pairs(u_out=u_out)
        if stream is None:
            stream = torch.cuda.current_stream(fixed[0].device)
        nadmm_register_batched(self.handle, fixed, moving, u_out, stream)
        return u_out

    def backward(self, fixed, moving, grad_u, stream=None):
        """Per-pair gradients (I0, I1, lambda, theta) of <grad_u[i], u[i]>
        through the last nadmm_register_batched (handle made with
        requires_grad=True)."""
        import torch
        self._require_pairs(fixed=fixed, moving=moving, grad_u=grad_u)
        if stream is None:
            stream = torch.cuda.current_stream(fixed[0].device)
        g0 = [torch.empty_like(f) for f in fixed]
        g1 = [torch.empty_like(m) for m in moving]
        par = torch.zeros((len(fixed), 8), dtype=torch.float32, device=fixed[0].device)
        base = par.data_ptr()
        nadmm_backward_batched(self.handle, fixed, moving, [g.contiguous() for g in grad_u], g0, g1,
                               [base + 32 * i for i in range(len(fixed))],
                               [base + 32 * i + 16 for i in range(len(fixed))], stream)
        return g0, g1, par[:, 0], par[:, 4]


# ---------------------------------------------------------------- autograd
def _autograd():
    import torch

    class RegisterFn(torch.autograd.Function):
        """u = register(I0, I1; lambda, theta) with its reverse mode
        (nadmm_backward).  The handle must be created with requires_grad."""

        @staticmethod
        def forward(ctx, fixed, moving, lam, theta, reg):
            params = (float(lam), float(theta))
            reg.set_params(*params)
            fixed, moving = fixed.contiguous(), moving.contiguous()
            u = reg.register(fixed, moving)
            ctx.reg, ctx.params, ctx.serial = reg, params, reg.serial
            ctx.save_for_backward(fixed, moving)
            return u

        @staticmethod
        def backward(ctx, gu):
            fixed, moving = ctx.saved_tensors
            reg = ctx.reg
            if reg.serial != ctx.serial or (reg.cfg.lambda_, reg.cfg.theta) != ctx.params:
                reg.set_params(*ctx.params)  # the handle ran another forward since: redo ours
                reg.register(fixed, moving)
                ctx.serial = reg.serial
            g0, g1, gl, gt = reg.backward(fixed, moving, gu)
            return g0, g1, gl, gt, None

    class SSDFn(torch.autograd.Function):
        """L = 1/2 sum (I1 o (Id + u) - I0)^2 on the handle's grid."""

        @staticmethod
        def forward(ctx, fixed, moving, u, reg):
            fixed, moving, u = fixed.contiguous(), moving.contiguous(), u.contiguous()
            loss = torch.empty(4, dtype=torch.float32, device=fixed.device)
            nadmm_ssd_after_warp(reg.handle, fixed, moving, u, loss,
                                 torch.cuda.current_stream(fixed.device))
            ctx.reg = reg
            ctx.save_for_backward(fixed, moving, u)
            return loss[0]

        @staticmethod
        def backward(ctx, gL):
            fixed, moving, u = ctx.saved_tensors
            g0, g1, gu = torch.empty_like(fixed), torch.empty_like(moving), torch.empty_like(u)
            gl = torch.zeros(4, dtype=torch.float32, device=fixed.device)
            gl[0] = gL
            nadmm_ssd_after_warp_backward(ctx.reg.handle, fixed, moving, u, gl, g0, g1, gu,
                                          torch.cuda.current_stream(fixed.device))
            return g0, g1, gu, None

    return RegisterFn, SSDFn


_fns = None


def register(fixed, moving, lam, theta, reg):
    """Differentiable registration: u with gradients to fixed, moving and the
    0-dim tensors lam, theta (reg: Registration(..., requires_grad=True))."""
    global _fns
    if _fns is None:
        _fns = _autograd()
    return _fns[0].apply(fixed, moving, lam, theta, reg)


def ssd_after_warp(fixed, moving, u, reg):
    """Differentiable 1/2 sum (I1 o (Id + u) - I0)^2."""
    global _fns
    if _fns is None:
        _fns = _autograd()
    return _fns[1].apply(fixed, moving, u, reg)

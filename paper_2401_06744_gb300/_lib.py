"""ctypes binding of libdi.so (the C ABI in include/di.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Tensors are torch CUDA tensors (PyTorch provides device memory and streams);
outputs are allocated with torch on the input's device when not given.
There is no CPU fallback: if libdi.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdi.so")

OK, INVALID_ARG, EMPTY_MASK, OOM, NOT_CONVERGED, CUDA_ERROR, TIMEOUT = range(7)
STOP_ERROR_ESTIMATE, STOP_RELATIVE_RESIDUAL, STOP_FIXED_CYCLES = range(3)
PREC_FP32, PREC_FP16, PREC_BF16 = range(3)
SCHED_REDUCED_FMG, SCHED_FULL_FMG, SCHED_MULTILEVEL, SCHED_SINGLE = range(4)
SMOOTH_ORAS, SMOOTH_CG = range(2)
GRAPH_ON, GRAPH_OFF = range(2)
START_CASCADE, START_GIVEN = range(2)


class di_config(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("overlap", ctypes.c_int),
                ("local_iters", ctypes.c_int), ("coarse_iters", ctypes.c_int),
                ("pre", ctypes.c_int), ("post", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("min_cycles", ctypes.c_int),
                ("alpha", ctypes.c_float), ("downsample", ctypes.c_int),
                ("stop_rule", ctypes.c_int), ("profile", ctypes.c_int),
                ("precision", ctypes.c_int), ("schedule", ctypes.c_int),
                ("smoother", ctypes.c_int), ("graph", ctypes.c_int),
                ("start", ctypes.c_int), ("local_iters_coarse", ctypes.c_int),
                ("local_stop", ctypes.c_float), ("refine_fp64", ctypes.c_int),
                ("local_iters_cascade", ctypes.c_int)]


class di_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("levels_used", ctypes.c_int),
                ("cycles", ctypes.c_int), ("converged", ctypes.c_int),
                ("est_error", ctypes.c_float), ("rel_residual", ctypes.c_float * 4),
                ("unknowns", ctypes.c_longlong), ("status", ctypes.c_int)]


class di_plan_info(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("width", ctypes.c_int * 24),
                ("height", ctypes.c_int * 24), ("blocks_x", ctypes.c_int * 24),
                ("blocks_y", ctypes.c_int * 24), ("local_problems", ctypes.c_longlong),
                ("workspace_bytes", ctypes.c_longlong)]


class di_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("oras_l0_launches", ctypes.c_longlong),
                ("oras_l0_ms", ctypes.c_double), ("oras_l0_pixel_channels", ctypes.c_longlong),
                ("oras_l0_cg_steps", ctypes.c_longlong), ("oras_l0_tasks", ctypes.c_longlong),
                ("device_decodes", ctypes.c_longlong), ("oras_l0_prolong", ctypes.c_longlong),
                ("reserved", ctypes.c_longlong * 1)]


class di_image(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p), ("c", ctypes.c_void_p), ("width", ctypes.c_int),
                ("height", ctypes.c_int), ("channels", ctypes.c_int), ("tol", ctypes.c_float),
                ("u", ctypes.c_void_p), ("status", ctypes.c_int), ("cycles", ctypes.c_int)]


class di_tune_space(ctypes.Structure):
    _fields_ = [("blocks", ctypes.POINTER(ctypes.c_int)), ("nblocks", ctypes.c_int),
                ("overlaps", ctypes.POINTER(ctypes.c_int)), ("noverlaps", ctypes.c_int),
                ("local_iters", ctypes.POINTER(ctypes.c_int)), ("nlocal_iters", ctypes.c_int),
                ("smoothing", ctypes.POINTER(ctypes.c_int)), ("nsmoothing", ctypes.c_int),
                ("schedules", ctypes.POINTER(ctypes.c_int)), ("nschedules", ctypes.c_int)]


class di_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cycles", ctypes.c_int),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("footprint_bytes", ctypes.c_longlong), ("copy_in_ms", ctypes.c_double),
                ("wait_decode_ms", ctypes.c_double), ("decode_ms", ctypes.c_double),
                ("wait_out_ms", ctypes.c_double), ("copy_out_ms", ctypes.c_double)]


class DiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float

_SIGS = {
    "di_plan": (_I, [ctypes.POINTER(di_config), _I, _I, _I, ctypes.POINTER(di_plan_info)]),
    "di_create": (_I, [ctypes.POINTER(di_config), _I, ctypes.POINTER(_P)]),
    "di_destroy": (None, [_P]),
    "di_inpaint": (_I, [_P, _P, _P, _I, _I, _I, _F, _P, _P]),
    "di_inpaint_async": (_I, [_P, _P, _P, _I, _I, _I, _F, _P, _P]),
    "di_get_stats": (_I, [_P, ctypes.POINTER(di_stats)]),
    "di_get_profile": (_I, [_P, ctypes.POINTER(di_profile)]),
    "di_reset_profile": (_I, [_P]),
    "di_inpaint_batch": (_I, [ctypes.POINTER(di_config), _I, ctypes.POINTER(di_image), _I, _I,
                              _P]),
    "di_batch_create": (_I, [ctypes.POINTER(di_config), _I, ctypes.POINTER(di_image), _I,
                             ctypes.POINTER(_P)]),
    "di_batch_run": (_I, [_P, ctypes.POINTER(di_image), _I, _P]),
    "di_batch_destroy": (None, [_P]),
    "di_pool_create": (_I, [ctypes.POINTER(di_config), _I, _I, ctypes.POINTER(_P)]),
    "di_pool_inpaint": (_I, [_P, ctypes.POINTER(di_image), _I, _P]),
    "di_pool_destroy": (None, [_P]),
    "di_autotune": (_I, [ctypes.POINTER(di_config), _I, ctypes.POINTER(di_image), _I,
                         ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I,
                         ctypes.POINTER(di_config), ctypes.POINTER(ctypes.c_double)]),
    "di_autotune_space": (_I, [ctypes.POINTER(di_config), _I, ctypes.POINTER(di_image), _I,
                               ctypes.POINTER(di_tune_space), _I, ctypes.POINTER(di_config),
                               ctypes.POINTER(ctypes.c_double)]),
    "di_server_create": (_I, [ctypes.POINTER(di_config), _I, _I, ctypes.c_longlong,
                              ctypes.POINTER(_P)]),
    "di_server_submit": (_I, [_P, _P, _P, _I, _I, _I, _F, _P, ctypes.POINTER(ctypes.c_longlong)]),
    "di_server_wait": (_I, [_P, ctypes.c_longlong, ctypes.POINTER(di_request_info)]),
    "di_server_destroy": (None, [_P]),
    "di_status_string": (ctypes.c_char_p, [_I]),
    "di_last_error": (ctypes.c_char_p, [_P]),
    "di_mask_downsample": (_I, [_P, _I, _I, _P, _P]),
    "di_values_downsample": (_I, [_P, _P, _I, _I, _I, _P, _P, _I, _P]),
    "di_pyramid_level": (_I, [_P, _P, _I, _I, _I, _P, _P, _P, _I, _P, _P]),
    "di_residual_norm": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _P]),
    "di_residual_norm_noalloc": (_I, [_P, _P, _I, _P, _I, _I, _I, _P, _P, _P]),
    "di_restrict_residual": (_I, [_P, _P, _I, _P, _I, _I, _I, _P, _P, _I, _P]),
    "di_prolong": (_I, [_P, _P, _P, _I, _I, _I, _P, _I, _P]),
    "di_oras_iteration": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _I, _P, _P]),
    "di_prolong_oras_iteration": (_I, [_P, _P, _I, _P, _P, _I, _P, _I, _I, _I, _I, _P, _P]),
    "di_selftest_bounded_wait": (_I, [_I, _I, _P]),
}


def load():
    """Load libdi.so (build it first with paper_2401_06744_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libdi.so not built ({LIB_PATH}); run "
                                   "python -m paper_2401_06744_gb300.build")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def status_string(st: int) -> str:
    return load().di_status_string(st).decode()


def _check(st: int, ctx=None):
    if st != OK:
        msg = status_string(st)
        if ctx is not None and ctx._h:
            extra = load().di_last_error(ctx._h).decode()
            if extra:
                msg += f" ({extra})"
        raise DiError(st, msg)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _img(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if t.dim() == 2:
        t = t.unsqueeze(0)
    if t.dim() != 3 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous [C,H,W] or [H,W] tensor")
    return t


def _mask(t: torch.Tensor) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.uint8:
        raise TypeError("mask must be a uint8 CUDA tensor")
    if t.dim() != 2 or not t.is_contiguous():
        raise ValueError("mask must be a contiguous [H,W] tensor")
    return t


def make_config(**kw) -> di_config:
    cfg = di_config()
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def plan(width: int, height: int, channels: int, **config) -> dict:
    """Level sizes, block counts and workspace bytes of a solve (host only)."""
    cfg = make_config(**config)
    out = di_plan_info()
    _check(load().di_plan(ctypes.byref(cfg), int(width), int(height), int(channels),
                          ctypes.byref(out)))
    L = out.levels
    return {"levels": L, "sizes": [(out.width[i], out.height[i]) for i in range(L)],
            "blocks": [(out.blocks_x[i], out.blocks_y[i]) for i in range(L)],
            "local_problems": out.local_problems, "workspace_bytes": out.workspace_bytes}


class Context:
    """A decoder context (di_create / di_destroy) with its device workspace."""

    def __init__(self, device: int | None = None, **config):
        lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        self.config = make_config(**config)
        h = _P()
        self._h = None
        _check(lib.di_create(ctypes.byref(self.config), int(device), ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h:
            load().di_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the decoder -------------------------------------------------------
    def inpaint(self, f: torch.Tensor, c: torch.Tensor, tol: float = 0.05,
                out: torch.Tensor | None = None, stream=None, check: bool = True):
        """u with (C + (I - C) L) u = C f per channel; returns (u, status)."""
        f3 = _img(f, "f")
        c = _mask(c)
        C, H, W = f3.shape
        if c.shape != (H, W):
            raise ValueError("mask shape does not match f")
        u = torch.empty_like(f3) if out is None else _img(out, "out")
        st = load().di_inpaint(self._h, f3.data_ptr(), c.data_ptr(), W, H, C, float(tol),
                               u.data_ptr(), _stream(stream))
        if check and st not in (OK, NOT_CONVERGED):
            _check(st, self)
        res = u if f.dim() == 3 else u[0]
        return res, st

    def inpaint_async(self, f: torch.Tensor, c: torch.Tensor, tol: float = 0.05,
                      out: torch.Tensor | None = None, stream=None):
        """Enqueue the decode on `stream` and return u at once (di_inpaint_async);
        stats() waits for the work and gives its status."""
        f3 = _img(f, "f")
        c = _mask(c)
        C, H, W = f3.shape
        if c.shape != (H, W):
            raise ValueError("mask shape does not match f")
        u = torch.empty_like(f3) if out is None else _img(out, "out")
        st = load().di_inpaint_async(self._h, f3.data_ptr(), c.data_ptr(), W, H, C, float(tol),
                                     u.data_ptr(), _stream(stream))
        _check(st, self)
        return u if f.dim() == 3 else u[0]

    def stats(self) -> dict:
        s = di_stats()
        _check(load().di_get_stats(self._h, ctypes.byref(s)), self)
        return {"levels": s.levels, "levels_used": s.levels_used, "cycles": s.cycles,
                "converged": bool(s.converged), "est_error": s.est_error,
                "rel_residual": list(s.rel_residual), "unknowns": s.unknowns,
                "status": s.status}

    def profile(self) -> dict:
        pr = di_profile()
        _check(load().di_get_profile(self._h, ctypes.byref(pr)), self)
        return {"launches": pr.launches, "oras_l0_launches": pr.oras_l0_launches,
                "oras_l0_ms": pr.oras_l0_ms, "oras_l0_pixel_channels": pr.oras_l0_pixel_channels,
                "oras_l0_cg_steps": pr.oras_l0_cg_steps, "oras_l0_tasks": pr.oras_l0_tasks,
                "device_decodes": pr.device_decodes, "oras_l0_prolong": pr.oras_l0_prolong}

    def reset_profile(self):
        _check(load().di_reset_profile(self._h), self)

    # -- single steps needing a context -----------------------------------
    def residual_norm(self, u, b, c, rhs_zero=False, want_r=True, stream=None):
        u3, b3, c = _img(u, "u"), _img(b, "b"), _mask(c)
        C, H, W = u3.shape
        r = torch.empty_like(u3) if want_r else None
        n2 = torch.empty(C, dtype=torch.float64, device=u3.device)
        st = load().di_residual_norm(self._h, u3.data_ptr(), b3.data_ptr(), int(bool(rhs_zero)),
                                     c.data_ptr(), W, H, C, r.data_ptr() if want_r else None,
                                     n2.data_ptr(), _stream(stream))
        _check(st, self)
        return r, n2

    def oras_iteration(self, u_in, b, c, local_iters, rhs_zero=False, out=None, stream=None):
        u3, b3, c = _img(u_in, "u_in"), _img(b, "b"), _mask(c)
        C, H, W = u3.shape
        uo = torch.empty_like(u3) if out is None else _img(out, "out")
        st = load().di_oras_iteration(self._h, u3.data_ptr(), b3.data_ptr(), int(bool(rhs_zero)),
                                      c.data_ptr(), W, H, C, int(local_iters), uo.data_ptr(),
                                      _stream(stream))
        _check(st, self)
        return uo

    def prolong_oras_iteration(self, uH, u_in, b, c, local_iters, rhs_zero=False, out=None,
                               stream=None, mode=1):
        """One ORAS iteration from a prolonged start (u_in unchanged): mode 1
        u_in + P uH off the mask, mode 0 u_in on the mask and P uH off it."""
        uH3, u3, b3, c = _img(uH, "uH"), _img(u_in, "u_in"), _img(b, "b"), _mask(c)
        C, H, W = u3.shape
        uo = torch.empty_like(u3) if out is None else _img(out, "out")
        st = load().di_prolong_oras_iteration(self._h, uH3.data_ptr(), int(mode), u3.data_ptr(),
                                              b3.data_ptr(), int(bool(rhs_zero)), c.data_ptr(),
                                              W, H, C, int(local_iters), uo.data_ptr(),
                                              _stream(stream))
        _check(st, self)
        return uo


# -- single steps without a context -----------------------------------------

def mask_downsample(c, stream=None):
    c = _mask(c)
    H, W = c.shape
    cH = torch.empty(((H + 1) // 2, (W + 1) // 2), dtype=torch.uint8, device=c.device)
    _check(load().di_mask_downsample(c.data_ptr(), W, H, cH.data_ptr(), _stream(stream)))
    return cH


def values_downsample(c, b, cH, modified=True, stream=None):
    c, b3, cH = _mask(c), _img(b, "b"), _mask(cH)
    C, H, W = b3.shape
    bH = torch.empty((C, (H + 1) // 2, (W + 1) // 2), dtype=torch.float32, device=b3.device)
    _check(load().di_values_downsample(c.data_ptr(), b3.data_ptr(), W, H, C, cH.data_ptr(),
                                       bH.data_ptr(), int(bool(modified)), _stream(stream)))
    return bH


def pyramid_level(c, b=None, modified=True, stream=None):
    """di_pyramid_level: (cH, bH or None, packed cH words [hH, wpr] int32, unknown count)."""
    c = _mask(c)
    H, W = c.shape
    hH, wH = (H + 1) // 2, (W + 1) // 2
    wpr = (wH + 31) // 32 + 1
    cH = torch.empty((hH, wH), dtype=torch.uint8, device=c.device)
    bits = torch.empty((hH, wpr), dtype=torch.int32, device=c.device)
    unk = torch.zeros(1, dtype=torch.int64, device=c.device)
    if b is not None:
        b3 = _img(b, "b")
        C = b3.shape[0]
        bH = torch.empty((C, hH, wH), dtype=torch.float32, device=c.device)
        bp, bHp = b3.data_ptr(), bH.data_ptr()
    else:
        C, bH, bp, bHp = 1, None, None, None
    _check(load().di_pyramid_level(c.data_ptr(), bp, W, H, C, cH.data_ptr(), bHp,
                                   bits.data_ptr(), int(bool(modified)), unk.data_ptr(),
                                   _stream(stream)))
    return cH, bH, bits, unk


NOALLOC_PARTIALS = 131072


def residual_norm_noalloc(u, b, c, rhs_zero=False, want_r=True, stream=None):
    """di_residual_norm_noalloc: residual and squared norm per channel without a
    context; the library allocates nothing (the outputs here are the
    caller's tensors)."""
    u3, b3, c = _img(u, "u"), _img(b, "b"), _mask(c)
    C, H, W = u3.shape
    r = torch.empty_like(u3) if want_r else None
    n2 = torch.empty(C, dtype=torch.float64, device=u3.device)
    _check(load().di_residual_norm_noalloc(u3.data_ptr(), b3.data_ptr(), int(bool(rhs_zero)),
                                           c.data_ptr(), W, H, C,
                                           r.data_ptr() if want_r else None, n2.data_ptr(),
                                           _stream(stream)))
    return r, n2


def restrict_residual(u, b, c, cH, rhs_zero=False, fp64=False, stream=None):
    u3, b3, c, cH = _img(u, "u"), _img(b, "b"), _mask(c), _mask(cH)
    C, H, W = u3.shape
    rH = torch.empty((C, (H + 1) // 2, (W + 1) // 2), dtype=torch.float32, device=u3.device)
    _check(load().di_restrict_residual(u3.data_ptr(), b3.data_ptr(), int(bool(rhs_zero)),
                                       c.data_ptr(), W, H, C, cH.data_ptr(), rH.data_ptr(),
                                       int(bool(fp64)), _stream(stream)))
    return rH


def prolong(uH, c, mode, b=None, u=None, stream=None):
    """mode 0: returns c ? b : P uH; mode 1: u += P uH off the mask (in place)."""
    uH3, c = _img(uH, "uH"), _mask(c)
    C = uH3.shape[0]
    H, W = c.shape
    if mode == 0:
        b3 = _img(b, "b")
        out = torch.empty((C, H, W), dtype=torch.float32, device=uH3.device)
        bp = b3.data_ptr()
    else:
        out = _img(u, "u")
        bp = None
    _check(load().di_prolong(uH3.data_ptr(), bp, c.data_ptr(), W, H, C, out.data_ptr(),
                             int(mode), _stream(stream)))
    return out


# -- batched and served decoding ---------------------------------------------

def _images(items):
    """items: iterable of (f, c, tol[, out]) with CUDA tensors -> (array, outputs)."""
    items = list(items)
    arr = (di_image * max(1, len(items)))()
    outs = []
    for i, it in enumerate(items):
        f, c, tol = it[0], it[1], it[2]
        f3, c2 = _img(f, "f"), _mask(c)
        u = it[3] if len(it) > 3 and it[3] is not None else torch.empty_like(f3)
        C, H, W = f3.shape
        arr[i] = di_image(f3.data_ptr(), c2.data_ptr(), W, H, C, float(tol), u.data_ptr(), 0, 0)
        outs.append(u)
    return arr, outs


def inpaint_batch(items, device=None, concurrency=0, stream=None, **config):
    """Decode a list of (f, c, tol) on one GPU with overlapping worker slots.
    Returns (outputs, statuses, cycles)."""
    if device is None:
        device = torch.cuda.current_device()
    cfg = make_config(**config)
    arr, outs = _images(items)
    n = len(outs)
    load().di_inpaint_batch(ctypes.byref(cfg), int(device), arr, n, int(concurrency),
                            _stream(stream))
    return outs, [arr[i].status for i in range(n)], [arr[i].cycles for i in range(n)]


def selftest_bounded_wait(limit=4096, device=None, stream=None) -> int:
    """Run the bounded-wait self test (di_selftest_bounded_wait); returns the
    status, TIMEOUT when the wait ran out as designed."""
    if device is None:
        device = torch.cuda.current_device()
    return load().di_selftest_bounded_wait(int(device), int(limit), _stream(stream))


class Batch:
    """The batched form (di_batch_*): a fixed list of (f, c, tol[, out]) images
    decoded together, one kernel launch per step over every image, the whole
    batch one CUDA graph.  run() decodes the images' current contents."""

    def __init__(self, items, device=None, **config):
        if device is None:
            device = torch.cuda.current_device()
        self.config = make_config(**config)
        self._arr, self.outputs = _images(items)
        self._keep = list(items)
        self._n = len(self.outputs)
        h = _P()
        self._h = None
        _check(load().di_batch_create(ctypes.byref(self.config), int(device), self._arr, self._n,
                                      ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        """Decode the batch; returns (outputs, statuses, cycles)."""
        load().di_batch_run(self._h, self._arr, self._n, _stream(stream))
        return (self.outputs, [self._arr[i].status for i in range(self._n)],
                [self._arr[i].cycles for i in range(self._n)])

    def close(self):
        if self._h:
            load().di_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pool:
    """Persistent decoder slots for repeated batches (di_pool_*)."""

    def __init__(self, concurrency=4, device=None, **config):
        if device is None:
            device = torch.cuda.current_device()
        self.config = make_config(**config)
        h = _P()
        self._h = None
        _check(load().di_pool_create(ctypes.byref(self.config), int(device), int(concurrency),
                                     ctypes.byref(h)))
        self._h = h

    def inpaint(self, items, stream=None):
        """Decode a list of (f, c, tol); returns (outputs, statuses, cycles)."""
        arr, outs = _images(items)
        n = len(outs)
        load().di_pool_inpaint(self._h, arr, n, _stream(stream))
        return outs, [arr[i].status for i in range(n)], [arr[i].cycles for i in range(n)]

    def close(self):
        if self._h:
            load().di_pool_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(items, blocks=(8, 16, 32), overlaps=(1, 2, 4), local_iters=(), smoothing=(),
             schedules=(), reps=2, device=None, **config):
    """Fastest converging configuration on the sample (f, c, tol) list over
    block x overlap x local CG steps x V(k, k) smoothing x schedule (empty
    lists keep the base value): returns (config dict, ms per pass)."""
    if device is None:
        device = torch.cuda.current_device()
    base = make_config(**config)
    arr, _ = _images(items)

    def arr_of(v):
        v = list(v)
        return (ctypes.c_int * max(1, len(v)))(*v), len(v)

    sp = di_tune_space()
    keep = []
    for name, vals in (("blocks", blocks), ("overlaps", overlaps), ("local_iters", local_iters),
                       ("smoothing", smoothing), ("schedules", schedules)):
        a, k = arr_of(vals)
        keep.append(a)
        setattr(sp, name, ctypes.cast(a, ctypes.POINTER(ctypes.c_int)))
        setattr(sp, "n" + name, k)
    best = di_config()
    ms = ctypes.c_double()
    _check(load().di_autotune_space(ctypes.byref(base), int(device), arr, len(items),
                                    ctypes.byref(sp), int(reps), ctypes.byref(best),
                                    ctypes.byref(ms)))
    return {k: getattr(best, k) for k, _ in di_config._fields_}, ms.value


class Server:
    """Serving loop over host buffers (di_server_*): submit numpy arrays, wait
    for the result.  Requests overlap on the GPU across `slots` worker slots and
    are admitted by device footprint within `mem_budget` bytes (0 = unlimited)."""

    def __init__(self, slots=4, mem_budget=0, device=None, **config):
        if device is None:
            device = torch.cuda.current_device()
        self.config = make_config(**config)
        h = _P()
        self._h = None
        _check(load().di_server_create(ctypes.byref(self.config), int(device), int(slots),
                                       int(mem_budget), ctypes.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, f, c, tol=0.05, out=None):
        """Queue one request.  f [C,H,W] (or [H,W]) float32 and c [H,W] uint8 are
        host arrays (numpy, or CPU tensors, e.g. pinned ones, whose memory is
        used in place); out (optional, same shape as f) receives u."""
        import numpy as np

        def host(a, dt):
            if isinstance(a, torch.Tensor):
                a = a.numpy()
            return np.ascontiguousarray(a, dtype=dt)

        f = host(f, np.float32)
        if f.ndim == 2:
            f = f[None]
        c = host(c, np.uint8)
        C, H, W = f.shape
        u = np.empty_like(f) if out is None else host(out, np.float32).reshape(f.shape)
        t = ctypes.c_longlong()
        _check(load().di_server_submit(self._h, f.ctypes.data, c.ctypes.data, W, H, C, float(tol),
                                       u.ctypes.data, ctypes.byref(t)))
        self._live[t.value] = (f, c, u)
        return t.value

    def wait(self, ticket):
        info = di_request_info()
        st = load().di_server_wait(self._h, int(ticket), ctypes.byref(info))
        f, c, u = self._live.pop(ticket)
        return u, {"status": st, "cycles": info.cycles, "latency_ms": info.latency_ms,
                   "queue_ms": info.queue_ms, "footprint_bytes": info.footprint_bytes,
                   "stages_ms": {"copy_in": info.copy_in_ms, "wait_decode": info.wait_decode_ms,
                                 "decode": info.decode_ms, "wait_out": info.wait_out_ms,
                                 "copy_out": info.copy_out_ms}}

    def close(self):
        if self._h:
            load().di_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""CPU oracle for homogeneous diffusion inpainting.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this package; the product path never
does, and it shares no code with the CUDA path.

* `cg_inpaint` solves (C + (I - C) L) u = C f exactly (up to FP64 CG with
  relative residual 1e-12) on the reduced SPD system (Section 2.2); this is the
  result the GPU solver must reach.  It is plain C (cg_oracle.c) built with
  gcc + OpenMP and called through ctypes.
* `method` restates every step of the reduced-FMG ORAS method in numpy FP64
  (pyramid, transfers, block tiling, weights, local solves, ORAS, V-cycle).

Parity status: `cg_inpaint` and every function of `method` are pinned by the
CPU tests (closed forms, invariants, dense direct solves, brute force, the
block count and level count the paper prints).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import method  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libcg_oracle.so")
_SRC = os.path.join(_HERE, "cg_oracle.c")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "invalid argument", 2: "empty mask", 3: "out of memory",
          4: "not converged"}


def build(force: bool = False) -> str:
    """Compile cg_oracle.c into oracle/_build/libcg_oracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC,
                        "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.oracle_cg_inpaint.restype = ctypes.c_int
            lib.oracle_cg_inpaint.argtypes = [
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def cg_inpaint(f: np.ndarray, c: np.ndarray, rel_tol: float = 1e-12,
               max_iter: int = 2_000_000, info: dict | None = None) -> np.ndarray:
    """Exact inpainting u (float64, same shape as f) of f [C,H,W] or [H,W]
    known on mask c [H,W].  Raises OracleError on invalid input / empty mask."""
    lib = _load()
    f = np.asarray(f, dtype=np.float32)
    squeeze = f.ndim == 2
    if squeeze:
        f = f[None]
    f = np.ascontiguousarray(f)
    C, H, W = f.shape
    c = np.ascontiguousarray(np.asarray(c).astype(np.uint8))
    if c.shape != (H, W):
        raise OracleError("mask shape does not match image")
    u = np.empty((C, H, W), dtype=np.float64)
    iters = np.zeros(C, dtype=np.int32)
    relres = np.zeros(C, dtype=np.float64)
    st = lib.oracle_cg_inpaint(f.ctypes.data, c.ctypes.data, W, H, C, float(rel_tol),
                               int(max_iter), u.ctypes.data, iters.ctypes.data,
                               relres.ctypes.data)
    if info is not None:
        info["status"] = STATUS.get(st, str(st))
        info["iters"] = iters.tolist()
        info["relres"] = relres.tolist()
    if st not in (0, 4):
        raise OracleError(STATUS.get(st, str(st)))
    if st == 4:
        raise OracleError(f"CG did not reach rel_tol={rel_tol}: {relres.tolist()}")
    return u[0] if squeeze else u

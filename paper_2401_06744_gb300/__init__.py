"""GB300-native homogeneous diffusion inpainting decoder.

Solves (C + (I - C) L) u = C f per colour channel (Kaemper, Chizhov, Weickert,
"Efficient Parallel Algorithms for Inpainting-Based Representations of 4K
Images - Part I", Section 2.2) by reduced full multigrid (Section 4.2) with an
optimized restricted additive Schwarz block smoother (Section 3, Algorithm 2),
in hand-written CUDA kernels for sm_103a behind the C ABI of include/di.h.

    import torch, paper_2401_06744_gb300 as di
    ctx = di.Context()
    u, status = ctx.inpaint(f_cuda_float32_CHW, mask_cuda_uint8_HW, tol=0.05)
"""
from ._lib import (  # noqa: F401
    CUDA_ERROR, EMPTY_MASK, INVALID_ARG, NOT_CONVERGED, OK, OOM, PREC_BF16, PREC_FP16, PREC_FP32,
    STOP_ERROR_ESTIMATE, SCHED_REDUCED_FMG, SCHED_FULL_FMG, SCHED_MULTILEVEL, SCHED_SINGLE,
    SMOOTH_ORAS, SMOOTH_CG, GRAPH_ON, GRAPH_OFF, START_CASCADE, START_GIVEN,
    STOP_FIXED_CYCLES, STOP_RELATIVE_RESIDUAL, TIMEOUT, Context, DiError, LIB_PATH,
    exported_symbols, load, mask_downsample, plan, prolong, pyramid_level, residual_norm_noalloc,
    restrict_residual, status_string, values_downsample, inpaint_batch, autotune, Server, Pool, Batch,
    selftest_bounded_wait)

__all__ = ["Context", "DiError", "load", "plan", "mask_downsample", "values_downsample",
           "residual_norm_noalloc", "inpaint_batch", "autotune", "Server", "Pool", "Batch",
           "restrict_residual", "prolong", "status_string", "exported_symbols", "LIB_PATH"]

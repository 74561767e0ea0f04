"""di_residual_norm_noalloc: the residual + squared-norm step for callers that
cannot allocate device memory when they call it (decoders with a device
footprint fixed up front, code running while another component owns the
device allocator, paths that cannot take the device-wide synchronisation of
cudaFree).  It must give the same results as di_residual_norm, which takes its
reduction scratch from a context's workspace.

This file is collected last on purpose: a failure here comes after every other
test has run."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import method as M

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def di():
    from paper_2401_06744_gb300 import build as b

    b.build()
    import paper_2401_06744_gb300 as di

    di.load()
    return di


def _case(h, w, C, d, seed):
    g = np.random.default_rng(seed)
    f = g.uniform(0, 255, size=(C, h, w)).astype(np.float32)
    c = (g.random((h, w)) < d).astype(np.uint8)
    c[0, 0] = 1
    u = np.where(c.astype(bool), f, g.uniform(0, 255, f.shape)).astype(np.float32)
    b = np.where(c.astype(bool), f, g.normal(size=f.shape)).astype(np.float32)
    return u, b, c


@pytest.mark.gpu
def test_noalloc_matches_context_entry_point_twice(di):
    # two calls in a row on different shapes: the shared scratch keeps the
    # first call's partial sums, which the second must not pick up.  Each
    # result is compared with the context entry point and with the oracle's
    # FP64 residual r = b - A u (Algorithm 2 step 1, eq. 2.6) and its squared
    # 2-norm per channel.
    cases = [((333, 171, 3), True, 1), ((1080, 1920, 1), False, 2)]
    with di.Context() as ctx:
        for (h, w, C), rhs_zero, seed in cases:
            u, b, c = _case(h, w, C, 0.05, seed)
            ut, bt, ct = (torch.from_numpy(a).to(DEV) for a in (u, b, c))
            r_ref, n_ref = ctx.residual_norm(ut, bt, ct, rhs_zero=rhs_zero)
            r_na, n_na = di.residual_norm_noalloc(ut, bt, ct, rhs_zero=rhs_zero)
            torch.cuda.synchronize()
            assert torch.isfinite(r_na).all()
            assert (r_na - r_ref).abs().max().item() <= 2e-4
            assert np.allclose(n_na.cpu().numpy(), n_ref.cpu().numpy(), rtol=1e-5, atol=1e-6)
            # b is read only on the mask when rhs_zero is set (b = C f there)
            rhs = M.rhs(b, c) if rhs_zero else b
            r_or = M.residual(u, rhs, c)
            assert np.abs(r_na.cpu().numpy() - r_or).max() <= 2e-4
            assert np.allclose(n_na.cpu().numpy(), (r_or ** 2).sum(axis=(1, 2)), rtol=1e-5,
                               atol=1e-6)


def test_noalloc_rejects_sizes_beyond_its_scratch_before_touching_the_gpu(di):
    # ceil(4096/32) * ceil(2304/8) * 4 = 147456 > DI_NOALLOC_PARTIALS: the call
    # must fail with an argument error without launching anything, so dummy
    # (never dereferenced) pointers are safe here, with or without a GPU
    lib = di.load()
    fake = ctypes.c_void_p(16)
    norm = ctypes.c_void_p(32)
    st = lib.di_residual_norm_noalloc(fake, fake, 1, fake, 4096, 2304, 4, None, norm, None)
    assert st == di.INVALID_ARG

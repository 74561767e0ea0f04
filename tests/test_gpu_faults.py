"""Failure detection on the GPU without a fault: the bounded device-side wait
of the block kernel runs out on a barrier that nothing completes, the host
reads the status, and the device and existing contexts stay usable."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def di():
    from paper_2401_06744_gb300 import build as b

    b.build()
    import paper_2401_06744_gb300 as di

    di.load()
    return di


def _decode(ctx, f, c):
    u, st = ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), tol=0.05)
    torch.cuda.synchronize()
    return u.cpu().numpy(), st


def test_bounded_wait_runs_out_and_the_device_stays_usable(di):
    f, c = synth.make_case(128, 96, 2, 0.05, "edge", 3)
    ref = oracle.cg_inpaint(f, c)
    with di.Context() as ctx:
        u0, st0 = _decode(ctx, f, c)
        assert st0 == di.OK
        for limit in (1, 64, 4096):
            assert di.selftest_bounded_wait(limit) == di.TIMEOUT
        s = torch.cuda.Stream(DEV)
        assert di.selftest_bounded_wait(256, stream=s) == di.TIMEOUT
        u1, st1 = _decode(ctx, f, c)  # the same context afterwards
    assert st1 == di.OK and np.array_equal(u0, u1)
    assert np.abs(u1.astype(np.float64) - ref).max() <= 0.05


def test_bounded_wait_rejects_bad_limit(di):
    assert di.selftest_bounded_wait(0) == di.INVALID_ARG

"""Given initial iterates (cfg.start = DI_START_GIVEN): the cascade is skipped
and the cycles start from the caller's u, e.g. the previous frame of a video
with a fixed mask.  The fixed point is the same system's solution, so every
result must stay within the decoder's tolerance of the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
TOL = 0.05


@pytest.fixture(scope="module")
def di():
    from paper_2401_06744_gb300 import build as b

    b.build()
    import paper_2401_06744_gb300 as di

    di.load()
    return di


def _decode(ctx, f, c, u0=None):
    ft, ct = torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV)
    out = torch.from_numpy(u0.astype(np.float32)).to(DEV) if u0 is not None else torch.empty_like(ft)
    _, st = ctx.inpaint(ft, ct, tol=TOL, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st, ctx.stats()


def test_start_from_solution_stops_after_one_cycle(di):
    f, c = synth.make_case(192, 120, 3, 0.04, "edge", 17)
    ref = oracle.cg_inpaint(f, c)
    with di.Context(start=di.START_GIVEN) as ctx:
        u, st, stats = _decode(ctx, f, c, ref)
    assert st == di.OK and stats["cycles"] == 1
    assert np.abs(u.astype(np.float64) - ref).max() <= TOL
    assert np.array_equal(u[:, c == 1], f[:, c == 1])


def test_start_values_on_the_mask_are_replaced(di):
    f, c = synth.make_case(96, 64, 2, 0.05, "uniform", 5)
    ref = oracle.cg_inpaint(f, c)
    g = np.random.default_rng(1)
    u0 = g.uniform(-1000, 1000, f.shape)  # wrong everywhere, also on the mask
    with di.Context(start=di.START_GIVEN, max_cycles=64) as ctx:
        u, st, _ = _decode(ctx, f, c, u0)
    assert st == di.OK
    assert np.array_equal(u[:, c == 1], f[:, c == 1])
    assert np.abs(u.astype(np.float64) - ref).max() <= TOL


@pytest.mark.parametrize("kind", ["edge", "uniform"])
def test_video_warm_start_matches_oracle(di, kind):
    # a moving disk: the previous frame is a good start away from the disk and
    # a poor one on its edge; every frame must still meet the tolerance
    seq, c = synth.make_video(320, 180, 3, 0.04, kind, 23, frames=5, speed=2.0)
    with di.Context() as cold, di.Context(start=di.START_GIVEN) as warm:
        prev = None
        for f in seq:
            ref = oracle.cg_inpaint(f, c)
            uc, stc, _ = _decode(cold, f, c)
            assert stc == di.OK
            assert np.abs(uc.astype(np.float64) - ref).max() <= TOL
            if prev is None:
                prev = uc
                continue
            uw, stw, _ = _decode(warm, f, c, prev)
            assert stw == di.OK
            assert np.abs(uw.astype(np.float64) - ref).max() <= TOL
            assert np.array_equal(uw[:, c == 1], f[:, c == 1])
            prev = uw


def test_static_video_warm_start_needs_one_cycle(di):
    # identical frames: the previous result is already converged
    seq, c = synth.make_video(256, 160, 3, 0.04, "edge", 29, frames=3, speed=0.0)
    with di.Context() as cold, di.Context(start=di.START_GIVEN) as warm:
        u0, st, s0 = _decode(cold, seq[0], c)
        assert st == di.OK
        u1, st, s1 = _decode(warm, seq[1], c, u0)
        assert st == di.OK and s1["cycles"] == 1 <= s0["cycles"]
        assert np.abs(u1 - u0).max() <= TOL

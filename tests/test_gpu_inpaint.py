"""GPU parity of the whole decoder (di_inpaint) against the FP64 CG oracle.

Bar: max-abs <= 0.05 and RMS <= 0.01 gray levels on the 0-255 scale, the
accuracy the decoder is specified to reach; mask pixels exact."""
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


def _run(di, f, c, tol=TOL, **cfg):
    fn = f.copy()
    fn[:, c == 0] = np.nan  # canaries: f off the mask must never be read
    with di.Context(**cfg) as ctx:
        u, st = ctx.inpaint(torch.from_numpy(fn).to(DEV), torch.from_numpy(c).to(DEV), tol=tol)
        torch.cuda.synchronize()
        stats = ctx.stats()
    return u.cpu().numpy(), st, stats


def _check(u, f, c, ref, tol=TOL):
    err = np.abs(u.astype(np.float64) - ref)
    assert np.isfinite(u).all()
    assert err.max() <= tol, err.max()
    assert np.sqrt((err ** 2).mean()) <= 0.01
    assert np.array_equal(u[:, c == 1], f[:, c == 1])


def test_256_uniform_4pct(di):
    # 256x256 single channel, uniform 4 % mask: the small parity workload
    f, c = synth.make_case(256, 256, 1, 0.04, "uniform", 2024)
    ref = oracle.cg_inpaint(f, c)
    u, st, stats = _run(di, f, c)
    assert st == di.OK, stats
    _check(u, f, c, ref)
    assert stats["levels"] == 4


@pytest.mark.parametrize("w,h,C,d,kind", [
    (512, 384, 3, 0.10, "edge"), (640, 360, 3, 0.04, "edge"), (640, 360, 3, 0.01, "edge"),
    (500, 300, 2, 0.04, "uniform"), (333, 171, 1, 0.01, "uniform"), (1024, 576, 3, 0.005, "edge"),
])
def test_synthetic_cases(di, w, h, C, d, kind):
    f, c = synth.make_case(w, h, C, d, kind, w + h)
    ref = oracle.cg_inpaint(f, c)
    u, st, stats = _run(di, f, c)
    assert st == di.OK, stats
    _check(u, f, c, ref)


@pytest.mark.parametrize("B,o,K", [(16, 4, 8), (16, 2, 8), (8, 2, 6), (8, 4, 6), (32, 4, 8),
                                   (16, 1, 8)])
def test_block_configs(di, B, o, K):
    f, c = synth.make_case(300, 200, 2, 0.03, "uniform", B * 10 + o)
    ref = oracle.cg_inpaint(f, c)
    u, st, stats = _run(di, f, c, block=B, overlap=o, local_iters=K, max_cycles=40)
    assert st == di.OK, stats
    _check(u, f, c, ref)


@pytest.mark.parametrize("w,h", [(1, 1), (1, 40), (40, 1), (3, 5), (32, 32), (33, 31),
                                 (65, 2), (2, 65)])
def test_tiny_and_degenerate_shapes(di, w, h):
    f, c = synth.make_case(w, h, 2, 0.2, "uniform", w * 100 + h)
    ref = oracle.cg_inpaint(f, c)
    u, st, stats = _run(di, f, c)
    assert st == di.OK, stats
    _check(u, f, c, ref)


def test_single_known_pixel_gives_constant(di):
    f = np.zeros((1, 90, 70), np.float32)
    c = np.zeros((90, 70), np.uint8)
    c[10, 60] = 1
    f[0, 10, 60] = 123.0
    u, st, _ = _run(di, f, c)
    assert st == di.OK
    assert np.abs(u - 123.0).max() <= TOL


def test_fully_known_mask_copies_f(di):
    f, _ = synth.make_case(50, 40, 3, 0.1, "uniform", 3)
    c = np.ones((40, 50), np.uint8)
    u, st, stats = _run(di, f, c)
    assert st == di.OK and stats["levels_used"] == 0
    assert np.array_equal(u, f)


def test_two_column_closed_form(di):
    # u is linear in x between two known columns, constant outside
    h, w, a, b = 64, 200, 20, 170
    f = np.zeros((1, h, w), np.float32)
    f[0, :, a], f[0, :, b] = 10.0, 250.0
    c = np.zeros((h, w), np.uint8)
    c[:, a] = c[:, b] = 1
    u, st, _ = _run(di, f, c)
    assert st == di.OK
    x = np.arange(w, dtype=np.float64)
    ref = np.where(x <= a, 10.0, np.where(x >= b, 250.0, 10.0 + (x - a) * 240.0 / (b - a)))
    assert np.abs(u[0] - ref[None, :]).max() <= TOL


def test_max_principle_and_determinism(di):
    f, c = synth.make_case(400, 300, 3, 0.02, "edge", 77)
    u1, st1, _ = _run(di, f, c)
    u2, st2, _ = _run(di, f, c)
    assert st1 == st2 == di.OK
    assert np.array_equal(u1, u2)
    for ch in range(3):
        known = f[ch][c == 1]
        assert u1[ch].min() >= known.min() - TOL and u1[ch].max() <= known.max() + TOL


def test_relative_residual_stop_rule(di):
    # the paper's criterion (Section 5.2); the reported residual meets it
    f, c = synth.make_case(300, 260, 1, 0.04, "uniform", 8)
    u, st, stats = _run(di, f, c, tol=1e-3, stop_rule=di.STOP_RELATIVE_RESIDUAL)
    assert st == di.OK
    assert 0 <= stats["rel_residual"][0] <= 1e-3
    from oracle import method as M
    r = M.residual(u.astype(np.float64), M.rhs(f, c), c)
    b = M.rhs(f, c)
    assert np.sqrt((r ** 2).sum() / (b ** 2).sum()) <= 1.1e-3


def test_errors(di):
    f, c = synth.make_case(40, 30, 1, 0.1, "uniform", 1)
    with di.Context() as ctx:
        ft = torch.from_numpy(f).to(DEV)
        with pytest.raises(di.DiError) as e:
            ctx.inpaint(ft, torch.zeros((30, 40), dtype=torch.uint8, device=DEV))
        assert e.value.status == di.EMPTY_MASK
        ct = torch.from_numpy(c).to(DEV)
        with pytest.raises(di.DiError) as e:
            ctx.inpaint(ft, ct, tol=0.0)
        assert e.value.status == di.INVALID_ARG
        with pytest.raises(di.DiError) as e:
            ctx.inpaint(ft, ct, out=ft)  # u aliases f
        assert e.value.status == di.INVALID_ARG
        # the context stays usable after argument errors
        u, st = ctx.inpaint(ft, ct)
        assert st == di.OK


def test_context_reuse_across_sizes(di):
    with di.Context() as ctx:
        for (w, h, C, seed) in [(64, 48, 1, 1), (300, 200, 3, 2), (90, 70, 2, 3)]:
            f, c = synth.make_case(w, h, C, 0.05, "uniform", seed)
            ref = oracle.cg_inpaint(f, c)
            u, st = ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV))
            assert st == di.OK
            _check(u.cpu().numpy(), f, c, ref)


def test_non_default_stream(di):
    f, c = synth.make_case(200, 150, 3, 0.05, "edge", 4)
    ref = oracle.cg_inpaint(f, c)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ft = torch.from_numpy(f).to(DEV)
        ct = torch.from_numpy(c).to(DEV)
        with di.Context() as ctx:
            u, st = ctx.inpaint(ft, ct, stream=s)
    s.synchronize()
    assert st == di.OK
    _check(u.cpu().numpy(), f, c, ref)


def test_full_size_bench_frames_in_bench_configuration(di):
    # all six 3840x2160 RGB bench frames ({10, 4, 1} % x {edge-clustered,
    # uniform}, the bench's seeds), decoded as the bench times them (its block,
    # overlap and local steps; two decoders with their own contexts and streams
    # at once), each against the FP64 oracle at the 0.05 / 0.01 bar
    import os
    import sys
    import threading

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    ks = list(range(len(bench.CASES)))
    frames = [synth.make_case(bench.W4K, bench.H4K, bench.C4K, *bench.CASES[k],
                              bench._case_seed(k)) for k in ks]
    cfg = dict(block=bench.BLOCK, overlap=bench.OVERLAP, local_iters=bench.LOCAL_ITERS,
               local_iters_coarse=bench.LOCAL_ITERS_COARSE, local_stop=bench.LOCAL_STOP)
    outs, sts = [None] * len(ks), [None] * len(ks)

    def work(t):
        s = torch.cuda.Stream(DEV)
        with di.Context(**cfg) as ctx, torch.cuda.stream(s):
            for j in range(t, len(ks), 2):
                f, c = frames[j]
                u, st = ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV),
                                    tol=TOL, stream=s)
                s.synchronize()
                outs[j], sts[j] = u.cpu().numpy(), st

    th = [threading.Thread(target=work, args=(t,)) for t in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for j, ((f, c), u, st) in enumerate(zip(frames, outs, sts)):
        assert st == di.OK, bench.CASES[j]
        _check(u, f, c, oracle.cg_inpaint(f, c))
        if j in (1, 2):  # the same result when decoded alone
            solo, st2, _ = _run(di, f, c, **cfg)
            assert st2 == di.OK and np.array_equal(u, solo)

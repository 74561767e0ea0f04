"""The device-driven decode: the whole decode as one CUDA graph whose stop
test (Section 5.2 criterion, or the error estimate in gray levels) runs on the
device after every V-cycle and whose level structure (the levels in use, the
cascade's start) is chosen on the device from the mask.  It must give the
same bits, statuses, cycle counts, statistics and kernel counts as the
host-driven loop (graph off), for every stop rule and the configurations that
change the graph's structure, and its asynchronous entry point must give the
same results as the synchronous one."""
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


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _decode(di, f, c, tol, **cfg):
    with di.Context(**cfg) as ctx:
        ctx.reset_profile()
        u, st = ctx.inpaint(T(f), T(c), tol=tol, check=False)
        torch.cuda.synchronize()
        pr = ctx.profile()
        # graph on: the decode ran as one device-driven graph; off: host loop
        device = cfg.get("graph", di.GRAPH_ON) == di.GRAPH_ON
        why = di.load().di_last_error(ctx._h).decode()
        assert pr["device_decodes"] == (1 if device else 0), (pr, why)
        return u.cpu().numpy(), st, ctx.stats(), pr["launches"]


def _same(di, f, c, tol, **cfg):
    a = _decode(di, f, c, tol, graph=di.GRAPH_ON, **cfg)
    b = _decode(di, f, c, tol, graph=di.GRAPH_OFF, **cfg)
    (u0, s0, st0, k0), (u1, s1, st1, k1) = a, b
    assert s0 == s1, (s0, s1)
    for key in ("cycles", "converged", "levels", "levels_used", "unknowns", "status"):
        assert st0[key] == st1[key], (key, st0[key], st1[key])
    assert st0["est_error"] == st1["est_error"] or (np.isinf(st0["est_error"]) and
                                                    np.isinf(st1["est_error"]))
    assert st0["rel_residual"] == st1["rel_residual"]
    assert np.array_equal(u0, u1)
    # the device-driven graph adds the plan kernel and one stop-test kernel
    # per cycle to the host loop's kernels
    assert k1 > 0 and k0 == k1 + 1 + st0["cycles"], (k0, k1, st0["cycles"])
    return u0, s0, st0


@pytest.mark.parametrize("stop", ["estimate", "residual", "fixed"])
def test_device_loop_matches_host_loop_stop_rules(di, stop):
    f, c = synth.make_case(200, 136, 2, 0.04, "edge", 61)
    rule = {"estimate": di.STOP_ERROR_ESTIMATE, "residual": di.STOP_RELATIVE_RESIDUAL,
            "fixed": di.STOP_FIXED_CYCLES}[stop]
    tol = 1e-4 if stop == "residual" else TOL
    u, st, stats = _same(di, f, c, tol, stop_rule=rule, max_cycles=5)
    if stop == "fixed":
        assert stats["cycles"] == 5


@pytest.mark.parametrize("w,h,C,d,kind,cfg", [
    # dense mask: the coarse levels are fully known, fewer levels in use
    (320, 200, 3, 0.10, "uniform", {}),
    (256, 256, 1, 0.30, "uniform", {}),
    # sparse mask: every level in use, the coarsest single-block solve
    (300, 170, 2, 0.005, "edge", {}),
    # overlap with shared pixels (combine passes), other block sizes
    (257, 131, 3, 0.04, "edge", {"overlap": 6}),
    (200, 120, 1, 0.04, "uniform", {"block": 16, "overlap": 4}),
    (150, 90, 2, 0.04, "uniform", {"block": 8, "overlap": 2}),
    # the global CG smoother, the given start, more smoothing steps
    (200, 120, 2, 0.04, "edge", {"smoother": 1}),
    (180, 100, 2, 0.04, "edge", {"pre": 2, "post": 2}),
    # the bench's solver setting
    (640, 360, 3, 0.04, "edge", {"overlap": 2, "local_iters": 10, "local_iters_coarse": 8}),
    # 16-bit coarse storage and local iterates; FP64 finest-grid residuals
    (400, 240, 3, 0.01, "edge", {"precision": 1}),
    (400, 240, 3, 0.04, "uniform", {"precision": 2, "overlap": 4}),
    (300, 200, 2, 0.02, "edge", {"refine_fp64": 1}),
])
def test_device_loop_matches_host_loop_configurations(di, w, h, C, d, kind, cfg):
    f, c = synth.make_case(w, h, C, d, kind, 1000 + w + h)
    u, st, stats = _same(di, f, c, TOL, max_cycles=32, **cfg)
    assert st == di.OK
    err = np.abs(u.astype(np.float64) - oracle.cg_inpaint(f, c))
    assert err.max() <= TOL and np.sqrt((err ** 2).mean()) <= 0.01


def test_device_loop_degenerate_masks(di):
    f, c = synth.make_case(96, 64, 2, 0.04, "uniform", 5)
    # every pixel known: u = f without cycles
    full = np.ones_like(c)
    u, st, stats = _same(di, f, full, TOL)
    assert st == di.OK and stats["cycles"] == 0 and np.array_equal(u, f)
    # no pixel known: the empty-mask status
    empty = np.zeros_like(c)
    _, st, _ = _same(di, f, empty, TOL)
    assert st == di.EMPTY_MASK
    # one known pixel: a constant image, every level in use
    one = np.zeros_like(c)
    one[10, 20] = 1
    u, st, _ = _same(di, f, one, TOL, max_cycles=64)
    assert st == di.OK
    for k in range(f.shape[0]):
        assert np.abs(u[k] - f[k, 10, 20]).max() <= TOL


def test_device_loop_not_converged_and_given_start(di):
    f, c = synth.make_case(200, 136, 2, 0.01, "edge", 62)
    _, st, stats = _same(di, f, c, 1e-6, max_cycles=2)
    assert st == di.NOT_CONVERGED and stats["cycles"] == 2
    # the given start (a warm start from a converged result needs one cycle)
    ref, st, _, _ = _decode(di, f, c, TOL)
    assert st == di.OK
    for mode in (di.GRAPH_ON, di.GRAPH_OFF):
        with di.Context(start=di.START_GIVEN, graph=mode) as ctx:
            u = T(ref)
            _, st = ctx.inpaint(T(f), T(c), tol=TOL, out=u)
            torch.cuda.synchronize()
            assert st == di.OK and ctx.stats()["cycles"] == 1


def test_async_entry_matches_sync_and_cached_graphs_follow_contents(di):
    # frames enqueued back to back on one stream without waiting; a context
    # reuses its graph for the same buffers with new contents
    frames = [synth.make_case(240, 160, 3, d, k, 80 + i)
              for i, (d, k) in enumerate([(0.05, "edge"), (0.02, "uniform"), (0.08, "edge")])]
    refs = [_decode(di, f, c, TOL) for f, c in frames]
    s = torch.cuda.Stream(DEV)
    with di.Context() as ctx, torch.cuda.stream(s):
        fb = torch.empty(frames[0][0].shape, dtype=torch.float32, device=DEV)
        cb = torch.empty(frames[0][1].shape, dtype=torch.uint8, device=DEV)
        ub = torch.empty_like(fb)
        outs = []
        for rep in range(2):
            for (f, c), ref in zip(frames, refs):
                fb.copy_(T(f))
                cb.copy_(T(c))
                ctx.inpaint_async(fb, cb, tol=TOL, out=ub, stream=s)
                outs.append(ub.clone())
                st = ctx.stats()  # waits for this decode
                assert st["status"] == di.OK and st["cycles"] == ref[2]["cycles"]
        s.synchronize()
        for i, u in enumerate(outs):
            assert np.array_equal(u.cpu().numpy(), refs[i % len(frames)][0])

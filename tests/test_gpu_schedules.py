"""Schedules and smoothers on the GPU (the comparison methods of Section 5 and
the scheme ablations of Section 4): full FMG with a V-cycle per cascade level
(Fig. 3), the cascade alone followed by finest-level smoothing (multilevel),
single-level iteration, and global CG in place of ORAS as the smoother.  Every
combination must reach the FP64 oracle's solution: within the decoder's error
tolerance under the error-estimate rule, and to a relative residual that an
FP64 recomputation confirms under the relative-residual rule."""
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


@pytest.fixture(scope="module")
def case():
    f, c = synth.make_case(200, 136, 2, 0.04, "edge", 61)
    return f, c, oracle.cg_inpaint(f, c)


def _run(di, f, c, tol, **cfg):
    with di.Context(**cfg) as ctx:
        u, st = ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), tol=tol)
        torch.cuda.synchronize()
        stats = ctx.stats()
    return u.cpu().numpy(), st, stats


def _check(u, f, c, ref, tol):
    assert np.isfinite(u).all()
    assert np.array_equal(u[:, c == 1], f[:, c == 1])
    err = np.abs(u.astype(np.float64) - ref)
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("smoother", ["oras", "cg"])
@pytest.mark.parametrize("schedule", ["reduced_fmg", "full_fmg"])
def test_fmg_schedules_error_estimate(di, case, schedule, smoother):
    f, c, ref = case
    sched = {"reduced_fmg": di.SCHED_REDUCED_FMG, "full_fmg": di.SCHED_FULL_FMG}[schedule]
    sm = {"oras": di.SMOOTH_ORAS, "cg": di.SMOOTH_CG}[smoother]
    u, st, stats = _run(di, f, c, TOL, schedule=sched, smoother=sm, max_cycles=64)
    assert st == di.OK and stats["converged"]
    _check(u, f, c, ref, TOL)


def test_full_fmg_cascade_is_at_least_as_good(di, case):
    # one V-cycle per cascade level before the finest-level cycles: after a
    # fixed single cycle the full schedule is no farther from the solution
    f, c, ref = case
    errs = {}
    for name, sched in (("reduced", di.SCHED_REDUCED_FMG), ("full", di.SCHED_FULL_FMG)):
        u, st, _ = _run(di, f, c, TOL, schedule=sched, stop_rule=di.STOP_FIXED_CYCLES,
                        max_cycles=1, min_cycles=1)
        assert st == di.OK
        errs[name] = np.abs(u.astype(np.float64) - ref).max()
    assert errs["full"] <= errs["reduced"] * 1.05 + 1e-3, errs


def _rel_residual_fp64(u, f, c):
    # ||b - A u|| / ||b - A u0|| per channel in FP64, u0 = f on the mask, 0 elsewhere
    from oracle import method as M

    out = []
    for ch in range(f.shape[0]):
        b = M.rhs(f[ch].astype(np.float64), c)
        r = M.residual(u[ch].astype(np.float64), b, c)
        r0 = M.residual(b, b, c)
        out.append(np.linalg.norm(r) / np.linalg.norm(r0))
    return out


@pytest.mark.parametrize("smoother", ["oras", "cg"])
@pytest.mark.parametrize("schedule", ["multilevel", "single"])
def test_non_multigrid_schedules_relative_residual(di, case, schedule, smoother):
    # the relative-residual rule of the comparison: the residual the library
    # reports must be the true one (recomputed in FP64), and a small residual
    # must mean a solution close to the oracle's (a residual bound is not an
    # error bound, hence the looser error check)
    f, c, ref = case
    sched = {"multilevel": di.SCHED_MULTILEVEL, "single": di.SCHED_SINGLE}[schedule]
    sm = {"oras": di.SMOOTH_ORAS, "cg": di.SMOOTH_CG}[smoother]
    rtol = 1e-5
    u, st, stats = _run(di, f, c, rtol, schedule=sched, smoother=sm,
                        stop_rule=di.STOP_RELATIVE_RESIDUAL, max_cycles=4000,
                        local_iters=8)
    assert st == di.OK and stats["converged"], stats
    assert max(stats["rel_residual"][:2]) <= rtol
    true_rr = _rel_residual_fp64(u, f, c)
    for ch in range(2):
        assert true_rr[ch] <= 1.2 * stats["rel_residual"][ch] + 1e-7, (true_rr, stats)
    _check(u, f, c, ref, 0.25)


def test_multilevel_oras_error_estimate(di, case):
    # the multilevel ORAS solver of the comparison, under the decoder's own stop rule
    f, c, ref = case
    u, st, stats = _run(di, f, c, TOL, schedule=di.SCHED_MULTILEVEL, max_cycles=2000)
    assert st == di.OK and stats["converged"]
    _check(u, f, c, ref, TOL)


def test_single_level_cg_matches_global_cg_steps(di):
    # single-level CG smoothing is global CG: with enough steps on a tiny
    # image it solves the system to the FP32 floor
    f, c = synth.make_case(48, 40, 1, 0.05, "uniform", 5)
    ref = oracle.cg_inpaint(f, c)
    u, st, stats = _run(di, f, c, 1e-5, schedule=di.SCHED_SINGLE, smoother=di.SMOOTH_CG,
                        stop_rule=di.STOP_RELATIVE_RESIDUAL, max_cycles=400, local_iters=4)
    assert st == di.OK
    assert np.abs(u.astype(np.float64) - ref).max() <= 1e-2


def test_naive_downsampling_still_converges(di, case):
    # ablation of the value downsampling (Section 4.3): the naive average
    # changes the cascade's start, not the fixed point
    f, c, ref = case
    u, st, stats = _run(di, f, c, TOL, downsample=1, max_cycles=64)
    assert st == di.OK and stats["converged"]
    _check(u, f, c, ref, TOL)


def test_plan_counts_cg_workspace(di):
    a = di.plan(640, 360, 3)["workspace_bytes"]
    b = di.plan(640, 360, 3, smoother=di.SMOOTH_CG)["workspace_bytes"]
    assert b - a == 4 * 640 * 360 * 3 * 4


def test_bad_schedule_and_smoother_rejected(di):
    with pytest.raises(Exception):
        di.Context(schedule=4)
    with pytest.raises(Exception):
        di.Context(smoother=2)


@pytest.mark.parametrize("stop", ["estimate", "residual", "fixed"])
def test_graph_replay_matches_direct_launches(di, case, stop):
    # the finest-level V-cycle replayed as a CUDA graph gives the same bits,
    # cycle count, launch count and profile counters as launching it kernel by
    # kernel
    f, c, _ = case
    rule = {"estimate": di.STOP_ERROR_ESTIMATE, "residual": di.STOP_RELATIVE_RESIDUAL,
            "fixed": di.STOP_FIXED_CYCLES}[stop]
    tol = 1e-4 if stop == "residual" else TOL
    res = {}
    for mode in (di.GRAPH_ON, di.GRAPH_OFF):
        with di.Context(graph=mode, stop_rule=rule, max_cycles=5, profile=1) as ctx:
            ft, ct = torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV)
            for _ in range(2):  # the second call updates the cached graph
                ctx.reset_profile()
                u, st = ctx.inpaint(ft, ct, tol=tol)
                torch.cuda.synchronize()
            res[mode] = (u.cpu().numpy(), st, ctx.stats(), ctx.profile())
    (u0, s0, st0, p0), (u1, s1, st1, p1) = res[di.GRAPH_ON], res[di.GRAPH_OFF]
    assert s0 == s1 and st0["cycles"] == st1["cycles"]
    assert np.array_equal(u0, u1)
    assert p0["launches"] == p1["launches"] and p0["launches"] > 0
    assert p0["oras_l0_launches"] == p1["oras_l0_launches"]
    assert p0["oras_l0_cg_steps"] == p1["oras_l0_cg_steps"]
    assert p0["oras_l0_prolong"] == p1["oras_l0_prolong"]
    assert p0["oras_l0_ms"] > 0 and p1["oras_l0_ms"] > 0


def test_graph_follows_changing_inputs(di):
    # one context, frames of different sizes and masks in turn: every result
    # equals a fresh context's (the cached graph is updated or rebuilt)
    cases = [synth.make_case(w, h, 3, d, k, 70 + i) for i, (w, h, d, k) in
             enumerate([(160, 96, 0.05, "edge"), (160, 96, 0.02, "uniform"),
                        (200, 120, 0.05, "edge"), (160, 96, 0.05, "edge")])]
    with di.Context() as ctx:
        for f, c in cases:
            u, st = ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), tol=TOL)
            torch.cuda.synchronize()
            ref, st2, _ = _run(di, f, c, TOL, graph=di.GRAPH_OFF)
            assert st == st2 == di.OK
            assert np.array_equal(u.cpu().numpy(), ref)


def test_coarse_level_local_steps(di, case):
    # fewer local steps on the coarse levels changes the iterates but not the
    # fixed point; the default (0) is the finest level's count
    f, c, ref = case
    u0, st0, _ = _run(di, f, c, TOL)
    u1, st1, _ = _run(di, f, c, TOL, local_iters_coarse=8)  # local_iters 8: same as default
    assert st0 == st1 == di.OK and np.array_equal(u0, u1)
    u2, st2, _ = _run(di, f, c, TOL, local_iters=10, local_iters_coarse=4, max_cycles=64)
    assert st2 == di.OK
    _check(u2, f, c, ref, TOL)


def test_cascade_local_steps(di, case):
    # a step limit of its own for the cascade's finest-level iteration changes
    # the iterates but not the fixed point; 0 (the default) is the level's own
    f, c, ref = case
    u0, st0, _ = _run(di, f, c, TOL)
    u1, st1, _ = _run(di, f, c, TOL, local_iters_cascade=8)  # local_iters 8: same as default
    assert st0 == st1 == di.OK and np.array_equal(u0, u1)
    u2, st2, _ = _run(di, f, c, TOL, local_iters=10, local_iters_cascade=3, max_cycles=64)
    assert st2 == di.OK
    _check(u2, f, c, ref, TOL)


def test_profile_counts_completed_local_steps(di, case):
    # the profile counts the local CG steps the finest-level local problems
    # completed: at most the step limit each, fewer with the local stop
    f, c, _ = case
    per_task = {}
    for ls in (-1.0, 0.2):
        with di.Context(profile=1, local_stop=ls) as ctx:
            ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), tol=TOL)
            torch.cuda.synchronize()
            pr = ctx.profile()
            st = ctx.stats()
        assert pr["oras_l0_tasks"] > 0
        assert 0 < pr["oras_l0_cg_steps"] <= 8 * pr["oras_l0_tasks"]  # default local_iters 8
        # the finest level's prolongations run inside its block kernel (32x32
        # blocks, even stride): the cascade's interpolation once, and one
        # correction per V-cycle where a coarser level carries unknowns
        assert st["levels"] >= 2
        assert pr["oras_l0_prolong"] == 1 + (st["cycles"] if st["levels_used"] >= 2 else 0)
        per_task[ls] = pr["oras_l0_cg_steps"] / pr["oras_l0_tasks"]
    assert per_task[0.2] <= per_task[-1.0]

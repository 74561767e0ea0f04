"""Batched and served decoding on the GPU (the batched and serving workloads):
every image of a batch, and every request served under load, must equal the
same image decoded alone (bit for bit: the decodes share no arithmetic) and
stay within 0.05 gray of the FP64 oracle where the oracle is run."""
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


def _case(w, h, C, d, kind, seed):
    f, c = synth.make_case(w, h, C, d, kind, seed)
    return f, c


def _solo(di, f, c, **cfg):
    with di.Context(**cfg) as ctx:
        u, st = ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), tol=TOL)
        torch.cuda.synchronize()
    assert st == di.OK
    return u.cpu().numpy()


def _check_oracle(u, f, c):
    ref = oracle.cg_inpaint(f, c)
    err = np.abs(u.astype(np.float64) - ref)
    assert err.max() <= TOL and np.sqrt((err ** 2).mean()) <= 0.01
    assert np.array_equal(u[:, c == 1], f[:, c == 1])


def test_batch_small_mixed_matches_oracle_and_solo(di):
    g = np.random.default_rng(3)
    sizes = [(96, 64), (160, 90), (200, 113), (257, 129), (320, 180), (64, 64)]
    cases = []
    for i in range(12):
        w, h = sizes[i % len(sizes)]
        C = int(g.integers(1, 4))
        d = float(g.uniform(0.01, 0.10))
        kind = "uniform" if i % 2 else "edge"
        cases.append(_case(w, h, C, d, kind, 100 + i))
    items = [(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), TOL) for f, c in cases]
    outs, sts, cyc = di.inpaint_batch(items, concurrency=4)
    torch.cuda.synchronize()
    assert all(s == di.OK for s in sts), sts
    for (f, c), u in zip(cases, outs):
        u = u.cpu().numpy()
        _check_oracle(u, f, c)
        assert np.array_equal(u, _solo(di, f, c))


def _config3_images():
    # 32 images with seeded sizes, channel counts and densities
    g = np.random.default_rng(20240112)
    sizes = [(512, 512), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]
    out = []
    for i in range(32):
        w, h = sizes[int(g.integers(0, len(sizes)))]
        C = int(g.integers(1, 4))
        d = float(g.uniform(0.01, 0.10))
        kind = "uniform" if g.random() < 0.5 else "edge"
        out.append((w, h, C, d, kind, 5000 + i))
    return out


def test_batch_config3_autotuned(di):
    specs = _config3_images()
    # autotune block size x overlap on the 512x512 images of the batch
    small = [s for s in specs if s[0] == 512][:2] or [(512, 512, 1, 0.04, "uniform", 1)]
    sample = []
    for (w, h, C, d, kind, seed) in small:
        f, c = _case(w, h, C, d, kind, seed)
        sample.append((torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), TOL))
    best, ms = di.autotune(sample, blocks=(8, 16, 32), overlaps=(1, 2, 4), reps=1)
    assert best["block"] in (8, 16, 32) and best["overlap"] in (1, 2, 4)
    assert ms > 0
    cfg = {"block": best["block"], "overlap": best["overlap"]}
    cases = [_case(*s) for s in specs]
    items = [(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), TOL) for f, c in cases]
    outs, sts, cyc = di.inpaint_batch(items, concurrency=4, **cfg)
    torch.cuda.synchronize()
    assert all(s == di.OK for s in sts), sts
    for k, ((f, c), u) in enumerate(zip(cases, outs)):
        u = u.cpu().numpy()
        assert np.isfinite(u).all()
        assert np.array_equal(u[:, c == 1], f[:, c == 1])
        for ch in range(f.shape[0]):
            known = f[ch][c == 1]
            assert u[ch].min() >= known.min() - TOL and u[ch].max() <= known.max() + TOL
        if k % 8 == 0:  # a quarter of them decoded alone as well
            assert np.array_equal(u, _solo(di, f, c, **cfg))
    # the first image of every size of the batch (512x512 ... 3840x2160)
    # against the FP64 oracle
    seen = set()
    for k, ((f, c), u) in enumerate(zip(cases, outs)):
        size = specs[k][:2]
        if size in seen:
            continue
        seen.add(size)
        _check_oracle(u.cpu().numpy(), f, c)
    assert len(seen) == 5, seen


def test_server_poisson_mixed_load(di):
    g = np.random.default_rng(7)
    sizes = [(1280, 720), (1920, 1080), (3840, 2160)]
    reqs = []
    for i in range(18):
        w, h = sizes[int(g.integers(0, 3))]
        d = float(g.uniform(0.005, 0.10))
        kind = "uniform" if g.random() < 0.5 else "edge"
        reqs.append(_case(w, h, 3, d, kind, 900 + i))
    gaps = g.exponential(1.0 / 120.0, size=len(reqs))  # Poisson arrivals, 120 / s
    import time

    results = []
    with di.Server(slots=4) as srv:
        tickets = []
        for (f, c), gap in zip(reqs, gaps):
            time.sleep(float(gap))
            tickets.append(srv.submit(f, c, TOL))
        for t in tickets:
            results.append(srv.wait(t))
    lat = sorted(r[1]["latency_ms"] for r in results)
    assert all(r[1]["status"] == di.OK for r in results)
    assert lat[-1] > 0
    for _, info in results:  # the stages after the start add up to the rest of the latency
        st = info["stages_ms"]
        assert min(st.values()) >= 0.0 and st["decode"] > 0.0
        assert abs(info["queue_ms"] + sum(st.values()) - info["latency_ms"]) < 1e-3
    for k, ((f, c), (u, info)) in enumerate(zip(reqs, results)):
        assert np.array_equal(u[:, c == 1], f[:, c == 1])
        if k % 3 == 0:  # same result alone as in the mix
            assert np.array_equal(u, _solo(di, f, c))
    # the first served request of each size (720p, 1080p, 4K) against the
    # FP64 oracle
    seen = set()
    for (f, c), (u, info) in zip(reqs, results):
        if f.shape[1:] in seen:
            continue
        seen.add(f.shape[1:])
        _check_oracle(u, f, c)
    assert len(seen) == 3, seen


def test_server_admission_budget_serialises_large_requests(di):
    f, c = _case(1920, 1080, 3, 0.04, "edge", 11)
    plan = di.plan(1920, 1080, 3)
    # room for one such request at a time
    budget = plan["workspace_bytes"] + 1920 * 1080 * (2 * 3 * 4 + 1)
    with di.Server(slots=3, mem_budget=budget) as srv:
        tickets = [srv.submit(f, c, TOL) for _ in range(4)]
        res = [srv.wait(t) for t in tickets]
    assert all(r[1]["status"] == di.OK for r in res)
    assert max(r[1]["queue_ms"] for r in res) > 0.0
    for u, _ in res[1:]:
        assert np.array_equal(u, res[0][0])


def test_pool_reuse_matches_solo(di):
    # a persistent pool decodes two batches in turn (slots, workspaces and
    # graphs reused); every image equals its solo decode bit for bit
    g = np.random.default_rng(12)
    sizes = [(160, 90), (257, 129), (96, 64), (320, 180)]
    batches = []
    for b in range(2):
        cases = []
        for i in range(5):
            w, h = sizes[(i + b) % len(sizes)]
            cases.append(_case(w, h, int(g.integers(1, 4)), float(g.uniform(0.02, 0.08)),
                               "edge" if i % 2 else "uniform", 300 + 10 * b + i))
        batches.append(cases)
    with di.Pool(concurrency=3) as pool:
        for cases in batches:
            items = [(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), TOL)
                     for f, c in cases]
            outs, sts, cyc = pool.inpaint(items)
            torch.cuda.synchronize()
            assert all(s == di.OK for s in sts), sts
            for (f, c), u in zip(cases, outs):
                assert np.array_equal(u.cpu().numpy(), _solo(di, f, c))


def test_autotune_over_local_steps_cycle_type_and_schedule(di):
    # the autotuner's full search space: block x overlap x local CG steps x
    # V(k, k) cycle type x schedule; the winner is one of the candidates and
    # decodes the sample within the bar
    sample_cases = [_case(320, 192, 3, 0.04, "edge", 31), _case(256, 256, 1, 0.02, "uniform", 32)]
    sample = [(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), TOL)
              for f, c in sample_cases]
    best, ms = di.autotune(sample, blocks=(32,), overlaps=(2, 4), local_iters=(6, 10),
                           smoothing=(1, 2), schedules=(di.SCHED_REDUCED_FMG, di.SCHED_FULL_FMG),
                           reps=1)
    assert ms > 0
    assert best["block"] == 32 and best["overlap"] in (2, 4)
    assert best["local_iters"] in (6, 10) and best["pre"] == best["post"] in (1, 2)
    assert best["schedule"] in (di.SCHED_REDUCED_FMG, di.SCHED_FULL_FMG)
    cfg = {k: best[k] for k in ("block", "overlap", "local_iters", "pre", "post", "schedule")}
    for f, c in sample_cases:
        _check_oracle(_solo(di, f, c, **cfg), f, c)


@pytest.mark.parametrize("cascade", [0, 4])
def test_batched_form_one_graph_matches_solo_and_oracle(di, cascade):
    # the batched form: a batch of uneven sizes and channel counts decoded as
    # one graph with one launch per step over every image; every image equals
    # its single-image decode bit for bit (the same arithmetic in the same
    # order) and, checked on the oracle, is within the bar
    g = np.random.default_rng(44)
    sizes = [(96, 64), (160, 90), (257, 129), (320, 180), (512, 512), (640, 360)]
    cases = []
    for i in range(10):
        w, h = sizes[i % len(sizes)]
        d = float(g.uniform(0.005, 0.10))
        cases.append(_case(w, h, int(g.integers(1, 4)), d, "edge" if i % 2 else "uniform",
                           600 + i))
    # one fully known image and one with a single known pixel ride along
    f1, c1 = _case(128, 96, 2, 0.05, "uniform", 650)
    cases.append((f1, np.ones_like(c1)))
    f2, c2 = _case(200, 120, 1, 0.05, "uniform", 651)
    one = np.zeros_like(c2)
    one[60, 100] = 1
    cases.append((f2, one))
    # cascade: the cascade's finest-level step limit (0: the level's own)
    cfg = dict(block=32, overlap=2, local_iters=10, local_iters_coarse=8, max_cycles=64,
               local_iters_cascade=cascade)
    items = [(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), TOL) for f, c in cases]
    with di.Batch(items, **cfg) as bt:
        for rep in range(2):  # the graph replays on the same buffers
            outs, sts, cyc = bt.run()
            torch.cuda.synchronize()
            assert all(s == di.OK for s in sts), sts
            for k, ((f, c), u) in enumerate(zip(cases, outs)):
                u = u.cpu().numpy()
                if rep == 0:
                    assert np.array_equal(u, _solo(di, f, c, **cfg)), k
                    if k < 6 or k >= 10:
                        _check_oracle(u, f, c)


def test_batched_form_config3_images_against_solo(di):
    # the 32-image mix of the batched workload (512x512 ... 3840x2160, 1-3
    # channels, 1-10 %) as one graph: bit-identical to the single-image
    # decodes of a sample and within the bar for one image of every size
    specs = _config3_images()
    cases = [_case(*s) for s in specs]
    cfg = dict(block=32, overlap=2, local_iters=10, local_iters_coarse=8)
    items = [(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), TOL) for f, c in cases]
    with di.Batch(items, **cfg) as bt:
        outs, sts, cyc = bt.run()
        torch.cuda.synchronize()
    assert all(s == di.OK for s in sts), sts
    seen = set()
    for k, ((f, c), u, sp) in enumerate(zip(cases, outs, specs)):
        u = u.cpu().numpy()
        if k % 8 == 0:
            assert np.array_equal(u, _solo(di, f, c, **cfg)), k
        if sp[:2] not in seen:
            seen.add(sp[:2])
            _check_oracle(u, f, c)

"""The precision workload: block CG vectors in FP16 or BF16 with FP32 dot
products, the coarse levels' corrections (iterates and restricted residuals)
stored in the same 16-bit type, FP32 residuals and FP32 update of u on the
finest grid, and optionally FP64 finest-grid residuals.  The decode must
still reach 0.05 gray max-abs of the FP64 oracle on every channel; the
per-channel errors are printed (pytest -s) for the record."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import method as M

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


def _decode(di, f, c, precision):
    with di.Context(precision=precision) as ctx:
        u, st = ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), tol=TOL)
        torch.cuda.synchronize()
        stats = ctx.stats()
    return u.cpu().numpy(), st, stats


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("w,h,d,kind", [(1280, 720, 0.005, "edge"), (640, 480, 0.04, "uniform"),
                                        (333, 171, 0.01, "edge")])
def test_narrow_iterates_reach_the_tolerance(di, prec, w, h, d, kind):
    code = {"fp16": di.PREC_FP16, "bf16": di.PREC_BF16}[prec]
    f, c = synth.make_case(w, h, 3, d, kind, w + 7)
    ref = oracle.cg_inpaint(f, c)
    u, st, stats = _decode(di, f, c, code)
    assert st == di.OK, stats
    assert np.array_equal(u[:, c == 1], f[:, c == 1])
    for ch in range(3):
        err = np.abs(u[ch].astype(np.float64) - ref[ch])
        print(f"{prec} {w}x{h} {kind} {d}: channel {ch} max {err.max():.4f} rms "
              f"{np.sqrt((err ** 2).mean()):.5f} cycles {stats['cycles']}")
        assert err.max() <= TOL and np.sqrt((err ** 2).mean()) <= 0.01


def test_precision_4k_rgb_half_percent_edge(di):
    # 3840x2160 RGB with a 0.5 % edge-clustered mask, FP16 and BF16 iterates
    f, c = synth.make_case(3840, 2160, 3, 0.005, "edge", 4004)
    ref = oracle.cg_inpaint(f, c)
    cycles = {}
    for code in (di.PREC_FP32, di.PREC_FP16, di.PREC_BF16):
        u, st, stats = _decode(di, f, c, code)
        assert st == di.OK, stats
        cycles[code] = stats["cycles"]
        for ch in range(3):
            err = np.abs(u[ch].astype(np.float64) - ref[ch])
            print(f"4K 0.5% edge precision {code}: channel {ch} max {err.max():.4f} rms "
                  f"{np.sqrt((err ** 2).mean()):.5f} cycles {stats['cycles']}")
            assert err.max() <= TOL and np.sqrt((err ** 2).mean()) <= 0.01
    # the local stop compares the normalised 16-bit residual with a level scaled the
    # same way, so narrow iterates need about as many V-cycles as FP32 ones
    for code in (di.PREC_FP16, di.PREC_BF16):
        assert cycles[code] <= cycles[di.PREC_FP32] + 2, cycles


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_narrow_oras_iteration_close_to_oracle_cg(di, prec):
    # one ORAS iteration: narrow local CG vs the FP64 restatement of the same
    # steps; 16-bit arithmetic (8 significant bits for BF16) bounds the agreement
    code = {"fp16": di.PREC_FP16, "bf16": di.PREC_BF16}[prec]
    g = np.random.default_rng(5)
    h, w = 96, 130
    f = g.uniform(0, 255, size=(2, h, w)).astype(np.float32)
    c = (g.random((h, w)) < 0.06).astype(np.uint8)
    u = np.where(c.astype(bool), f, g.uniform(0, 255, f.shape)).astype(np.float32)
    with di.Context(precision=code) as ctx:
        out = ctx.oras_iteration(torch.from_numpy(u).to(DEV), torch.from_numpy(f).to(DEV),
                                 torch.from_numpy(c).to(DEV), 8, rhs_zero=True)
        torch.cuda.synchronize()
    out = out.cpu().numpy()
    ref = M.oras_iteration(u, M.rhs(f, c), c, 32, 6, 0.5, ("cg", 8))
    scale = np.abs(ref - u).max()
    assert np.abs(out - ref).max() < 0.05 * scale
    assert np.array_equal(out[:, c == 1], u[:, c == 1])


def _decode_cfg(di, f, c, tol, **cfg):
    with di.Context(**cfg) as ctx:
        u, st = ctx.inpaint(torch.from_numpy(f).to(DEV), torch.from_numpy(c).to(DEV), tol=tol)
        torch.cuda.synchronize()
        stats = ctx.stats()
    return u.cpu().numpy(), st, stats


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_fp64_refinement_residual_reaches_a_tight_target(di, prec):
    # sixteen fixed V-cycles: with FP64 finest-grid residuals the decode ends
    # at least as close to the FP64 oracle as with FP32 residuals, far inside
    # the 0.05 gray bar, in every precision mode
    code = {"fp32": di.PREC_FP32, "fp16": di.PREC_FP16, "bf16": di.PREC_BF16}[prec]
    f, c = synth.make_case(640, 360, 3, 0.01, "edge", 4242)
    ref = oracle.cg_inpaint(f, c)
    errs = {}
    for refine in (0, 1):
        u, st, stats = _decode_cfg(di, f, c, TOL, precision=code, refine_fp64=refine,
                                   stop_rule=di.STOP_FIXED_CYCLES, max_cycles=16,
                                   min_cycles=16)
        assert st == di.OK and stats["cycles"] == 16
        assert np.array_equal(u[:, c == 1], f[:, c == 1])
        errs[refine] = float(np.abs(u.astype(np.float64) - ref).max())
    print(f"{prec}: max error after 16 cycles, FP32 residuals {errs[0]:.2e}, "
          f"FP64 residuals {errs[1]:.2e}")
    assert errs[1] <= 0.01
    assert errs[1] <= errs[0] + 1e-3


def test_fp64_restriction_matches_oracle_more_closely(di):
    # the refinement residual of one restriction (finest level to the first
    # coarse level) against the oracle's FP64 restriction: FP64 arithmetic
    # errs no more than FP32
    g = np.random.default_rng(9)
    f, c = synth.make_case(250, 130, 2, 0.04, "uniform", 19)
    u = np.where(c.astype(bool), f, f + g.normal(scale=1e-3, size=f.shape)).astype(np.float32)
    cH = M.mask_downsample(c)
    ref = M.restrict_residual(M.residual(u, M.rhs(f, c), c), cH)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    out = {}
    for refine in (0, 1):
        rH = di.restrict_residual(T(u), T(f), T(c), T(cH.astype(np.uint8)), rhs_zero=True,
                                  fp64=bool(refine))
        torch.cuda.synchronize()
        out[refine] = float(np.abs(rH.cpu().numpy() - ref).max())
    assert out[1] <= out[0] + 1e-7
    # FP64 arithmetic, one rounding to FP32 at the end: within one FP32 ulp
    assert out[1] <= float(np.abs(ref).max()) * 2.0 ** -23

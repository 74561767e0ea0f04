"""Pins for the CPU oracle: each check comes from the paper's definitions or
from mathematics, never from the oracle itself or from the CUDA path."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import method as M

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_case(h, w, c=1, d=0.1, seed=0):
    g = np.random.default_rng(seed)
    f = g.uniform(0, 255, size=(c, h, w)).astype(np.float32)
    m = (g.random((h, w)) < d).astype(np.uint8)
    if not m.any():
        m[g.integers(h), g.integers(w)] = 1
    return f, m


def _dense_A(c):
    """A = C + (I - C) L assembled entry by entry from its definition
    (Section 2.2), independent of the oracle's stencil code."""
    h, w = c.shape
    n = h * w
    A = np.zeros((n, n))
    for y in range(h):
        for x in range(w):
            i = y * w + x
            if c[y, x]:
                A[i, i] = 1.0
                continue
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                yy, xx = y + dy, x + dx
                if 0 <= yy < h and 0 <= xx < w:
                    A[i, i] += 1.0
                    A[i, yy * w + xx] -= 1.0
    return A


# ---------------------------------------------------------------------------
# FP64 CG oracle (Section 2.2)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("h,w,seed", [(1, 1, 0), (1, 7, 1), (5, 1, 2), (3, 5, 3), (8, 8, 4),
                                      (16, 16, 5), (11, 16, 6), (16, 9, 7)])
def test_cg_matches_dense_direct_solve(h, w, seed):
    f, c = _rand_case(h, w, 2, 0.15, seed)
    u = oracle.cg_inpaint(f, c)
    A = _dense_A(c)
    for ch in range(2):
        b = np.where(c.astype(bool), f[ch].astype(np.float64), 0.0).ravel()
        ref = np.linalg.solve(A, b).reshape(h, w)
        assert np.abs(u[ch] - ref).max() < 1e-10 * 255


def test_cg_mask_pixels_exact_and_max_principle():
    f, c = synth.make_case(64, 48, 3, 0.03, "uniform", 3)
    u = oracle.cg_inpaint(f, c)
    cm = c.astype(bool)
    for ch in range(3):
        assert np.array_equal(u[ch][cm], f[ch][cm].astype(np.float64))
        lo, hi = f[ch][cm].min(), f[ch][cm].max()
        assert u[ch].min() >= lo - 1e-9 and u[ch].max() <= hi + 1e-9


def test_cg_one_dimensional_closed_form():
    h, w, a, b = 9, 40, 7, 30
    f = np.zeros((1, h, w), np.float32)
    f[0, :, a] = 20.0
    f[0, :, b] = 200.0
    c = np.zeros((h, w), np.uint8)
    c[:, a] = 1
    c[:, b] = 1
    u = oracle.cg_inpaint(f, c)[0]
    x = np.arange(w, dtype=np.float64)
    ref = np.where(x <= a, 20.0, np.where(x >= b, 200.0, 20.0 + (x - a) * 180.0 / (b - a)))
    assert np.abs(u - ref[None, :]).max() < 1e-9


def test_cg_single_pixel_and_constant_data():
    f = np.full((1, 13, 17), np.nan, np.float32)
    c = np.zeros((13, 17), np.uint8)
    c[4, 9] = 1
    f[0, 4, 9] = 77.0
    u = oracle.cg_inpaint(f, c)
    assert np.abs(u - 77.0).max() < 1e-9
    f2, c2 = _rand_case(20, 30, 1, 0.05, 9)
    f2[:] = 42.5
    assert np.abs(oracle.cg_inpaint(f2, c2) - 42.5).max() < 1e-9


def test_cg_mean_value_property():
    f, c = synth.make_case(40, 33, 1, 0.05, "uniform", 5)
    u = oracle.cg_inpaint(f, c)[0]
    lap = M.neg_laplacian(u)  # independent check below on a few pixels by hand
    h, w = c.shape
    for (y, x) in [(0, 0), (0, 5), (7, 0), (h - 1, w - 1), (20, 17), (h - 1, 3)]:
        if c[y, x]:
            continue
        nb = [(y + dy, x + dx) for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0))
              if 0 <= y + dy < h and 0 <= x + dx < w]
        assert abs(len(nb) * u[y, x] - sum(u[p] for p in nb)) < 1e-9 * 255
    assert np.abs(np.where(c.astype(bool), 0.0, lap)).max() < 1e-9 * 255


def test_cg_linearity_and_channel_independence():
    f, c = _rand_case(24, 31, 2, 0.08, 11)
    f = np.round(f)  # integer data: the combination below is exact in float32
    u = oracle.cg_inpaint(f, c)
    g = np.stack([f[1], f[0]])
    ug = oracle.cg_inpaint(g, c)
    assert np.abs(ug[0] - u[1]).max() < 1e-9 and np.abs(ug[1] - u[0]).max() < 1e-9
    comb = (0.25 * f[0] + 0.5 * f[1])[None]
    uc = oracle.cg_inpaint(comb, c)[0]
    assert np.abs(uc - (0.25 * u[0] + 0.5 * u[1])).max() < 1e-8


@pytest.mark.parametrize("op", ["flipx", "flipy", "transpose", "rot90"])
def test_cg_dihedral_equivariance(op):
    f, c = _rand_case(19, 26, 1, 0.06, 13)
    u = oracle.cg_inpaint(f, c)[0]
    tf = {"flipx": lambda a: a[..., ::-1], "flipy": lambda a: a[..., ::-1, :],
          "transpose": lambda a: np.swapaxes(a, -1, -2),
          "rot90": lambda a: np.rot90(a, axes=(-2, -1))}[op]
    u2 = oracle.cg_inpaint(np.ascontiguousarray(tf(f)), np.ascontiguousarray(tf(c)))[0]
    assert np.abs(u2 - tf(u)).max() < 1e-9


def test_cg_errors():
    f = np.zeros((1, 4, 4), np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.cg_inpaint(f, np.zeros((4, 4), np.uint8))
    with pytest.raises(oracle.OracleError):
        oracle.cg_inpaint(f, np.zeros((3, 4), np.uint8))


# ---------------------------------------------------------------------------
# Constants the paper prints
# ---------------------------------------------------------------------------


def test_paper_block_count_and_levels():
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    assert M.block_count(g["height"], g["width"], g["channels"], g["block"],
                         g["overlap"]) == g["local_problems"]
    assert M.num_levels(g["height"], g["width"], g["block"]) == g["levels"]


# ---------------------------------------------------------------------------
# Grid transfers (Section 4.3, 4.4)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("h,w", [(1, 1), (1, 5), (4, 4), (5, 7), (9, 2), (33, 17)])
def test_mask_downsample_brute_force(h, w):
    g = np.random.default_rng(h * 100 + w)
    c = (g.random((h, w)) < 0.2).astype(np.uint8)
    cH = M.mask_downsample(c)
    H, W = (h + 1) // 2, (w + 1) // 2
    assert cH.shape == (H, W)
    for Y in range(H):
        for X in range(W):
            kids = [c[y, x] for y in (2 * Y, 2 * Y + 1) for x in (2 * X, 2 * X + 1)
                    if y < h and x < w]
            assert cH[Y, X] == max(kids)


def test_modified_downsample_golden():
    gold = json.load(open(os.path.join(GOLD, "modified_downsample.json")))
    case = gold["cases"][0]
    c = np.array(case["mask"], np.uint8)
    b = np.array(case["values"], np.float64)
    cH = M.mask_downsample(c)
    assert np.array_equal(cH, np.array(case["coarse_mask"]))
    assert np.array_equal(M.modified_weights(c, cH), np.array(case["weights"], np.float64))
    assert np.allclose(M.values_downsample_modified(c, b, cH), case["modified"], atol=1e-12)
    assert np.allclose(M.values_downsample_naive(c, b), case["naive"], atol=1e-12)
    case = gold["cases"][1]
    c = np.array(case["mask"], np.uint8)
    b = np.array(case["values"], np.float64)
    out = M.values_downsample_modified(c, b)
    for y, x, v in case["modified_at"]:
        assert abs(out[int(y), int(x)] - v) < 1e-12


def test_modified_equals_naive_for_isolated_mask_pixels():
    # no mask pixel has a masked direct neighbour (fine or coarse) -> all
    # weights are 4 and the modified rule reduces to the naive average
    h, w = 16, 20
    c = np.zeros((h, w), np.uint8)
    c[0::4, 0::4] = 1
    g = np.random.default_rng(1)
    b = g.uniform(0, 255, (h, w))
    cH = M.mask_downsample(c)
    assert np.allclose(M.values_downsample_modified(c, b, cH), M.values_downsample_naive(c, b))


def test_restriction_consistent_with_rediscretised_operator():
    # e = x^2 + y^2: L e = -4 on the fine grid (h = 1); sampled at coarse
    # cell centres (spacing 2) the unit stencil gives -16 = 4 * mean(-4).
    h, w = 16, 12
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    e = xs ** 2 + ys ** 2
    r = -M.neg_laplacian(e)  # = Laplacian, +4 in the interior
    rH = M.restrict_residual(r, np.zeros(((h + 1) // 2, (w + 1) // 2), np.uint8))
    Ys, Xs = np.mgrid[0:h // 2, 0:w // 2].astype(np.float64)
    eH = (2 * Xs + 0.5) ** 2 + (2 * Ys + 0.5) ** 2
    lapH = -M.neg_laplacian(eH)
    assert np.allclose(rH[1:-1, 1:-1], lapH[1:-1, 1:-1])
    assert np.allclose(rH[1:-1, 1:-1], 16.0)


def test_restriction_masks_and_ragged_edges():
    r = np.ones((5, 7))
    cH = np.zeros((3, 4), np.uint8)
    cH[0, 0] = 1
    rH = M.restrict_residual(r, cH)
    assert rH[0, 0] == 0.0
    assert np.allclose(rH.ravel()[1:], 4.0)  # mean over 1, 2 or 4 existing children


def test_prolongation_constant_and_linear():
    H, W = 6, 9
    h, w = 12, 17
    assert np.allclose(M.prolong(np.full((H, W), 3.5), h, w), 3.5)
    Ys, Xs = np.mgrid[0:H, 0:W].astype(np.float64)
    uH = 2.0 * (2 * Xs + 0.5) - 3.0 * (2 * Ys + 0.5)
    u = M.prolong(uH, h, w)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    ref = 2.0 * xs - 3.0 * ys
    # exact away from the clamped border
    assert np.allclose(u[1:-1, 1:-1][: 2 * H - 2, : 2 * W - 2], ref[1:-1, 1:-1][: 2 * H - 2, : 2 * W - 2])


def test_prolongation_brute_force_weights():
    g = np.random.default_rng(4)
    H, W, h, w = 3, 4, 5, 8
    uH = g.random((H, W))
    u = M.prolong(uH, h, w)
    for y in range(h):
        for x in range(w):
            Y, X = y // 2, x // 2
            Yf = min(max(Y - 1 if y % 2 == 0 else Y + 1, 0), H - 1)
            Xf = min(max(X - 1 if x % 2 == 0 else X + 1, 0), W - 1)
            ref = (9 * uH[Y, X] + 3 * uH[Y, Xf] + 3 * uH[Yf, X] + uH[Yf, Xf]) / 16
            assert abs(u[y, x] - ref) < 1e-14


def test_prolong_modes_respect_mask():
    c = np.zeros((6, 6), np.uint8)
    c[2, 3] = 1
    b = np.zeros((6, 6))
    b[2, 3] = 99.0
    uH = np.ones((3, 3))
    us = M.prolong_solution(uH, b, c)
    assert us[2, 3] == 99.0 and np.allclose(np.delete(us.ravel(), 2 * 6 + 3), 1.0)
    uc = M.prolong_correct(np.full((6, 6), 5.0), uH, c)
    assert uc[2, 3] == 5.0 and np.allclose(np.delete(uc.ravel(), 2 * 6 + 3), 6.0)


# ---------------------------------------------------------------------------
# Block decomposition, weights, local problems (Section 3)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("n,B,o", [(1, 32, 6), (32, 32, 6), (33, 32, 6), (60, 32, 6),
                                   (100, 16, 4), (77, 8, 2), (50, 8, 4), (41, 8, 1),
                                   (2160, 32, 6)])
def test_partition_of_unity(n, B, o):
    wts = M.axis_weights(n, B, o)
    assert np.allclose(wts.sum(axis=0), 1.0)
    spans = M.axis_blocks(n, B, o)
    assert spans[0][0] == 0 and spans[-1][1] == n
    for k in range(1, len(spans)):
        a, e = spans[k]
        assert spans[k - 1][1] - a == o  # every overlap is o wide
        if o >= 2:
            assert wts[k, a] == 0.0 and wts[k - 1, a] == 1.0           # outermost 0
            assert wts[k, a + o - 1] == 1.0 and wts[k - 1, a + o - 1] == 0.0
    # no pixel is covered by more than two blocks
    assert ((wts > 0).sum(axis=0) <= 2).all()


def test_partition_of_unity_2d():
    h, w, B, o = 70, 57, 16, 4
    wy, wx = M.axis_weights(h, B, o), M.axis_weights(w, B, o)
    tot = np.zeros((h, w))
    for ky in range(wy.shape[0]):
        for kx in range(wx.shape[0]):
            tot += wy[ky][:, None] * wx[kx][None, :]
    assert np.allclose(tot, 1.0)


def test_local_operator_robin_rows_by_hand():
    # 3x3 block in the middle of a 5x5 image without mask: interior pixel has
    # 4 in-block neighbours; edge-centre pixels 3 in-block + 1 Robin side;
    # corners 2 + 2 Robin sides.
    c = np.zeros((5, 5), np.uint8)
    a = 0.3
    diag, couple, cb = M.local_operator(c, 1, 4, 1, 4, a)
    exp = np.array([[2 + 2 * a, 3 + a, 2 + 2 * a], [3 + a, 4, 3 + a], [2 + 2 * a, 3 + a, 2 + 2 * a]])
    assert np.allclose(diag, exp)
    # a block at the image corner: image edges are reflecting (no term)
    diag, _, _ = M.local_operator(c, 0, 2, 0, 2, a)
    assert np.allclose(diag, [[2, 2 + a], [2 + a, 2 + 2 * a]])
    # mask pixel: identity row, and it is not coupled to its neighbours
    c[2, 2] = 1
    diag, couple, cb = M.local_operator(c, 1, 4, 1, 4, a)
    assert diag[1, 1] == 1.0 and cb[1, 1]
    assert couple[1][1, 0] == 0.0  # right neighbour of (2,1) is the mask pixel
    assert np.allclose(diag[0, 1], 3 + a)


def test_oras_single_block_is_exact_solve():
    f, c = _rand_case(20, 24, 2, 0.05, 21)
    u_ex = oracle.cg_inpaint(f, c)
    b = M.rhs(f, c)
    u0 = np.where(c.astype(bool), b, 0.0)
    u1 = M.oras_iteration(u0, b, c, block=32, overlap=6)
    assert np.abs(u1 - u_ex).max() < 1e-9


def test_oras_fixed_point_and_convergence():
    f, c = _rand_case(40, 45, 1, 0.05, 22)
    u_ex = oracle.cg_inpaint(f, c)
    b = M.rhs(f, c)
    assert np.abs(M.oras_iteration(u_ex, b, c, 16, 4) - u_ex).max() < 1e-9
    u = np.where(c.astype(bool), b, 0.0)
    errs = []
    for _ in range(30):
        u = M.oras_iteration(u, b, c, 16, 4, 0.5)
        errs.append(np.abs(u - u_ex).max())
    assert errs[-1] < 1e-3 * errs[0]
    assert np.all(np.diff(errs[5:]) <= 1e-12)


def test_local_cg_reaches_exact_local_solve():
    f, c = _rand_case(12, 12, 1, 0.1, 23)
    g = np.random.default_rng(0).normal(size=(1, 8, 8))
    rb = np.where(c[2:10, 3:11].astype(bool), 0.0, g)
    ex = M.solve_local_exact(c, 2, 10, 3, 11, 0.5, rb)
    pc = M.solve_local_cg(c, 2, 10, 3, 11, 0.5, rb, 64)
    assert np.abs(ex - pc).max() < 1e-9


# ---------------------------------------------------------------------------
# Multigrid (Algorithm 3, Section 4.2)
# ---------------------------------------------------------------------------


def test_reduced_fmg_converges_to_cg_solution():
    f, c = synth.make_case(96, 80, 1, 0.04, "uniform", 1)
    u_ex = oracle.cg_inpaint(f, c)
    hist = []
    M.reduced_fmg(f, c, cycles=4, history=hist)
    errs = [np.abs(h - u_ex).max() for h in hist]
    assert errs[-1] < 1e-5
    assert all(errs[k + 1] < 0.2 * errs[k] for k in range(len(errs) - 1))


def test_vcycle_with_exact_coarse_reduces_error_two_grid():
    # two levels only (block 64 > coarse size): a two-grid cycle (Algorithm 3)
    f, c = synth.make_case(100, 90, 1, 0.03, "uniform", 2)
    u_ex = oracle.cg_inpaint(f, c)
    levels = M.build_pyramid(f, c, 64)
    assert len(levels) == 2
    b = levels[0][1]
    u = np.where(c.astype(bool), b, 0.0)
    e0 = np.abs(u - u_ex).max()
    u = M.vcycle(levels, 0, u, b, 64, 8, 0.5, "exact")
    assert np.abs(u - u_ex).max() < 0.05 * e0


def test_modified_downsampling_reduces_leakage():
    # Section 4.3: with one-way (cascadic) multigrid only, the modified rule
    # gives less colour bleeding than the naive one on edge-heavy data.
    better = 0
    for seed in range(3):
        f, c = synth.make_case(128, 128, 1, 0.02, "edge", 40 + seed)
        u_ex = oracle.cg_inpaint(f, c)
        um = M.reduced_fmg(f, c, cycles=0, downsample="modified")
        un = M.reduced_fmg(f, c, cycles=0, downsample="naive")
        em = np.sqrt(((um - u_ex) ** 2).mean())
        en = np.sqrt(((un - u_ex) ** 2).mean())
        better += em < en
    assert better >= 2

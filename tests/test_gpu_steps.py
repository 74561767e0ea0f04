"""GPU parity of each step of the path against the oracle's restatement of
the same step (oracle.method), through the C ABI.

Tolerances: integer/mask work is bit-exact.  Floating-point steps compute in
FP32 against an FP64 oracle on values of at most 255 gray; a single FP32
operation on such values carries an error of about 255 * 2^-24 = 1.5e-5, so
stencil-sized expressions are compared at 2e-4 (absolute) and the ORAS
iteration, whose local PCG amplifies rounding over its steps, at 1e-3 of the
largest correction plus 2e-4."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import method as M

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def di():
    from paper_2401_06744_gb300 import build as b

    b.build()
    import paper_2401_06744_gb300 as di

    di.load()
    return di


def T(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def N(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _case(h, w, C, d, seed, nan=True):
    g = np.random.default_rng(seed)
    f = g.uniform(0, 255, size=(C, h, w)).astype(np.float32)
    c = (g.random((h, w)) < d).astype(np.uint8)
    if not c.any():
        c[g.integers(h), g.integers(w)] = 1
    fn = f.copy()
    if nan:
        fn[:, c == 0] = np.nan  # never read at unknown pixels
    return f, fn, c


SIZES = [(1, 1), (1, 9), (7, 1), (3, 5), (17, 33), (64, 64), (101, 67), (130, 257), (66, 128), (2, 2)]


@pytest.mark.parametrize("h,w", SIZES)
def test_mask_downsample_bit_exact(di, h, w):
    _, _, c = _case(h, w, 1, 0.15, h * 7 + w)
    cH = di.mask_downsample(T(c))
    assert np.array_equal(N(cH), M.mask_downsample(c))


@pytest.mark.parametrize("h,w", SIZES)
@pytest.mark.parametrize("modified", [True, False])
def test_values_downsample(di, h, w, modified):
    f, fn, c = _case(h, w, 3, 0.3, h * 11 + w)
    cH = M.mask_downsample(c)
    out = N(di.values_downsample(T(c), T(fn), T(cH), modified=modified))
    ref = (M.values_downsample_modified(c, f, cH) if modified
           else M.values_downsample_naive(c, f))
    assert np.isfinite(out).all()
    assert np.abs(out - ref).max() < 2e-4


@pytest.mark.parametrize("h,w", SIZES + [(1080, 1920), (33, 2000)])
@pytest.mark.parametrize("modified", [True, False])
def test_pyramid_level_one_pass_bit_exact(di, h, w, modified):
    # the decoder's one-pass pyramid level: the coarse mask bit-exact with the
    # oracle's 2x2 max pooling, the mask values bit-identical to the separate
    # downsampling step and within rounding of the oracle, the packed words
    # and the unknown count exactly those of the coarse mask
    f, fn, c = _case(h, w, 2, 0.2, h * 5 + w)
    cH, bH, bits, unk = di.pyramid_level(T(c), T(fn), modified=modified)
    cH_ref = M.mask_downsample(c)
    assert np.array_equal(N(cH), cH_ref)
    sep = N(di.values_downsample(T(c), T(fn), T(cH_ref), modified=modified))
    assert np.array_equal(N(bH), sep)
    ref = (M.values_downsample_modified(c, f, cH_ref) if modified
           else M.values_downsample_naive(c, f))
    assert np.abs(N(bH) - ref).max() < 2e-4
    hH, wH = cH_ref.shape
    wpr = (wH + 31) // 32 + 1
    words = N(bits).astype(np.int64) & 0xFFFFFFFF
    known = np.ones((hH, 32 * wpr), dtype=bool)
    known[:, :wH] = cH_ref.astype(bool)
    ref_words = (known.reshape(hH, wpr, 32) * (1 << np.arange(32, dtype=np.int64))).sum(axis=2)
    assert np.array_equal(words, ref_words)
    assert int(N(unk)[0]) == int((cH_ref == 0).sum())
    # masks only
    cH2, bH2, bits2, unk2 = di.pyramid_level(T(c))
    assert bH2 is None and np.array_equal(N(cH2), cH_ref) and np.array_equal(N(bits2), N(bits))


@pytest.mark.parametrize("h,w", SIZES)
def test_residual_and_norm(di, h, w):
    f, fn, c = _case(h, w, 2, 0.1, h * 13 + w)
    g = np.random.default_rng(5)
    u = np.where(c.astype(bool), f, g.uniform(0, 255, f.shape)).astype(np.float32)
    with di.Context() as ctx:
        # b = C f (values off the mask never read) ...
        r, n2 = ctx.residual_norm(T(u), T(fn), T(c), rhs_zero=True)
        ref = M.residual(u, M.rhs(f, c), c)
        assert np.abs(N(r) - ref).max() < 2e-4
        assert np.allclose(N(n2), (ref ** 2).sum(axis=(1, 2)), rtol=1e-5, atol=1e-6)
        # ... and a general right-hand side at unknown pixels
        b = np.where(c.astype(bool), f, g.normal(size=f.shape)).astype(np.float32)
        r, n2 = ctx.residual_norm(T(u), T(b), T(c), rhs_zero=False)
        ref = M.residual(u, b, c)
        assert np.abs(N(r) - ref).max() < 2e-4


@pytest.mark.parametrize("h,w", SIZES)
def test_restrict_residual(di, h, w):
    f, fn, c = _case(h, w, 2, 0.05, h * 17 + w)
    g = np.random.default_rng(6)
    u = np.where(c.astype(bool), f, g.uniform(0, 255, f.shape)).astype(np.float32)
    cH = M.mask_downsample(c)
    rH = N(di.restrict_residual(T(u), T(fn), T(c), T(cH), rhs_zero=True))
    ref = M.restrict_residual(M.residual(u, M.rhs(f, c), c), cH)
    assert np.abs(rH - ref).max() < 1e-3
    b = np.where(c.astype(bool), 0.0, g.normal(size=f.shape)).astype(np.float32)
    u2 = np.where(c.astype(bool), 0.0, g.normal(size=f.shape)).astype(np.float32)
    rH = N(di.restrict_residual(T(u2), T(b), T(c), T(cH), rhs_zero=False))
    ref = M.restrict_residual(M.residual(u2, b, c), cH)
    assert np.abs(rH - ref).max() < 1e-4


@pytest.mark.parametrize("h,w", SIZES)
def test_prolong_both_modes(di, h, w):
    f, fn, c = _case(h, w, 2, 0.2, h * 19 + w)
    H, W = M.coarse_shape(h, w)
    g = np.random.default_rng(7)
    uH = g.uniform(0, 255, (2, H, W)).astype(np.float32)
    out = N(di.prolong(T(uH), T(c), 0, b=T(fn)))
    ref = M.prolong_solution(uH, f, c)
    assert np.abs(out - ref).max() < 1e-4
    assert np.array_equal(out[:, c == 1], f[:, c == 1])  # mask values exact
    u = g.uniform(0, 255, (2, h, w)).astype(np.float32)
    ut = T(u)
    di.prolong(T(uH), T(c), 1, u=ut)
    ref = M.prolong_correct(u, uH, c)
    out = N(ut)
    assert np.abs(out - ref).max() < 1e-4
    assert np.array_equal(out[:, c == 1], u[:, c == 1])


ORAS_CASES = [  # (h, w, block, overlap, iters)
    (32, 32, 32, 6, 8), (70, 95, 32, 6, 8), (77, 61, 16, 4, 6), (61, 77, 16, 2, 5),
    (45, 38, 8, 2, 4), (45, 38, 8, 4, 3), (40, 41, 8, 1, 4), (50, 33, 16, 1, 2),
    (130, 100, 32, 6, 0), (130, 100, 32, 6, 1), (9, 120, 32, 6, 8), (120, 9, 16, 4, 8),
    (70, 96, 32, 2, 8), (130, 100, 32, 2, 10), (33, 35, 32, 2, 4), (70, 95, 32, 3, 8),
]


@pytest.mark.parametrize("h,w,B,o,K", ORAS_CASES)
def test_oras_iteration_matches_oracle_cg(di, h, w, B, o, K):
    f, fn, c = _case(h, w, 2, 0.06, h * 23 + w + B)
    g = np.random.default_rng(8)
    # an iterate that equals b on the mask (cascadic form, b = C f) ...
    u = np.where(c.astype(bool), f, g.uniform(0, 255, f.shape)).astype(np.float32)
    with di.Context(block=B, overlap=o, alpha=0.5) as ctx:
        out = N(ctx.oras_iteration(T(u), T(fn), T(c), K, rhs_zero=True))
        ref = M.oras_iteration(u, M.rhs(f, c), c, B, o, 0.5, ("cg", K))
        scale = np.abs(ref - u).max()
        assert np.abs(out - ref).max() < 1e-3 * scale + 2e-4
        assert np.array_equal(out[:, c == 1], u[:, c == 1])
        # ... and the correction form (zero on the mask, general right-hand side)
        b = np.where(c.astype(bool), 0.0, g.normal(size=f.shape)).astype(np.float32)
        e = np.where(c.astype(bool), 0.0, g.normal(size=f.shape)).astype(np.float32)
        out = N(ctx.oras_iteration(T(e), T(b), T(c), K, rhs_zero=False))
        ref = M.oras_iteration(e, b, c, B, o, 0.5, ("cg", K))
        scale = np.abs(ref - e).max()
        assert np.abs(out - ref).max() < 1e-3 * scale + 1e-5


@pytest.mark.parametrize("B,o", [(32, 6), (16, 4), (8, 2)])
def test_oras_converged_local_solves_match_exact(di, B, o):
    # with enough local PCG steps each block solve is exact: compare with the
    # oracle's direct local solves (Algorithm 2 as printed)
    f, fn, c = _case(48, 53, 1, 0.08, 99 + B)
    g = np.random.default_rng(9)
    u = np.where(c.astype(bool), f, g.uniform(0, 255, f.shape)).astype(np.float32)
    with di.Context(block=B, overlap=o) as ctx:
        out = N(ctx.oras_iteration(T(u), T(fn), T(c), 3 * B * B, rhs_zero=True))
    ref = M.oras_iteration(u, M.rhs(f, c), c, B, o, 0.5, "exact")
    assert np.abs(out - ref).max() < 2e-3


def test_oras_is_deterministic(di):
    f, fn, c = _case(300, 257, 3, 0.05, 5)
    u = np.where(c.astype(bool), f, 100.0).astype(np.float32)
    with di.Context() as ctx:
        a = N(ctx.oras_iteration(T(u), T(fn), T(c), 8, rhs_zero=True))
        b = N(ctx.oras_iteration(T(u), T(fn), T(c), 8, rhs_zero=True))
    assert np.array_equal(a, b)


def test_oras_rejects_aliasing(di):
    f, fn, c = _case(40, 40, 1, 0.1, 1)
    with di.Context() as ctx:
        ut = T(f)
        with pytest.raises(di.DiError):
            ctx.oras_iteration(ut, T(fn), T(c), 4, rhs_zero=True, out=ut)


def _unaligned(a):
    # the same values in a tensor whose data starts 4 bytes past a 16-byte
    # boundary: the block kernel then copies its tiles with cp.async, not TMA
    flat = torch.empty(a.size + 1, dtype=torch.float32, device=DEV)
    v = flat[1:].view(a.shape)
    v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    assert v.data_ptr() % 16 == 4
    return v


@pytest.mark.parametrize("o,rhs_zero", [(2, True), (6, True), (2, False), (6, False)])
def test_oras_tma_and_cp_async_tiles_agree(di, o, rhs_zero):
    # widths that are multiples of 4 with 16-byte aligned images take the TMA
    # path; the same data 4 bytes off that alignment takes cp.async: identical
    # tiles, identical bits
    h, w = 70, 96
    f, fn, c = _case(h, w, 3, 0.06, 4242 + o)
    g = np.random.default_rng(9)
    u = np.where(c.astype(bool), f, g.uniform(0, 255, f.shape)).astype(np.float32)
    b = fn if rhs_zero else g.uniform(-5, 5, f.shape).astype(np.float32)
    with di.Context(block=32, overlap=o) as ctx:
        a = N(ctx.oras_iteration(T(u), T(b), T(c), 8, rhs_zero=rhs_zero))
        bq = N(ctx.oras_iteration(_unaligned(u), _unaligned(b), T(c), 8, rhs_zero=rhs_zero))
    assert np.array_equal(a, bq)
    assert np.isfinite(a).all()


@pytest.mark.parametrize("h,w", [(64, 96), (31, 130)])
def test_transfers_vector_and_scalar_paths_agree(di, h, w):
    # even widths with 8-byte aligned images take the 8-byte-word paths of the
    # restriction and prolongation, the same data 4 bytes off alignment the
    # scalar paths: identical bits
    f, fn, c = _case(h, w, 2, 0.05, 77 + w)
    g = np.random.default_rng(3)
    u = np.where(c.astype(bool), 0.0, g.normal(size=f.shape)).astype(np.float32)
    b = np.where(c.astype(bool), 0.0, g.normal(size=f.shape)).astype(np.float32)
    cH = T(M.mask_downsample(c))
    ra = N(di.restrict_residual(T(u), T(b), T(c), cH, rhs_zero=False))
    rb = N(di.restrict_residual(_unaligned(u), _unaligned(b), T(c), cH, rhs_zero=False))
    assert np.array_equal(ra, rb)
    H, W = M.coarse_shape(h, w)
    e = g.uniform(-3, 3, (2, H, W)).astype(np.float32)
    ua, ub = T(u), _unaligned(u)
    di.prolong(T(e), T(c), 1, u=ua)
    di.prolong(T(e), T(c), 1, u=ub)
    assert np.array_equal(N(ua), N(ub))
    pa = N(di.prolong(T(e), T(c), 0, b=T(fn)))
    pb = N(di.prolong(T(e), T(c), 0, b=_unaligned(fn)))
    assert np.array_equal(pa, pb)


PRO_CASES = [  # (h, w, overlap, rhs_zero, aligned)
    (70, 96, 2, True, True), (70, 96, 2, False, False), (70, 96, 6, False, True),
    (33, 35, 2, False, True), (130, 100, 2, True, False), (61, 250, 6, True, True),
    (1, 9, 2, False, True), (7, 1, 2, True, True), (3, 5, 6, False, False),
    (17, 33, 2, False, True), (95, 64, 4, False, True), (71, 96, 2, False, True),
    (129, 160, 6, True, True),
]


@pytest.mark.parametrize("h,w,o,rhs_zero,aligned", PRO_CASES)
def test_prolong_oras_iteration_bit_identical_to_two_steps(di, h, w, o, rhs_zero, aligned):
    # the decoder's correction step inside the first post-smoothing iteration
    # (mode 1): the same bits as the prolongation on a copy followed by the
    # plain iteration, through both tile paths (TMA where aligned) and the
    # ragged right and bottom blocks
    C = 3
    f, fn, c = _case(h, w, C, 0.08, 31 * h + w + o)
    g = np.random.default_rng(h + 7 * w)
    H, W = M.coarse_shape(h, w)
    if rhs_zero:
        u = np.where(c.astype(bool), f, g.uniform(0, 255, f.shape)).astype(np.float32)
        b = fn
    else:
        u = np.where(c.astype(bool), 0.0, g.normal(size=f.shape)).astype(np.float32)
        b = np.where(c.astype(bool), 0.0, g.normal(size=f.shape)).astype(np.float32)
    uH = g.normal(scale=4.0, size=(C, H, W)).astype(np.float32)
    put = T if aligned else _unaligned
    with di.Context(block=32, overlap=o) as ctx:
        ut = put(u)
        fused = N(ctx.prolong_oras_iteration(T(uH), ut, put(b), T(c), 8, rhs_zero=rhs_zero))
        assert np.array_equal(N(ut), u)  # u_in is not modified
        up = put(u)
        di.prolong(T(uH), T(c), 1, u=up)
        two = N(ctx.oras_iteration(up, put(b), T(c), 8, rhs_zero=rhs_zero))
    assert np.array_equal(fused, two)
    # and against the oracle's two steps
    start = M.prolong_correct(u.astype(np.float64), uH, c)
    ref = M.oras_iteration(start, M.rhs(f, c) if rhs_zero else b, c, 32, o, 0.5, ("cg", 8))
    scale = np.abs(ref - start).max() + np.abs(start).max() * 1e-5
    assert np.abs(fused - ref).max() < 1e-3 * scale + 2e-4


@pytest.mark.parametrize("h,w,o,aligned", [(70, 96, 2, True), (70, 96, 6, False),
                                           (33, 35, 2, True), (1, 9, 2, True),
                                           (130, 100, 2, False), (61, 250, 4, True)])
def test_prolong_oras_iteration_interpolation_bit_identical(di, h, w, o, aligned):
    # the cascade's step (mode 0): u_in = b (not finite off the mask, where it
    # must not be read), the start is b on the mask and P uH elsewhere
    C = 3
    f, fn, c = _case(h, w, C, 0.08, 17 * h + w + o)
    g = np.random.default_rng(2 * h + w)
    H, W = M.coarse_shape(h, w)
    uH = g.uniform(0, 255, size=(C, H, W)).astype(np.float32)
    put = T if aligned else _unaligned
    with di.Context(block=32, overlap=o) as ctx:
        fused = N(ctx.prolong_oras_iteration(T(uH), put(fn), put(fn), T(c), 8, rhs_zero=True,
                                             mode=0))
        start = di.prolong(T(uH), T(c), 0, b=put(fn))
        two = N(ctx.oras_iteration(start, put(fn), T(c), 8, rhs_zero=True))
    assert np.isfinite(fused).all()
    assert np.array_equal(fused, two)
    s0 = M.prolong_solution(uH, f, c)
    ref = M.oras_iteration(s0, M.rhs(f, c), c, 32, o, 0.5, ("cg", 8))
    assert np.abs(fused - ref).max() < 1e-3 * np.abs(ref - s0).max() + 2e-4


def test_prolong_oras_iteration_4k_rgb(di):
    # the finest level of the bench frames' size (3840 x 2160 x 3): bit-identical
    # to the two steps
    h, w, C = 2160, 3840, 3
    g = torch.Generator(device=DEV).manual_seed(5)
    c = (torch.rand((h, w), generator=g, device=DEV) < 0.04).to(torch.uint8)
    f = torch.rand((C, h, w), generator=g, device=DEV) * 255
    u = torch.where(c.bool(), f, torch.full_like(f, 128.0))
    uH = torch.randn((C, (h + 1) // 2, (w + 1) // 2), generator=g, device=DEV) * 4
    with di.Context(block=32, overlap=2) as ctx:
        fused = ctx.prolong_oras_iteration(uH, u, f, c, 10, rhs_zero=True)
        up = u.clone()
        di.prolong(uH, c, 1, u=up)
        two = ctx.oras_iteration(up, f, c, 10, rhs_zero=True)
    torch.cuda.synchronize()
    assert torch.equal(fused, two)


@pytest.mark.parametrize("kw", [dict(block=32, overlap=3), dict(block=16, overlap=2),
                                dict(block=32, overlap=2, precision=1)])
def test_prolong_oras_iteration_rejects_other_configurations(di, kw):
    f, fn, c = _case(40, 40, 1, 0.1, 3)
    uH = np.zeros((1, 20, 20), np.float32)
    with di.Context(**kw) as ctx:
        with pytest.raises(di.DiError):
            ctx.prolong_oras_iteration(T(uH), T(f), T(fn), T(c), 4, rhs_zero=True)

"""Plain FP64 restatement of each step of the reduced-FMG ORAS inpainting method.

TEST INFRASTRUCTURE ONLY: imported by the tests, the package smoke check and
the benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA path.  Every function is written from the paper's text, in its
order and notation; the readings taken where the text is silent or garbled are
stated beside the code.  Arrays are numpy float64; images are planar
[channels][height][width], masks uint8/bool [height][width] shared by channels.

Steps and where they come from:
  apply_A / residual        Section 2.2, eq. (2.6): A = C + (I - C) L, b = C f
  mask_downsample           Section 4.3, "Mask Downsampling" (2x2 max pooling)
  values_downsample_naive   Section 4.3, "Naive Mask Values Downsampling"
  values_downsample_modified Section 4.3, "Modified Mask Values Downsampling"
  restrict_residual         Section 4.4 ("simple averaging" outside the mask),
                            Algorithm 3 step 3, with the coarse-spacing factor 4
  prolong / prolong_*       Section 4.4 (bilinear; mask handling per mode)
  axis_blocks / axis_weights Section 3.1 (32x32 blocks, overlap 6, separable
                            linear partition-of-unity weights)
  local_operator / solve_*  Section 3, Algorithm 2 step 2 (A_i with Robin rows)
  oras_iteration            Algorithm 2
  vcycle                    Algorithm 3 applied recursively (Section 4.2)
  reduced_fmg               Section 4.2 (reduced FMG) and Section 4.4
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ----------------------------------------------------------------------------
# Operator (Section 2.2)
# ----------------------------------------------------------------------------


def neg_laplacian(u: np.ndarray) -> np.ndarray:
    """L u with the 5-point stencil, h = 1 and reflecting boundaries:
    (L u)_i = sum over in-image 4-neighbours j of (u_i - u_j)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    out[..., :, 1:] += u[..., :, 1:] - u[..., :, :-1]
    out[..., :, :-1] += u[..., :, :-1] - u[..., :, 1:]
    out[..., 1:, :] += u[..., 1:, :] - u[..., :-1, :]
    out[..., :-1, :] += u[..., :-1, :] - u[..., 1:, :]
    return out


def apply_A(u: np.ndarray, c: np.ndarray) -> np.ndarray:
    """A u with A = C + (I - C) L (eq. 2.6)."""
    cm = np.asarray(c).astype(bool)
    return np.where(cm, u, neg_laplacian(u))


def rhs(f: np.ndarray, c: np.ndarray) -> np.ndarray:
    """b = C f.  A select, not a product, so f at unknown pixels is never read."""
    cm = np.asarray(c).astype(bool)
    return np.where(cm, np.asarray(f, dtype=np.float64), 0.0)


def residual(u: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """r = b - A u (Algorithm 2, step 1)."""
    return np.asarray(b, dtype=np.float64) - apply_A(u, c)


# ----------------------------------------------------------------------------
# Grid hierarchy (Section 4.3, 4.4)
# ----------------------------------------------------------------------------


def coarse_shape(h: int, w: int) -> tuple[int, int]:
    """Dyadic coarsening; odd sizes round up, so an edge coarse cell may have
    only one or two fine children."""
    return (h + 1) // 2, (w + 1) // 2


def num_levels(h: int, w: int, block: int) -> int:
    """Levels such that the coarsest one fits in a single block (Section 4.4:
    8 levels for 3840x2160 with 32x32 blocks)."""
    n = 1
    while max(h, w) > block:
        h, w = coarse_shape(h, w)
        n += 1
    return n


def mask_downsample(c: np.ndarray) -> np.ndarray:
    """A coarse pixel is a mask pixel iff any of its fine children is
    (max pooling, Section 4.3)."""
    c = np.asarray(c).astype(np.uint8)
    h, w = c.shape
    H, W = coarse_shape(h, w)
    pad = np.zeros((2 * H, 2 * W), dtype=np.uint8)
    pad[:h, :w] = c
    return pad.reshape(H, 2, W, 2).max(axis=(1, 3)).astype(np.uint8)


def _children(a: np.ndarray, fill: float):
    """The four children of every coarse cell as arrays [.., H, W], plus a
    validity mask for children that lie inside the fine image."""
    h, w = a.shape[-2:]
    H, W = coarse_shape(h, w)
    pad = np.full(a.shape[:-2] + (2 * H, 2 * W), fill, dtype=np.float64)
    pad[..., :h, :w] = a
    valid = np.zeros((2 * H, 2 * W), dtype=bool)
    valid[:h, :w] = True
    kids, vkids = [], []
    for dy in (0, 1):
        for dx in (0, 1):
            kids.append(pad[..., dy::2, dx::2])
            vkids.append(valid[dy::2, dx::2])
    return kids, vkids


def values_downsample_naive(c: np.ndarray, b: np.ndarray) -> np.ndarray:
    """b_H = sum(c_h b_h) / max(1, sum c_h) over the 2x2 children."""
    kc, _ = _children(np.asarray(c, dtype=np.float64), 0.0)
    kb, _ = _children(rhs(b, c), 0.0)
    num = sum(kc[i] * kb[i] for i in range(4))
    den = np.maximum(1.0, sum(kc))
    return num / den


def modified_weights(c: np.ndarray, cH: np.ndarray) -> np.ndarray:
    """w_h = c_h (4 - sum of the masks of the four direct neighbours).

    Reading of the garbled formulas (the w^{3,4}, w^{4,3}, w^{4,4} lines list a
    diagonal child or one child twice): each fine pixel has two direct
    neighbours inside its own coarse cell, whose fine masks count, and two in
    the adjacent coarse cells, whose max-pooled coarse masks count, as the text
    before the formulas says.  A neighbour outside the image counts as a
    non-mask pixel.  Returned on the fine grid [h, w]."""
    c = np.asarray(c).astype(np.int64)
    cH = np.asarray(cH).astype(np.int64)
    h, w = c.shape
    H, W = cH.shape
    ys, xs = np.mgrid[0:h, 0:w]
    count = np.zeros((h, w), dtype=np.int64)
    # x direction: partner inside the cell is x^1; the outer neighbour is x-1
    # (x even) or x+1 (x odd), which lies in the coarse cell to the left/right.
    xin = xs ^ 1
    ok = xin < w
    count += np.where(ok, c[ys, np.minimum(xin, w - 1)], 0)
    xout = np.where(xs % 2 == 0, xs - 1, xs + 1)
    ok = (xout >= 0) & (xout < w)
    cx = np.clip(xout // 2, 0, W - 1)
    count += np.where(ok, cH[ys // 2, cx], 0)
    yin = ys ^ 1
    ok = yin < h
    count += np.where(ok, c[np.minimum(yin, h - 1), xs], 0)
    yout = np.where(ys % 2 == 0, ys - 1, ys + 1)
    ok = (yout >= 0) & (yout < h)
    cy = np.clip(yout // 2, 0, H - 1)
    count += np.where(ok, cH[cy, xs // 2], 0)
    return (c * (4 - count)).astype(np.float64)


def values_downsample_modified(c: np.ndarray, b: np.ndarray,
                               cH: np.ndarray | None = None) -> np.ndarray:
    """b_H = sum(w_h b_h) / max(1, sum w_h) with the weights above.

    Gap in the text: where the coarse cell is a mask pixel but every weight is
    0 (each fine mask child is surrounded by mask pixels), the printed formula
    would give 0 at a mask pixel; the naive average is used there instead."""
    if cH is None:
        cH = mask_downsample(c)
    wgt = modified_weights(c, cH)
    kw, _ = _children(wgt, 0.0)
    kb, _ = _children(rhs(b, c), 0.0)
    num = sum(kw[i] * kb[i] for i in range(4))
    den = sum(kw)
    mod = num / np.maximum(1.0, den)
    naive = values_downsample_naive(c, b)
    return np.where((den == 0) & (np.asarray(cH) > 0), naive, mod)


def restrict_residual(r: np.ndarray, cH: np.ndarray) -> np.ndarray:
    """Coarse right-hand side of the error equation.

    Outside the coarse mask the fine residual is averaged over the existing
    children (Section 4.4); the coarse operator is rediscretised with spacing
    H = 2h, which with the unit-spacing stencil used on every level means the
    average is multiplied by H^2/h^2 = 4.  At coarse mask pixels the error is
    0 (Section 4.4: corrections vanish at mask pixels), so the entry is 0."""
    kr, vk = _children(np.asarray(r, dtype=np.float64), 0.0)
    cnt = sum(v.astype(np.float64) for v in vk)
    mean = sum(kr) / cnt
    return np.where(np.asarray(cH).astype(bool), 0.0, 4.0 * mean)


def _prolong_axis(n: int, nc: int):
    x = np.arange(n)
    near = x // 2
    far = np.where(x % 2 == 0, near - 1, near + 1)
    far = np.clip(far, 0, nc - 1)
    return near, far


def prolong(uH: np.ndarray, h: int, w: int) -> np.ndarray:
    """Cell-centred bilinear interpolation: each fine pixel takes 9/16 of its
    parent, 3/16 of the two edge-adjacent coarse cells on its side and 1/16 of
    the diagonal one; coarse indices are clamped at the border (reflecting)."""
    uH = np.asarray(uH, dtype=np.float64)
    H, W = uH.shape[-2:]
    ny, fy = _prolong_axis(h, H)
    nx, fx = _prolong_axis(w, W)
    a = uH[..., ny[:, None], nx[None, :]]
    bx = uH[..., ny[:, None], fx[None, :]]
    by = uH[..., fy[:, None], nx[None, :]]
    d = uH[..., fy[:, None], fx[None, :]]
    return (9.0 * a + 3.0 * bx + 3.0 * by + d) / 16.0


def prolong_solution(uH: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Cascadic prolongation: interpolate, then impose u = b on the fine mask
    (the interpolation condition C P u_H = C f, Section 4.4)."""
    h, w = np.asarray(c).shape
    return np.where(np.asarray(c).astype(bool), np.asarray(b, dtype=np.float64),
                    prolong(uH, h, w))


def prolong_correct(u: np.ndarray, eH: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Correction step u + P e_H with the correction set to 0 on the fine mask
    (Algorithm 3 step 5, Section 4.4)."""
    h, w = np.asarray(c).shape
    e = prolong(eH, h, w)
    return np.asarray(u, dtype=np.float64) + np.where(np.asarray(c).astype(bool), 0.0, e)


# ----------------------------------------------------------------------------
# Block decomposition and partition of unity (Section 3.1)
# ----------------------------------------------------------------------------


def axis_blocks(n: int, block: int, overlap: int) -> list[tuple[int, int]]:
    """[start, end) of the blocks along one axis.  Starts are k*(B - o) for
    k < ceil((n - o)/(B - o)) (which gives the 36852 local problems of a 4K
    colour image, Section 3.1); the last block is clipped at the image edge,
    so every overlap is exactly o wide."""
    s = block - overlap
    nb = max(1, -(-(n - overlap) // s))
    return [(k * s, min(k * s + block, n)) for k in range(nb)]


def axis_weights(n: int, block: int, overlap: int) -> np.ndarray:
    """[num_blocks, n] one-dimensional weights: 0 outside the block, 1 in its
    non-shared part, and linear ramps in each overlap with weight 0 on the
    block's outermost pixel and 1 on the innermost (Section 3.1), so the two
    blocks sharing an overlap sum to 1.  An overlap of width 1 takes 1/2 each
    (the 0/1 rule cannot hold there)."""
    spans = axis_blocks(n, block, overlap)
    nb = len(spans)
    wts = np.zeros((nb, n), dtype=np.float64)
    for k, (a, e) in enumerate(spans):
        wk = np.ones(e - a, dtype=np.float64)
        if k > 0:
            wo = spans[k - 1][1] - a
            j = np.arange(wo, dtype=np.float64)
            wk[:wo] *= j / (wo - 1) if wo > 1 else 0.5
        if k < nb - 1:
            a2 = spans[k + 1][0]
            wo = e - a2
            j = np.arange(wo, dtype=np.float64)
            wk[a2 - a:] *= (1.0 - j / (wo - 1)) if wo > 1 else 0.5
        wts[k, a:e] = wk
    return wts


def block_count(h: int, w: int, channels: int, block: int, overlap: int) -> int:
    return len(axis_blocks(h, block, overlap)) * len(axis_blocks(w, block, overlap)) * channels


# ----------------------------------------------------------------------------
# Local problems (Section 3, Algorithm 2 step 2)
# ----------------------------------------------------------------------------


def local_operator(c: np.ndarray, y0: int, y1: int, x0: int, x1: int, alpha: float):
    """Coefficients of A_i on block [y0,y1) x [x0,x1).

    Rows of mask pixels are identity rows (v = r there).  For an unknown pixel
    the global row of A is kept for neighbours inside the block; a neighbour
    outside the image contributes nothing (reflecting boundary); a neighbour
    inside the image but outside the block lies across an inner subdomain
    boundary, where the Robin condition d_n v + alpha v = 0 is discretised
    with the ghost value (1 - alpha) v_i, adding alpha to the diagonal.
    Returns (diag[hb, wb], couple[4, hb, wb]) for the neighbours
    (left, right, up, down): 1.0 where the neighbour is an in-block unknown
    that enters the row with coefficient -1, else 0; and mask[hb, wb]."""
    H, W = np.asarray(c).shape
    cb = np.asarray(c)[y0:y1, x0:x1].astype(bool)
    hb, wb = cb.shape
    ys, xs = np.mgrid[y0:y1, x0:x1]
    diag = np.zeros((hb, wb), dtype=np.float64)
    couple = np.zeros((4, hb, wb), dtype=np.float64)
    offs = [(0, -1), (0, 1), (-1, 0), (1, 0)]
    for k, (dy, dx) in enumerate(offs):
        ny, nx = ys + dy, xs + dx
        in_img = (ny >= 0) & (ny < H) & (nx >= 0) & (nx < W)
        in_blk = (ny >= y0) & (ny < y1) & (nx >= x0) & (nx < x1)
        diag += np.where(in_img & in_blk, 1.0, 0.0)
        diag += np.where(in_img & ~in_blk, alpha, 0.0)
        nb_unknown = np.zeros_like(cb)
        sel = in_blk
        nb_unknown[sel] = ~cb[(ny - y0)[sel], (nx - x0)[sel]]
        couple[k] = np.where(in_blk & nb_unknown & ~cb, 1.0, 0.0)
    diag = np.where(cb, 1.0, diag)
    return diag, couple, cb


def local_matrix(c, y0, y1, x0, x1, alpha) -> sp.csr_matrix:
    """A_i as a sparse matrix over the block's pixels in row-major order.
    Mask-neighbour entries of unknown rows are kept (v_j = r_j enters them)."""
    diag, couple, cb = local_operator(c, y0, y1, x0, x1, alpha)
    hb, wb = cb.shape
    idx = np.arange(hb * wb).reshape(hb, wb)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [diag.ravel()]
    offs = [(0, -1), (0, 1), (-1, 0), (1, 0)]
    for dy, dx in offs:
        ys, xs = np.mgrid[0:hb, 0:wb]
        ny, nx = ys + dy, xs + dx
        ok = (ny >= 0) & (ny < hb) & (nx >= 0) & (nx < wb) & ~cb
        rows.append(idx[ok])
        cols.append(idx[ny[ok], nx[ok]])
        vals.append(-np.ones(int(ok.sum())))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(hb * wb, hb * wb))


def solve_local_exact(c, y0, y1, x0, x1, alpha, rb: np.ndarray) -> np.ndarray:
    """v_i = A_i^{-1} R_i r for every channel of rb [C, hb, wb]."""
    A = local_matrix(c, y0, y1, x0, x1, alpha).tocsc()
    lu = spla.splu(A)
    C, hb, wb = rb.shape
    out = np.empty_like(rb, dtype=np.float64)
    for ch in range(C):
        out[ch] = lu.solve(rb[ch].reshape(-1).astype(np.float64)).reshape(hb, wb)
    return out


def _apply_local(diag, couple, cb, v):
    """A_i v restricted to unknown rows (mask entries of v are 0)."""
    q = diag * v
    q[..., :, 1:] -= couple[0][:, 1:] * v[..., :, :-1]
    q[..., :, :-1] -= couple[1][:, :-1] * v[..., :, 1:]
    q[..., 1:, :] -= couple[2][1:, :] * v[..., :-1, :]
    q[..., :-1, :] -= couple[3][:-1, :] * v[..., 1:, :]
    return np.where(cb, 0.0, q)


def solve_local_cg(c, y0, y1, x0, x1, alpha, rb: np.ndarray, iters: int) -> np.ndarray:
    """`iters` steps of plain conjugate gradients (Hestenes-Stiefel; Section
    3.1 solves the local problems with unpreconditioned CG) on A_i v = R_i r
    from v = 0, over the unknown pixels of the block; v = r at mask pixels (the scheduler keeps r = 0 there).  Breakdown
    guards: a step with p.Ap <= 0 takes alpha = 0, and r.r = 0 gives beta = 0
    (both happen only when the block's residual is exactly zero).  The paper
    stops its local CG at a fraction of the global residual; a fixed step
    count is this build's reading."""
    diag, couple, cb = local_operator(c, y0, y1, x0, x1, alpha)
    rb = np.asarray(rb, dtype=np.float64)
    v = np.zeros_like(rb)
    r = np.where(cb, 0.0, rb)
    for ch in range(rb.shape[0]):
        x = v[ch]
        rr = r[ch].copy()
        p = rr.copy()
        rho = float((rr * rr).sum())
        for _ in range(iters):
            q = _apply_local(diag, couple, cb, p)
            pq = float((p * q).sum())
            a = rho / pq if pq > 0.0 else 0.0
            x += a * p
            rr -= a * q
            rho_new = float((rr * rr).sum())
            beta = rho_new / rho if rho > 0.0 else 0.0
            rho = rho_new
            p = rr + beta * p
        v[ch] = x
    return np.where(cb, rb, v)


# ----------------------------------------------------------------------------
# ORAS (Algorithm 2), V-cycle (Algorithm 3, Section 4.2), reduced FMG
# ----------------------------------------------------------------------------


def oras_iteration(u, b, c, block=32, overlap=6, alpha=0.5, local="exact"):
    """One ORAS iteration (Algorithm 2): r = b - A u; A_i v_i = R_i r for every
    block; u + sum_i R_i^T D_i v_i.  local = "exact" or ("cg", iters)."""
    u = np.asarray(u, dtype=np.float64)
    if u.ndim == 2:
        u = u[None]
    b = np.asarray(b, dtype=np.float64).reshape(u.shape)
    H, W = u.shape[-2:]
    r = residual(u, b, c)
    wy = axis_weights(H, block, overlap)
    wx = axis_weights(W, block, overlap)
    du = np.zeros_like(u)
    for ky, (y0, y1) in enumerate(axis_blocks(H, block, overlap)):
        for kx, (x0, x1) in enumerate(axis_blocks(W, block, overlap)):
            rb = r[:, y0:y1, x0:x1]
            if local == "exact":
                v = solve_local_exact(c, y0, y1, x0, x1, alpha, rb)
            else:
                v = solve_local_cg(c, y0, y1, x0, x1, alpha, rb, int(local[1]))
            d = wy[ky, y0:y1][:, None] * wx[kx, x0:x1][None, :]
            du[:, y0:y1, x0:x1] += d * v
    return u + du


def build_pyramid(f, c, block, downsample="modified"):
    """[(c_l, b_l)] from finest (l = 0) to coarsest; b_0 = C f."""
    c0 = np.asarray(c).astype(np.uint8)
    b0 = rhs(f, c0)
    if b0.ndim == 2:
        b0 = b0[None]
    levels = [(c0, b0)]
    h, w = c0.shape
    for _ in range(num_levels(h, w, block) - 1):
        cf, bf = levels[-1]
        cH = mask_downsample(cf)
        if downsample == "modified":
            bH = values_downsample_modified(cf, bf, cH)
        else:
            bH = values_downsample_naive(cf, bf)
        bH = np.where(cH.astype(bool), bH, 0.0)
        levels.append((cH, bH))
    return levels


def vcycle(levels, l, u, b, block, overlap, alpha, local, pre=1, post=1,
           coarse_local="exact"):
    """Algorithm 3 with the coarse solve replaced recursively by the same cycle;
    on the coarsest level (one block) a single ORAS iteration with the local
    solver `coarse_local` solves the problem."""
    c = levels[l][0]
    if l == len(levels) - 1:
        return oras_iteration(u, b, c, block, overlap, alpha, coarse_local)
    for _ in range(pre):
        u = oras_iteration(u, b, c, block, overlap, alpha, local)
    r = residual(u, b, c)
    cH = levels[l + 1][0]
    rH = restrict_residual(r, cH)
    eH = vcycle(levels, l + 1, np.zeros_like(rH), rH, block, overlap, alpha, local, pre, post,
                coarse_local)
    u = prolong_correct(u, eH, c)
    for _ in range(post):
        u = oras_iteration(u, b, c, block, overlap, alpha, local)
    return u


def reduced_fmg(f, c, cycles=1, block=32, overlap=6, alpha=0.5, local="exact",
                downsample="modified", coarse_local=None, history=None):
    """Reduced FMG (Section 4.2, Fig. 4; Section 4.4): a one-way cascade from
    the coarsest level with a single ORAS iteration per level, then `cycles`
    V(1,1)-cycles on the finest level.  coarse_local sets the local solver of
    the coarsest level (default: exact).  If `history` is a list, the iterate
    after the cascade and after every cycle is appended to it."""
    levels = build_pyramid(f, c, block, downsample)
    if coarse_local is None:
        coarse_local = "exact"
    L = len(levels)
    cL, bL = levels[-1]
    u = np.where(cL.astype(bool), bL, 0.0)
    u = oras_iteration(u, bL, cL, block, overlap, alpha, coarse_local)
    for l in range(L - 2, -1, -1):
        cl, bl = levels[l]
        u = prolong_solution(u, bl, cl)
        u = oras_iteration(u, bl, cl, block, overlap, alpha, local)
    if history is not None:
        history.append(u.copy())
    b0 = levels[0][1]
    for _ in range(cycles):
        u = vcycle(levels, 0, u, b0, block, overlap, alpha, local, 1, 1, coarse_local)
        if history is not None:
            history.append(u.copy())
    return u

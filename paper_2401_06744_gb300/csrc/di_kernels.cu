// CUDA kernels (sm_103a) of the reduced-FMG ORAS inpainting decoder.
//
// Problem (Section 2.2, eq. 2.6): (C + (I - C) L) u = C f per channel, L the
// 5-point negated Laplacian with reflecting boundaries and unit spacing on
// every level (coarse right-hand sides carry the (H/h)^2 = 4 factor).
//
// Kernels:
//   k_count_mask     known / unknown pixel counts of the finest mask
//   k_mask_down      Section 4.3 mask downsampling (2x2 max pooling)
//   k_values_down    Section 4.3 modified (or naive) mask-value downsampling
//   k_residual       r = b - A u with per-CTA partial sums of r^2 (Algorithm 2 step 1)
//   k_reduce         fixed-order sum of the partials (one global scalar product)
//   k_restrict       Algorithm 3 steps 2-3 fused: residual + 2x2 averaging (x4)
//   k_prolong        Section 4.4 bilinear prolongation, cascadic or correction mode
//   k_select         u = c ? b : 0
//   k_oras_block     Algorithm 2 step 2 and the D_i-weighted part of step 3:
//                    one CTA per (block, channel); the block and a one-pixel
//                    halo are staged in shared memory and the local Robin
//                    problem is solved there by Jacobi-PCG held in registers
//   k_oras_combine   Algorithm 2 step 3 for pixels shared by several blocks:
//                    sums the weighted block contributions in a fixed order
//
// Layout: images planar [C][h][w] float32, masks [h][w] uint8.  The ORAS
// block pass writes pixels that only one block weights (weight 1) straight to
// u_out and parks weighted contributions of shared pixels in four parity
// planes [4][C][h][w] (blocks with equal (kx & 1, ky & 1) never overlap, so
// every plane pixel has one writer); the combine pass adds them in a fixed
// order, which keeps the result deterministic without atomics.
#include "di_internal.h"

#include <cfloat>
#include <cmath>

namespace di {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, d));
    return v;
}

// Weight of block k (of nb along this axis, stride s, overlap o) at local
// coordinate l: linear ramps with 0 at the block's outermost overlap pixel and
// 1 at its innermost one (Section 3.1); 1/2 for an overlap of width 1.
__device__ __forceinline__ float axis_weight(int l, int k, int nb, int s, int o) {
    float wgt = 1.f;
    if (k > 0 && l < o) wgt *= (o == 1) ? 0.5f : (float)l / (float)(o - 1);
    if (k < nb - 1 && l >= s) {
        const int j = l - s;
        wgt *= (o == 1) ? 0.5f : 1.f - (float)j / (float)(o - 1);
    }
    return wgt;
}

// Blocks with nonzero weight at global coordinate g along one axis: returns
// 1 (k0) or 2 (k0 < k1).
__device__ __forceinline__ int axis_contrib(int g, int s, int o, int nb, int& k0, int& k1) {
    int k = g / s;
    if (k > nb - 1) k = nb - 1;
    const int j = g - k * s;
    k1 = k;
    if (k > 0 && j < o) {
        if (o == 1) { k0 = k - 1; return 2; }
        if (j == 0) { k0 = k - 1; return 1; }
        if (j == o - 1) { k0 = k; return 1; }
        k0 = k - 1;
        return 2;
    }
    k0 = k;
    return 1;
}

// ---------------------------------------------------------------------------
// Mask pyramid (Section 4.3)
// ---------------------------------------------------------------------------

__global__ void k_count_mask(const uint8_t* __restrict__ c, size_t n,
                             unsigned long long* __restrict__ out) {
    unsigned known = 0, unknown = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        if (c[i]) ++known; else ++unknown;
    }
    for (int d = 16; d > 0; d >>= 1) {
        known += __shfl_xor_sync(kFull, known, d);
        unknown += __shfl_xor_sync(kFull, unknown, d);
    }
    if ((threadIdx.x & 31) == 0) {
        if (known) atomicAdd(&out[0], (unsigned long long)known);
        if (unknown) atomicAdd(&out[1], (unsigned long long)unknown);
    }
}

__global__ void k_mask_down(const uint8_t* __restrict__ c, int w, int h,
                            uint8_t* __restrict__ cH, int wH, int hH,
                            unsigned long long* __restrict__ unknownH) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    bool unk = false;
    if (X < wH && Y < hH) {
        const int x = 2 * X, y = 2 * Y;
        const bool x1 = x + 1 < w, y1 = y + 1 < h;
        const uint8_t* row = c + (size_t)y * w;
        bool m = row[x] != 0;
        if (x1) m |= row[x + 1] != 0;
        if (y1) {
            const uint8_t* row2 = row + w;
            m |= row2[x] != 0;
            if (x1) m |= row2[x + 1] != 0;
        }
        cH[(size_t)Y * wH + X] = m ? 1 : 0;
        unk = !m;
    }
    if (unknownH) {
        const unsigned bal = __ballot_sync(kFull, unk);
        const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
        if (lane == 0 && bal) atomicAdd(unknownH, (unsigned long long)__popc(bal));
    }
}

// One coarse cell: weights of its (up to four) fine children.
__global__ void k_values_down(const uint8_t* __restrict__ c, const float* __restrict__ b,
                              int w, int h, int C, const uint8_t* __restrict__ cH,
                              float* __restrict__ bH, int wH, int hH, int modified) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    if (X >= wH || Y >= hH) return;
    const size_t n = (size_t)w * h, nH = (size_t)wH * hH, P = (size_t)Y * wH + X;
    if (!cH[P]) {
        for (int ch = 0; ch < C; ++ch) bH[ch * nH + P] = 0.f;
        return;
    }
    float wt[4];
    size_t idx[4];
    float den = 0.f, cnt = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = 2 * X + (k & 1), y = 2 * Y + (k >> 1);
        wt[k] = 0.f;
        idx[k] = 0;
        if (x >= w || y >= h) continue;
        const size_t p = (size_t)y * w + x;
        idx[k] = p;
        if (!c[p]) continue;
        cnt += 1.f;
        if (!modified) { wt[k] = 1.f; continue; }
        int m = 0;
        const int xi = x ^ 1, yi = y ^ 1;               // partners inside the cell
        if (xi < w) m += c[(size_t)y * w + xi] != 0;
        if (yi < h) m += c[(size_t)yi * w + x] != 0;
        const int xo = (x & 1) ? x + 1 : x - 1;          // neighbours across the cell
        const int yo = (y & 1) ? y + 1 : y - 1;
        if (xo >= 0 && xo < w) m += cH[(size_t)Y * wH + (xo >> 1)] != 0;
        if (yo >= 0 && yo < h) m += cH[(size_t)(yo >> 1) * wH + X] != 0;
        wt[k] = (float)(4 - m);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) den += wt[k];
    if (den == 0.f) {  // gap of the printed rule: fall back to the naive average
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = 2 * X + (k & 1), y = 2 * Y + (k >> 1);
            wt[k] = (x < w && y < h && c[idx[k]]) ? 1.f : 0.f;
        }
        den = cnt;
    }
    const float inv = 1.f / fmaxf(1.f, den);
    for (int ch = 0; ch < C; ++ch) {
        const float* bc = b + ch * n;
        float num = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (wt[k] != 0.f) num += wt[k] * bc[idx[k]];
        bH[ch * nH + P] = num * inv;
    }
}

// ---------------------------------------------------------------------------
// Residual and its norm (Algorithm 2 step 1; Section 2.2 "single global scalar
// product")
// ---------------------------------------------------------------------------

__device__ __forceinline__ float residual_at(const float* __restrict__ u, int zero_u,
                                             const float* __restrict__ b, int rhs_zero,
                                             const uint8_t* __restrict__ c, int w, int h,
                                             int x, int y) {
    const size_t p = (size_t)y * w + x;
    if (c[p]) return b[p] - (zero_u ? 0.f : u[p]);
    const float rhs = rhs_zero ? 0.f : b[p];
    if (zero_u) return rhs;
    const float uc = u[p];
    float lu = 0.f;
    if (x > 0) lu += uc - u[p - 1];
    if (x < w - 1) lu += uc - u[p + 1];
    if (y > 0) lu += uc - u[p - w];
    if (y < h - 1) lu += uc - u[p + w];
    return rhs - lu;
}

constexpr int kResBX = 32, kResBY = 8;

__global__ void __launch_bounds__(kResBX * kResBY)
k_residual(const float* __restrict__ u, int zero_u, const float* __restrict__ b, int rhs_zero,
           const uint8_t* __restrict__ c, int w, int h, float* __restrict__ r,
           double* __restrict__ partials) {
    const int x = blockIdx.x * kResBX + threadIdx.x;
    const int y = blockIdx.y * kResBY + threadIdx.y;
    const int ch = blockIdx.z;
    const size_t n = (size_t)w * h;
    float rv = 0.f;
    if (x < w && y < h) {
        rv = residual_at(u + ch * n, zero_u, b + ch * n, rhs_zero, c, w, h, x, y);
        if (r) r[ch * n + (size_t)y * w + x] = rv;
    }
    __shared__ double s_part[kResBX * kResBY / 32];
    const int t = threadIdx.y * kResBX + threadIdx.x;
    double v = warp_sum_d((double)rv * (double)rv);
    if ((t & 31) == 0) s_part[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int i = 0; i < kResBX * kResBY / 32; ++i) s += s_part[i];
        const size_t nparts = (size_t)gridDim.x * gridDim.y;
        partials[ch * nparts + (size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256)
k_reduce(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
    const int ch = blockIdx.x;
    const double* p = partials + (size_t)ch * nparts;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += p[i];
    __shared__ double s_w[8];
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_w[i];
        out[ch] = t;
    }
}

// ---------------------------------------------------------------------------
// Grid transfers (Algorithm 3, Section 4.4)
// ---------------------------------------------------------------------------

__global__ void k_restrict(const float* __restrict__ u, const float* __restrict__ b,
                           int rhs_zero, const uint8_t* __restrict__ c, int w, int h,
                           const uint8_t* __restrict__ cH, float* __restrict__ rH, int wH,
                           int hH) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    const int ch = blockIdx.z;
    if (X >= wH || Y >= hH) return;
    const size_t n = (size_t)w * h, nH = (size_t)wH * hH, P = (size_t)Y * wH + X;
    if (cH[P]) { rH[ch * nH + P] = 0.f; return; }
    const float* uc = u + ch * n;
    const float* bc = b + ch * n;
    float sum = 0.f;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = 2 * X + (k & 1), y = 2 * Y + (k >> 1);
        if (x >= w || y >= h) continue;
        sum += residual_at(uc, 0, bc, rhs_zero, c, w, h, x, y);
        ++cnt;
    }
    rH[ch * nH + P] = 4.f * sum / (float)cnt;
}

// One thread per fine pixel column position; each CTA walks down rows with a
// stride so the grid stays a few thousand CTAs and the per-CTA maximum of the
// correction costs one atomic per CTA.
__global__ void __launch_bounds__(256)
k_prolong(const float* __restrict__ uH, int wH, int hH, const float* __restrict__ b,
          const uint8_t* __restrict__ c, int w, int h, float* __restrict__ u, int mode,
          unsigned* __restrict__ maxupd) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.z;
    const size_t n = (size_t)w * h, nH = (size_t)wH * hH;
    const float* e = uH + ch * nH;
    float amax = 0.f;
    if (x < w) {
        const int X = x >> 1;
        const int Xf = min(max((x & 1) ? X + 1 : X - 1, 0), wH - 1);
        for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < h;
             y += gridDim.y * blockDim.y) {
            const size_t p = (size_t)y * w + x;
            if (c[p]) {
                if (mode == 0) u[ch * n + p] = b[ch * n + p];
                continue;
            }
            const int Y = y >> 1;
            const int Yf = min(max((y & 1) ? Y + 1 : Y - 1, 0), hH - 1);
            const float v = (9.f * e[(size_t)Y * wH + X] + 3.f * e[(size_t)Y * wH + Xf] +
                             3.f * e[(size_t)Yf * wH + X] + e[(size_t)Yf * wH + Xf]) *
                            (1.f / 16.f);
            if (mode == 0) u[ch * n + p] = v;
            else { u[ch * n + p] += v; amax = fmaxf(amax, fabsf(v)); }
        }
    }
    if (maxupd) {
        __shared__ float s_m[8];
        const int t = threadIdx.y * blockDim.x + threadIdx.x;
        amax = warp_max(amax);
        if ((t & 31) == 0) s_m[t >> 5] = amax;
        __syncthreads();
        if (t == 0) {
            float m = 0.f;
            for (int i = 0; i < (int)(blockDim.x * blockDim.y) / 32; ++i) m = fmaxf(m, s_m[i]);
            if (m > 0.f) atomicMax(maxupd, __float_as_uint(m));
        }
    }
}

__global__ void k_select(const float* __restrict__ b, const uint8_t* __restrict__ c, size_t n,
                         float* __restrict__ u) {
    const int ch = blockIdx.y;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        u[ch * n + i] = c[i] ? b[ch * n + i] : 0.f;
}

// ---------------------------------------------------------------------------
// ORAS (Algorithm 2)
// ---------------------------------------------------------------------------

// One CTA solves one block of one channel.  Thread t owns column lx = t % B of
// the block and the R rows [strip * R, strip * R + R) with strip = t / B, so a
// B-lane segment of a warp covers R full rows: horizontal neighbours come from
// lane shuffles, vertical ones from registers, and only the strip ends go
// through shared memory.  Pixels of a block clipped at the image edge that
// fall outside the image are inert (zero rows, zero couplings).
template <int B, int R>
__global__ void __launch_bounds__(B * B / R)
k_oras_block(const float* __restrict__ u_in, int zero_in, const float* __restrict__ rhs,
             int rhs_zero, const uint8_t* __restrict__ c, int w, int h, int o, int nbx, int nby,
             float alpha, int iters, float rtol2, float* __restrict__ u_out,
             float* __restrict__ planes, unsigned* __restrict__ maxupd) {
    constexpr int T = B * B / R;
    constexpr int NS = B / R;
    constexpr int NW = T / 32;
    static_assert(T % 32 == 0 && B <= 32 && R <= 32, "block shape");

    const int s = B - o;
    const int kx = blockIdx.x % nbx, ky = blockIdx.x / nbx;
    const int ch = blockIdx.y, C = gridDim.y;
    const int x0 = kx * s, y0 = ky * s;
    const int bw = min(B, w - x0), bh = min(B, h - y0);
    const size_t n = (size_t)w * h;
    const float* uc = u_in + ch * n;

    __shared__ float s_u[B + 2][B + 3];
    __shared__ uint8_t s_c[B][B + 4];
    __shared__ float s_ztop[NS][B], s_zbot[NS][B];
    __shared__ float s_red1[NW], s_red2[NW], s_max[NW];

    const int t = threadIdx.x;
    const int lx = t % B, strip = t / B;
    const int lane = t & 31, warp = t >> 5;

    for (int i = t; i < (B + 2) * (B + 2); i += T) {
        const int yy = i / (B + 2), xx = i % (B + 2);
        const int gy = y0 - 1 + yy, gx = x0 - 1 + xx;
        float v = 0.f;
        if (!zero_in && gy >= 0 && gy < h && gx >= 0 && gx < w) v = uc[(size_t)gy * w + gx];
        s_u[yy][xx] = v;
    }
    for (int i = t; i < B * B; i += T) {
        const int yy = i / B, xx = i % B;
        s_c[yy][xx] = (yy < bh && xx < bw) ? (c[(size_t)(y0 + yy) * w + x0 + xx] != 0) : 1;
    }
    __syncthreads();

    // Local operator A_i: every unknown pixel couples with -1 to its in-block
    // 4-neighbours; its diagonal counts in-block neighbours (1 each) and
    // in-image neighbours across the block edge (Robin: alpha each), while
    // image edges add nothing (reflecting).  Search directions vanish on mask
    // pixels and outside the block (z = D^-1 r with D^-1 = 0 there), so the
    // stencil needs no per-neighbour coupling flags: only the lanes at the
    // block's left and right edges drop the wrapped-around shuffle value.
    float x[R], r[R], p[R], z[R], dg[R], di[R];
    unsigned act = 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int ly = strip * R + i;
        const int gx = x0 + lx, gy = y0 + ly;
        x[i] = 0.f;
        r[i] = 0.f;
        dg[i] = 0.f;
        di[i] = 0.f;
        if (lx < bw && ly < bh && !s_c[ly][lx]) {
            float diag = 0.f, nb = 0.f;
            int deg = 0;
            if (gx > 0) { ++deg; nb += s_u[ly + 1][lx]; diag += lx > 0 ? 1.f : alpha; }
            if (gx < w - 1) { ++deg; nb += s_u[ly + 1][lx + 2]; diag += lx + 1 < bw ? 1.f : alpha; }
            if (gy > 0) { ++deg; nb += s_u[ly][lx + 1]; diag += ly > 0 ? 1.f : alpha; }
            if (gy < h - 1) { ++deg; nb += s_u[ly + 2][lx + 1]; diag += ly + 1 < bh ? 1.f : alpha; }
            const float bb = rhs_zero ? 0.f : rhs[ch * n + (size_t)gy * w + gx];
            r[i] = bb - ((float)deg * s_u[ly + 1][lx + 1] - nb);
            dg[i] = diag;
            di[i] = 1.f / diag;
            act |= 1u << i;
        }
    }
    const float ml = lx > 0 ? 1.f : 0.f;
    const float mr = lx < B - 1 ? 1.f : 0.f;

    // z = D^-1 r, p = z, rho = r.z
    float rz = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        z[i] = di[i] * r[i];
        p[i] = z[i];
        rz += r[i] * z[i];
    }
    s_ztop[strip][lx] = z[0];
    s_zbot[strip][lx] = z[R - 1];
    rz = warp_sum(rz);
    if (lane == 0) s_red2[warp] = rz;
    __syncthreads();
    rz = 0.f;
#pragma unroll
    for (int i = 0; i < NW; ++i) rz += s_red2[i];
    float pu = strip > 0 ? s_zbot[strip - 1][lx] : 0.f;       // p of the row above the strip
    float pd = strip < NS - 1 ? s_ztop[strip + 1][lx] : 0.f;  // p of the row below
    // Stop once r.z <= max(rtol2, 1e-14) * (r.z)_0.  1e-14 is the FP32
    // floor (relative residual ~1e-7): iterating past it only feeds rounding
    // noise back into x.  rz and pq are identical in every thread, so every
    // exit below is taken by the whole block at once.
    const float rz_stop = fmaxf(rtol2, 1e-14f) * rz;

    for (int it = 0; it < iters; ++it) {
        if (!(rz > rz_stop)) break;
        float q[R];
        float pq = 0.f;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const float left = __shfl_up_sync(kFull, p[i], 1, B);
            const float right = __shfl_down_sync(kFull, p[i], 1, B);
            const float up = i > 0 ? p[i - 1] : pu;
            const float dn = i < R - 1 ? p[i + 1] : pd;
            float nbs = up + dn;
            nbs = fmaf(ml, left, nbs);
            nbs = fmaf(mr, right, nbs);
            q[i] = ((act >> i) & 1u) ? fmaf(dg[i], p[i], -nbs) : 0.f;
            pq = fmaf(p[i], q[i], pq);
        }
        pq = warp_sum(pq);
        if (lane == 0) s_red1[warp] = pq;
        __syncthreads();
        pq = 0.f;
#pragma unroll
        for (int i = 0; i < NW; ++i) pq += s_red1[i];
        if (!(pq > 0.f) || pq == INFINITY) break;
        const float a = rz / pq;
        float rzn = 0.f;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            x[i] = fmaf(a, p[i], x[i]);
            r[i] = fmaf(-a, q[i], r[i]);
            z[i] = di[i] * r[i];
            rzn = fmaf(r[i], z[i], rzn);
        }
        s_ztop[strip][lx] = z[0];
        s_zbot[strip][lx] = z[R - 1];
        rzn = warp_sum(rzn);
        if (lane == 0) s_red2[warp] = rzn;
        __syncthreads();
        rzn = 0.f;
#pragma unroll
        for (int i = 0; i < NW; ++i) rzn += s_red2[i];
        const float beta = rzn / rz;
        rz = rzn;
#pragma unroll
        for (int i = 0; i < R; ++i) p[i] = fmaf(beta, p[i], z[i]);
        pu = strip > 0 ? fmaf(beta, pu, s_zbot[strip - 1][lx]) : 0.f;
        pd = strip < NS - 1 ? fmaf(beta, pd, s_ztop[strip + 1][lx]) : 0.f;
    }

    // u_out = u_in + sum_i R_i^T D_i v_i: weight-1 pixels directly, shared
    // pixels through the parity planes.
    const int par = (kx & 1) | ((ky & 1) << 1);
    float* plane = planes + ((size_t)par * C + ch) * n;
    float* uo = u_out + ch * n;
    const float wx = axis_weight(lx, kx, nbx, s, o);
    float vmax = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int ly = strip * R + i;
        if (lx < bw && ly < bh) {
            const size_t gp = (size_t)(y0 + ly) * w + x0 + lx;
            const float v = ((act >> i) & 1u) ? x[i] : 0.f;
            const float d = wx * axis_weight(ly, ky, nby, s, o);
            if (d == 1.f) uo[gp] = s_u[ly + 1][lx + 1] + v;
            else if (d > 0.f) plane[gp] = d * v;
            if (d > 0.f) vmax = fmaxf(vmax, fabsf(v));
        }
    }
    if (maxupd) {
        vmax = warp_max(vmax);
        if (lane == 0) s_max[warp] = vmax;
        __syncthreads();
        if (t == 0) {
            float m = 0.f;
            for (int i = 0; i < NW; ++i) m = fmaxf(m, s_max[i]);
            if (m > 0.f) atomicMax(maxupd, __float_as_uint(m));
        }
    }
}

__global__ void k_oras_combine(const float* __restrict__ u_in, int zero_in,
                               const float* __restrict__ planes, int w, int h, int s, int o,
                               int nbx, int nby, float* __restrict__ u_out) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    const int gy = blockIdx.y * blockDim.y + threadIdx.y;
    const int ch = blockIdx.z, C = gridDim.z;
    if (gx >= w || gy >= h) return;
    int kx0, kx1, ky0, ky1;
    const int nx = axis_contrib(gx, s, o, nbx, kx0, kx1);
    const int ny = axis_contrib(gy, s, o, nby, ky0, ky1);
    if (nx == 1 && ny == 1) return;  // written by the block pass
    const size_t n = (size_t)w * h, gp = (size_t)gy * w + gx;
    float acc = 0.f;
    for (int a = 0; a < ny; ++a) {
        const int ky = a ? ky1 : ky0;
        for (int bb = 0; bb < nx; ++bb) {
            const int kx = bb ? kx1 : kx0;
            const int par = (kx & 1) | ((ky & 1) << 1);
            acc += planes[((size_t)par * C + ch) * n + gp];
        }
    }
    const float uo = zero_in ? 0.f : u_in[ch * n + gp];
    u_out[ch * n + gp] = uo + acc;
}

inline dim3 grid2(int w, int h, dim3 blk, int z = 1) {
    return dim3((unsigned)((w + blk.x - 1) / blk.x), (unsigned)((h + blk.y - 1) / blk.y),
                (unsigned)z);
}

template <int B, int R>
cudaError_t launch_oras_t(const float* u_in, int zero_in, const float* rhs, int rhs_zero,
                          const uint8_t* c, int w, int h, int C, int o, float alpha, int iters,
                          float rtol2, float* u_out, float* planes, unsigned* maxupd,
                          cudaStream_t s) {
    const int nbx = axis_blocks(w, B, o), nby = axis_blocks(h, B, o);
    dim3 grid((unsigned)(nbx * nby), (unsigned)C);
    k_oras_block<B, R><<<grid, B * B / R, 0, s>>>(u_in, zero_in, rhs, rhs_zero, c, w, h, o, nbx,
                                                  nby, alpha, iters, rtol2, u_out, planes,
                                                  maxupd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Overlap 2 gives 0/1 weights: no pixel is shared, the combine is empty.
    if (o != 2 && (nbx > 1 || nby > 1)) {
        dim3 blk(32, 8);
        k_oras_combine<<<grid2(w, h, blk, C), blk, 0, s>>>(u_in, zero_in, planes, w, h, B - o, o,
                                                           nbx, nby, u_out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------

cudaError_t launch_count_mask(const uint8_t* c, size_t n, unsigned long long* out,
                              cudaStream_t s) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_count_mask<<<(unsigned)blocks, 256, 0, s>>>(c, n, out);
    return cudaGetLastError();
}

cudaError_t launch_mask_down(const uint8_t* c, int w, int h, uint8_t* cH,
                             unsigned long long* unknownH, cudaStream_t s) {
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    dim3 blk(32, 8);
    k_mask_down<<<grid2(wH, hH, blk), blk, 0, s>>>(c, w, h, cH, wH, hH, unknownH);
    return cudaGetLastError();
}

cudaError_t launch_values_down(const uint8_t* c, const float* b, int w, int h, int C,
                               const uint8_t* cH, float* bH, int modified, cudaStream_t s) {
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    dim3 blk(32, 8);
    k_values_down<<<grid2(wH, hH, blk), blk, 0, s>>>(c, b, w, h, C, cH, bH, wH, hH, modified);
    return cudaGetLastError();
}

size_t residual_partials_per_channel(int w, int h) {
    return (size_t)((w + kResBX - 1) / kResBX) * (size_t)((h + kResBY - 1) / kResBY);
}

cudaError_t launch_residual(const float* u, int zero_u, const float* b, int rhs_zero,
                            const uint8_t* c, int w, int h, int C, float* r, double* partials,
                            int* nparts, cudaStream_t s) {
    dim3 blk(kResBX, kResBY);
    dim3 grid = grid2(w, h, blk, C);
    *nparts = (int)(grid.x * grid.y);
    k_residual<<<grid, blk, 0, s>>>(u, zero_u, b, rhs_zero, c, w, h, r, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, int nparts, int C, double* out,
                                   cudaStream_t s) {
    k_reduce<<<C, 256, 0, s>>>(partials, nparts, out);
    return cudaGetLastError();
}

cudaError_t launch_restrict(const float* u, const float* b, int rhs_zero, const uint8_t* c,
                            int w, int h, int C, const uint8_t* cH, float* rH, cudaStream_t s) {
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    dim3 blk(32, 8);
    k_restrict<<<grid2(wH, hH, blk, C), blk, 0, s>>>(u, b, rhs_zero, c, w, h, cH, rH, wH, hH);
    return cudaGetLastError();
}

cudaError_t launch_prolong(const float* uH, const float* b, const uint8_t* c, int w, int h,
                           int C, float* u, int mode, unsigned* maxupd, cudaStream_t s) {
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    dim3 blk(32, 8);
    dim3 grid = grid2(w, h, blk, C);
    // about 16 CTAs of 256 threads per SM in total; each walks rows with a stride
    const unsigned target = 152u * 16u;
    const unsigned per_row = grid.x * grid.z;
    unsigned gy = (target + per_row - 1) / per_row;
    if (gy < 1) gy = 1;
    if (gy < grid.y) grid.y = gy;
    k_prolong<<<grid, blk, 0, s>>>(uH, wH, hH, b, c, w, h, u, mode, mode == 1 ? maxupd : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_select(const float* b, const uint8_t* c, int w, int h, int C, float* u,
                          cudaStream_t s) {
    const size_t n = (size_t)w * h;
    size_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    k_select<<<dim3((unsigned)blocks, (unsigned)C), 256, 0, s>>>(b, c, n, u);
    return cudaGetLastError();
}

cudaError_t launch_oras(const float* u_in, int zero_in, const float* rhs, int rhs_zero,
                        const uint8_t* c, int w, int h, int C, int B, int o, float alpha,
                        int iters, float rtol2, float* u_out, float* planes, unsigned* maxupd,
                        cudaStream_t s) {
    switch (B) {
        case 32:
            return launch_oras_t<32, 8>(u_in, zero_in, rhs, rhs_zero, c, w, h, C, o, alpha, iters,
                                        rtol2, u_out, planes, maxupd, s);
        case 16:
            return launch_oras_t<16, 4>(u_in, zero_in, rhs, rhs_zero, c, w, h, C, o, alpha, iters,
                                        rtol2, u_out, planes, maxupd, s);
        case 8:
            return launch_oras_t<8, 2>(u_in, zero_in, rhs, rhs_zero, c, w, h, C, o, alpha, iters,
                                       rtol2, u_out, planes, maxupd, s);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace di

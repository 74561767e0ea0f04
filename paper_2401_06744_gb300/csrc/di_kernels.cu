// CUDA kernels (sm_103a) of the reduced-FMG ORAS inpainting decoder.
//
// Problem (Section 2.2, eq. 2.6): (C + (I - C) L) u = C f per channel, L the
// 5-point negated Laplacian with reflecting boundaries and unit spacing on
// every level (coarse right-hand sides carry the (H/h)^2 = 4 factor).
//
// Kernels:
//   k_pyramid_level  Section 4.3: one pyramid level in one pass (2x2 max pooling of
//                    the mask, modified or naive mask values, packed mask words,
//                    unknown count); k_mask_down, k_values_down and k_pack_mask
//                    are the separate steps (single-step entry points, the finest
//                    level's packing)
//   k_residual       r = b - A u with per-CTA partial sums of r^2 (Algorithm 2 step 1)
//   k_reduce         fixed-order sum of the partials (one global scalar product)
//   k_restrict       Algorithm 3 steps 2-3 fused: residual + 2x2 averaging (x4)
//   k_prolong        Section 4.4 bilinear prolongation, cascadic or correction mode
//                    (where the block kernel cannot form its start by prolongation)
//   k_select         u = c ? b : 0 (or c ? b : u for a given start)
//   k_oras_2w        Algorithm 2 steps 1-3 for 32x32 blocks: two warps per (block,
//                    channel), plain CG in registers as packed FP32 pairs, tiles by
//                    TMA; optionally the start formed by prolongation inside it
//   k_oras_2w_h      the same with FP16 / BF16 local iterates
//   k_oras_warp      8x8 and 16x16 blocks: one warp per (block, channel)
//   k_combine_rows/cols  Algorithm 2 step 3 for pixels shared by several
//                    blocks: sum the weighted block contributions in a fixed
//                    order (shared rows full width, then shared columns)
//   k_plan, k_stop   the device-driven decode: levels in use and start, and the
//                    stop test after every V-cycle (conditional graph nodes)
//   k_batch_*        the batched form: the same steps over the segment tables of
//                    every image of a batch
//   k_cg_*           the global CG smoother of the comparison methods (Section 5)
//
// Layout: images planar [C][h][w] float32, masks [h][w] uint8.  The ORAS
// block pass writes pixels that only one block weights (weight 1) straight to
// u_out and parks weighted contributions of shared pixels in four parity
// planes [4][C][h][w] (blocks with equal (kx & 1, ky & 1) never overlap, so
// every plane pixel has one writer); the combine pass adds them in a fixed
// order, which keeps the result deterministic without atomics.
#include "di_internal.h"
#include "../../include/di.h"

#include <cfloat>
#include <cstring>
#include <cmath>

#include <atomic>
#include <mutex>
#include <type_traits>

#include <cuda.h>  // CUtensorMap and its enums (the encoder comes from the runtime)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace di {

static std::atomic<long long> g_launches{0};
// the calling thread's own launches: captures count their kernels with it, so
// that decodes finishing on other threads meanwhile do not enter the count
static thread_local long long t_launches = 0;
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
long long thread_launch_count() { return t_launches; }
void add_launches(long long k) {
    g_launches.fetch_add(k, std::memory_order_relaxed);
    t_launches += k;
}

namespace {

constexpr unsigned kFull = 0xffffffffu;

inline void count(int k = 1) {
    g_launches.fetch_add(k, std::memory_order_relaxed);
    t_launches += k;
}

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

// Element access of an array stored as float, FP16 or BF16 (the narrow
// coarse-level storage); arithmetic is FP32 throughout.
template <class T> __device__ __forceinline__ float ldf(const T* p);
template <> __device__ __forceinline__ float ldf<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ldf<__half>(const __half* p) { return __half2float(*p); }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <class T> __device__ __forceinline__ void stf(T* p, float v);
template <> __device__ __forceinline__ void stf<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void stf<__half>(__half* p, float v) { *p = __float2half_rn(v); }
template <> __device__ __forceinline__ void stf<__nv_bfloat16>(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
}

// Block index k = min(g / s, nb - 1) without an integer division: a float
// estimate from the reciprocal, corrected by one step either way.
__device__ __forceinline__ int block_of(int g, int s, float inv_s, int nb) {
    int k = __float2int_rd(((float)g + 0.5f) * inv_s);
    if (k * s > g) --k;
    else if ((k + 1) * s <= g) ++k;
    return k > nb - 1 ? nb - 1 : k;
}

// Blocks with nonzero weight at global coordinate g along one axis: returns
// 1 (k0) or 2 (k0 < k1).
__device__ __forceinline__ int axis_contrib(int g, int s, int o, int nb, int& k0, int& k1,
                                            float inv_s) {
    const int k = block_of(g, s, inv_s, nb);
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

__device__ __forceinline__ void mask_down_body(const uint8_t* __restrict__ c, int w, int h,
                            uint8_t* __restrict__ cH, int wH, int hH, int bx, int by) {
    const int X = bx * blockDim.x + threadIdx.x;
    const int Y = by * blockDim.y + threadIdx.y;
    if (X >= wH || Y >= hH) return;
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
}

__global__ void k_mask_down(const uint8_t* __restrict__ c, int w, int h,
                            uint8_t* __restrict__ cH, int wH, int hH) {
    mask_down_body(c, w, h, cH, wH, hH, blockIdx.x, blockIdx.y);
}

// One coarse cell: weights of its (up to four) fine children.
__device__ __forceinline__ void values_down_body(const uint8_t* __restrict__ c, const float* __restrict__ b,
                              int w, int h, int C, const uint8_t* __restrict__ cH,
                              float* __restrict__ bH, int wH, int hH, int modified, int bx, int by) {
    const int X = bx * blockDim.x + threadIdx.x;
    const int Y = by * blockDim.y + threadIdx.y;
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
            if (wt[k] != 0.f) num = __fmaf_rn(wt[k], bc[idx[k]], num);
        bH[ch * nH + P] = num * inv;
    }
}

__global__ void k_values_down(const uint8_t* __restrict__ c, const float* __restrict__ b,
                              int w, int h, int C, const uint8_t* __restrict__ cH,
                              float* __restrict__ bH, int wH, int hH, int modified) {
    values_down_body(c, b, w, h, C, cH, bH, wH, hH, modified, blockIdx.x, blockIdx.y);
}

// One level of the pyramid in one pass (Section 4.3): thread (X, Y) forms the
// coarse mask cell cH = max over its children, the mask value bH (modified or
// naive downsampling, the same weights and sums as values_down_body), and the
// warp of 32 consecutive X packs the 32 mask bits of its row (known or beyond
// the image = 1) and counts the unknown ones; the CTAs of the last column
// write the padding word of their rows.  Each thread reads its four children's
// mask bytes once (as byte pairs where the image allows); the modified
// weights take the four neighbouring coarse cells' masks from a shared tile
// of the CTA's cells and their one-cell halo, so the level needs no second
// pass.  values = 0: masks only (a given start).  A CTA of 32 x 8 threads;
// (bx, by) its position, nbx the CTAs along x (one column per packed word of
// a coarse row but the padding word).
__device__ __forceinline__ void pyramid_level_body(
    const uint8_t* __restrict__ c, const float* __restrict__ b, int w, int h, int C,
    uint8_t* __restrict__ cH, float* __restrict__ bH, int wH, int hH, int modified, int values,
    uint32_t* __restrict__ bits, int wpr, unsigned long long* __restrict__ unknown, int bx,
    int by, int nbx) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int X = bx * 32 + tx;
    const int Y = by * 8 + ty;
    const int lane = tx;
    // children bytes of coarse cell (Xc, Yc), 0 where a child is off the image
    const bool pairs = (w & 1) == 0 && (reinterpret_cast<uintptr_t>(c) & 1) == 0;
    auto children = [&](int Xc, int Yc, uint32_t& c00, uint32_t& c01, uint32_t& c10,
                        uint32_t& c11) {
        const int x = 2 * Xc, y = 2 * Yc;
        const uint8_t* row = c + (size_t)y * w + x;
        const bool y1 = y + 1 < h;
        if (pairs) {
            const uchar2 r0 = *reinterpret_cast<const uchar2*>(row);
            const uchar2 r1 = y1 ? *reinterpret_cast<const uchar2*>(row + w) : make_uchar2(0, 0);
            c00 = r0.x; c01 = r0.y; c10 = r1.x; c11 = r1.y;
        } else {
            const bool x1 = x + 1 < w;
            c00 = row[0];
            c01 = x1 ? row[1] : 0u;
            c10 = y1 ? row[w] : 0u;
            c11 = (x1 && y1) ? row[w + 1] : 0u;
        }
    };
    auto known = [&](int Xc, int Yc) -> bool {
        if (Xc < 0 || Xc >= wH || Yc < 0 || Yc >= hH) return false;
        uint32_t a0, a1, a2, a3;
        children(Xc, Yc, a0, a1, a2, a3);
        return (a0 | a1 | a2 | a3) != 0u;
    };
    const bool inside = X < wH && Y < hH;
    uint32_t ck[4] = {0u, 0u, 0u, 0u};
    if (inside) children(X, Y, ck[0], ck[1], ck[2], ck[3]);
    const bool kn = (ck[0] | ck[1] | ck[2] | ck[3]) != 0u;
    // masks of the CTA's coarse cells and their direct neighbours
    __shared__ uint8_t s_kn[10][34];
    const bool nbrs = values && modified;  // uniform over the grid
    if (nbrs) {
        s_kn[ty + 1][tx + 1] = kn ? 1 : 0;
        if (ty == 0) s_kn[0][tx + 1] = known(X, Y - 1) ? 1 : 0;
        if (ty == 7) s_kn[9][tx + 1] = known(X, Y + 1) ? 1 : 0;
        if (tx == 0) s_kn[ty + 1][0] = known(X - 1, Y) ? 1 : 0;
        if (tx == 31) s_kn[ty + 1][33] = known(X + 1, Y) ? 1 : 0;
        __syncthreads();
    }
    if (inside) {
        const size_t nH = (size_t)wH * hH, P = (size_t)Y * wH + X;
        cH[P] = kn ? 1 : 0;
        if (values) {
            const size_t n = (size_t)w * h;
            if (!kn) {
                for (int ch = 0; ch < C; ++ch) bH[ch * nH + P] = 0.f;
            } else {
                const bool kl = nbrs && s_kn[ty + 1][tx], kr = nbrs && s_kn[ty + 1][tx + 2];
                const bool ku = nbrs && s_kn[ty][tx + 1], kd = nbrs && s_kn[ty + 2][tx + 1];
                float wt[4];
                float den = 0.f, cnt = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int x = 2 * X + (k & 1), y = 2 * Y + (k >> 1);
                    wt[k] = 0.f;
                    if (x >= w || y >= h || !ck[k]) continue;
                    cnt += 1.f;
                    if (!modified) { wt[k] = 1.f; continue; }
                    // partners inside the cell (0 off the image), then the
                    // neighbours across the cell's sides
                    int m = (ck[k ^ 1] != 0u) + (ck[k ^ 2] != 0u);
                    const int xo = (x & 1) ? x + 1 : x - 1;
                    const int yo = (y & 1) ? y + 1 : y - 1;
                    if (xo >= 0 && xo < w) m += (x & 1) ? kr : kl;
                    if (yo >= 0 && yo < h) m += (y & 1) ? kd : ku;
                    wt[k] = (float)(4 - m);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) den += wt[k];
                if (den == 0.f) {  // gap of the printed rule: the naive average
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int x = 2 * X + (k & 1), y = 2 * Y + (k >> 1);
                        wt[k] = (x < w && y < h && ck[k]) ? 1.f : 0.f;
                    }
                    den = cnt;
                }
                const float inv = 1.f / fmaxf(1.f, den);
                const size_t p0 = (size_t)(2 * Y) * w + 2 * X;
                for (int ch = 0; ch < C; ++ch) {
                    const float* bc = b + ch * n + p0;
                    float num = 0.f;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (wt[k] != 0.f)
                            num = __fmaf_rn(wt[k], bc[(k >> 1) * (size_t)w + (k & 1)], num);
                    bH[ch * nH + P] = num * inv;
                }
            }
        }
    }
    // the packed mask row of this warp: bit set = known or beyond the image
    const unsigned word = __ballot_sync(0xffffffffu, X >= wH || kn);
    unsigned unk = 0;
    if (Y < hH) {
        if (lane == 0) bits[(size_t)Y * wpr + bx] = word;
        unk = X < wH && !kn ? 1u : 0u;
        if (bx == nbx - 1 && lane == 0)
            bits[(size_t)Y * wpr + wpr - 1] = 0xffffffffu;  // the padding word
    }
    if (unknown) {
        __shared__ unsigned s_u[8];
        const unsigned c8 = __reduce_add_sync(0xffffffffu, unk);
        if (lane == 0) s_u[ty] = c8;
        __syncthreads();
        if (tx == 0 && ty == 0) {
            unsigned long long a = 0;
            for (int i = 0; i < 8; ++i) a += s_u[i];
            if (a) atomicAdd(unknown, a);
        }
    }
}

__global__ void __launch_bounds__(256)
k_pyramid_level(const uint8_t* __restrict__ c, const float* __restrict__ b, int w, int h, int C,
                uint8_t* __restrict__ cH, float* __restrict__ bH, int wH, int hH, int modified,
                int values, uint32_t* __restrict__ bits, int wpr,
                unsigned long long* __restrict__ unknown) {
    pyramid_level_body(c, b, w, h, C, cH, bH, wH, hH, modified, values, bits, wpr, unknown,
                       blockIdx.x, blockIdx.y, gridDim.x);
}

// ---------------------------------------------------------------------------
// Residual and its norm (Algorithm 2 step 1; Section 2.2 "single global scalar
// product")
// ---------------------------------------------------------------------------

template <bool F64 = false>
__device__ __forceinline__ float residual_at(const float* __restrict__ u, int zero_u,
                                             const float* __restrict__ b, int rhs_zero,
                                             const uint8_t* __restrict__ c, int w, int h,
                                             int x, int y) {
    typedef typename std::conditional<F64, double, float>::type R;
    const size_t p = (size_t)y * w + x;
    if (c[p]) return b[p] - (zero_u ? 0.f : u[p]);
    const R rhs = rhs_zero ? (R)0 : (R)b[p];
    if (zero_u) return (float)rhs;
    const R uc = u[p];
    R lu = 0;
    if (x > 0) lu += uc - (R)u[p - 1];
    if (x < w - 1) lu += uc - (R)u[p + 1];
    if (y > 0) lu += uc - (R)u[p - w];
    if (y < h - 1) lu += uc - (R)u[p + w];
    return (float)(rhs - lu);
}

constexpr int kResBX = 32, kResBY = 8;

template <bool F64>
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
        rv = residual_at<F64>(u + ch * n, zero_u, b + ch * n, rhs_zero, c, w, h, x, y);
        if (r) r[ch * n + (size_t)y * w + x] = rv;
    }
    // FP32 within the warp, FP64 across the warps and CTAs (fixed order)
    __shared__ double s_part[kResBX * kResBY / 32];
    const int t = threadIdx.y * kResBX + threadIdx.x;
    const float v = warp_sum(rv * rv);
    if ((t & 31) == 0) s_part[t >> 5] = (double)v;
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
// Global CG on one level, the comparison smoother of Section 5 (CG in place of
// ORAS, and single-level CG).  x is the correction of the iterate, r = b - A(u
// + x) is kept by recurrence; p and r vanish on known pixels.  Per channel
// the device keeps sc[ch * 4 + 0/1] = r.r of even/odd steps and sc[ch*4 + 2] =
// p.Ap, so a step needs no host round trip.
//
// The kernels stride over 32x8 pixel tiles with a fixed number of CTAs per
// channel (kCgCtas in total), so a dot product leaves one partial per CTA.
// Products are summed in FP32 within a thread and a warp and in FP64 across
// the warps and CTAs, all in a fixed order: GB300 issues FP64 at a small
// fraction of its FP32 rate, and per-element FP64 arithmetic would dominate
// these memory-bound passes.
// ---------------------------------------------------------------------------

constexpr int kCgBX = 32, kCgBY = 8, kCgCtas = 152 * 8;

// Sum of one float per thread of a 256-thread CTA, written to
// partials[ch * nparts + blockIdx.x]: FP32 within each warp, FP64 across the
// eight warps in warp order.
__device__ __forceinline__ void block_partial(float v, double* __restrict__ partials, int ch,
                                              int nparts) {
    __shared__ double s_p[kCgBX * kCgBY / 32];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    v = warp_sum(v);
    if ((t & 31) == 0) s_p[t >> 5] = (double)v;
    __syncthreads();
    if (t == 0) {
        double a = 0.0;
        for (int i = 0; i < kCgBX * kCgBY / 32; ++i) a += s_p[i];
        partials[(size_t)ch * nparts + blockIdx.x] = a;
    }
}

struct CgTiles {
    int w, h, tiles_x, ntiles;
    __device__ __forceinline__ void pixel(int t, int* X, int* Y) const {
        const int ty = t / tiles_x;
        *X = (t - ty * tiles_x) * kCgBX + threadIdx.x;
        *Y = ty * kCgBY + threadIdx.y;
    }
};

__global__ void __launch_bounds__(kCgBX * kCgBY)
k_cg_init(CgTiles g, const float* __restrict__ u, int zero_u, const float* __restrict__ b,
          int rhs_zero, const uint8_t* __restrict__ c, float* __restrict__ r,
          float* __restrict__ p, float* __restrict__ x, double* __restrict__ partials) {
    const int ch = blockIdx.y;
    const size_t n = (size_t)g.w * g.h;
    float acc = 0.f;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int X, Y;
        g.pixel(t, &X, &Y);
        if (X >= g.w || Y >= g.h) continue;
        const size_t pix = (size_t)Y * g.w + X, i = ch * n + pix;
        float rv = 0.f;
        if (!c[pix])
            rv = residual_at(u + ch * n, zero_u, b + ch * n, rhs_zero, c, g.w, g.h, X, Y);
        r[i] = rv;
        p[i] = rv;
        x[i] = 0.f;
        acc = fmaf(rv, rv, acc);
    }
    block_partial(acc, partials, ch, gridDim.x);
}

__global__ void __launch_bounds__(kCgBX * kCgBY)
k_cg_matvec(CgTiles g, const float* __restrict__ p, const uint8_t* __restrict__ c,
            float* __restrict__ q, double* __restrict__ partials) {
    const int ch = blockIdx.y;
    const int w = g.w, h = g.h;
    const size_t n = (size_t)w * h;
    const float* pc = p + ch * n;
    float acc = 0.f;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int X, Y;
        g.pixel(t, &X, &Y);
        if (X >= w || Y >= h) continue;
        const size_t pix = (size_t)Y * w + X;
        float qv = 0.f;
        if (!c[pix]) {
            const float pv = pc[pix];
            float sn = 0.f;
            int deg = 0;
            if (X > 0) { ++deg; sn += pc[pix - 1]; }
            if (X < w - 1) { ++deg; sn += pc[pix + 1]; }
            if (Y > 0) { ++deg; sn += pc[pix - w]; }
            if (Y < h - 1) { ++deg; sn += pc[pix + w]; }
            qv = (float)deg * pv - sn;  // known neighbours have p = 0
            acc = fmaf(pv, qv, acc);
        }
        q[ch * n + pix] = qv;
    }
    block_partial(acc, partials, ch, gridDim.x);
}

__global__ void __launch_bounds__(kCgBX * kCgBY)
k_cg_update(CgTiles g, const float* __restrict__ p, const float* __restrict__ q,
            float* __restrict__ x, float* __restrict__ r, const double* __restrict__ sc, int par,
            double* __restrict__ partials) {
    const int ch = blockIdx.y;
    const size_t n = (size_t)g.w * g.h;
    const double rr = sc[ch * 4 + par], pq = sc[ch * 4 + 2];
    const float a = pq > 0.0 ? (float)(rr / pq) : 0.f;
    float acc = 0.f;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int X, Y;
        g.pixel(t, &X, &Y);
        if (X >= g.w || Y >= g.h) continue;
        const size_t i = ch * n + (size_t)Y * g.w + X;
        x[i] = fmaf(a, p[i], x[i]);
        const float rv = fmaf(-a, q[i], r[i]);
        r[i] = rv;
        acc = fmaf(rv, rv, acc);
    }
    block_partial(acc, partials, ch, gridDim.x);
}

__global__ void k_cg_direction(float* __restrict__ p, const float* __restrict__ r, size_t n,
                               const double* __restrict__ sc, int par) {
    const int ch = blockIdx.y;
    const double rr_old = sc[ch * 4 + par], rr_new = sc[ch * 4 + (par ^ 1)];
    const float beta = rr_old > 0.0 ? (float)(rr_new / rr_old) : 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[ch * n + i] = fmaf(beta, p[ch * n + i], r[ch * n + i]);
}

// out = in + x (in may be zero); the largest |x| goes into *maxupd (nullable)
__global__ void k_cg_finish(const float* __restrict__ in, int zero_in,
                            const float* __restrict__ x, float* __restrict__ out, size_t n,
                            unsigned* __restrict__ maxupd) {
    const int ch = blockIdx.y;
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float xv = x[ch * n + i];
        out[ch * n + i] = (zero_in ? 0.f : in[ch * n + i]) + xv;
        m = fmaxf(m, fabsf(xv));
    }
    if (maxupd) {
        m = warp_max(m);
        if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(maxupd, __float_as_uint(m));
    }
}

__global__ void __launch_bounds__(256)
k_reduce_slot(const double* __restrict__ partials, int nparts, double* __restrict__ sc, int slot) {
    const int ch = blockIdx.x;
    const double* pp = partials + (size_t)ch * nparts;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += pp[i];
    __shared__ double s_w[8];
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_w[i];
        sc[ch * 4 + slot] = t;
    }
}

// ---------------------------------------------------------------------------
// Grid transfers (Algorithm 3, Section 4.4)
// ---------------------------------------------------------------------------

// One thread per coarse cell.  A coarse cell off the coarse mask has four
// unknown children (max pooling), so their residuals need no mask loads: the
// 4x4 patch of u around the children is read at once (zero outside the image)
// and the in-image neighbour count gives the reflecting boundary.  u is stored
// as TU, the right-hand side b as TB, rH as TO (FP16/BF16 on the coarse levels
// in the 16-bit precision modes).  F64: the children's residuals are formed
// and summed in FP64 (the finest-grid refinement residual) and rounded once.
template <bool VEC, class TU, class TB, class TO, bool F64>
__device__ __forceinline__ void restrict_body(const TU* __restrict__ u, const TB* __restrict__ b, int rhs_zero,
           int w, int h, const uint8_t* __restrict__ cH, TO* __restrict__ rH, int wH,
           int hH, int bx, int by, int bz) {
    typedef typename std::conditional<F64, double, float>::type R;
    const int X = bx * blockDim.x + threadIdx.x;
    const int Y = by * blockDim.y + threadIdx.y;
    const int ch = bz;
    if (X >= wH || Y >= hH) return;
    const size_t n = (size_t)w * h, nH = (size_t)wH * hH, P = (size_t)Y * wH + X;
    if (cH[P]) { stf(rH + ch * nH + P, 0.f); return; }
    const TU* uc = u + ch * n;
    const int x0 = 2 * X - 1, y0 = 2 * Y - 1;
    if (VEC && X >= 1 && Y >= 1 && 2 * X + 2 < w && 2 * Y + 2 < h) {
        // a cell whose 4x4 patch lies inside the image (all but the border
        // cells): every child has four neighbours and the count is 4, so the
        // same sums as below without a bounds test (the same bits)
        const TU* r0 = uc + (size_t)y0 * w + x0;
        float t[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 mid = *reinterpret_cast<const float2*>(r0 + (size_t)j * w + 1);
            t[j][1] = mid.x;
            t[j][2] = mid.y;
            t[j][0] = (j == 1 || j == 2) ? ldf(r0 + (size_t)j * w) : 0.f;
            t[j][3] = (j == 1 || j == 2) ? ldf(r0 + (size_t)j * w + 3) : 0.f;
        }
        R sum = 0;
#pragma unroll
        for (int j = 1; j <= 2; ++j) {
            float2 rb = make_float2(0.f, 0.f);
            if (!rhs_zero)
                rb = *reinterpret_cast<const float2*>(b + ch * n + (size_t)(y0 + j) * w + x0 + 1);
#pragma unroll
            for (int i = 1; i <= 2; ++i) {
                const R lu = (R)4 * (R)t[j][i] -
                             ((R)t[j][i - 1] + (R)t[j][i + 1] + (R)t[j - 1][i] + (R)t[j + 1][i]);
                const R rhs = rhs_zero ? (R)0 : (R)(i == 1 ? rb.x : rb.y);
                sum += rhs - lu;
            }
        }
        stf(rH + ch * nH + P, (float)sum);
        return;
    }
    float t[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = y0 + j;
        const bool yok = y >= 0 && y < h;
        if (VEC) {
            // the two children's columns as one 8-byte word, the outer
            // columns (rows 1 and 2 only) as single words
            float2 mid = make_float2(0.f, 0.f);
            if (yok) mid = *reinterpret_cast<const float2*>(uc + (size_t)y * w + x0 + 1);
            t[j][1] = mid.x;
            t[j][2] = mid.y;
            const bool inner = j == 1 || j == 2;
            t[j][0] = (inner && yok && x0 >= 0) ? ldf(uc + (size_t)y * w + x0) : 0.f;
            t[j][3] = (inner && yok && x0 + 3 < w) ? ldf(uc + (size_t)y * w + x0 + 3) : 0.f;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int x = x0 + i;
                const bool corner = (i == 0 || i == 3) && (j == 0 || j == 3);
                t[j][i] = (!corner && yok && x >= 0 && x < w) ? ldf(uc + (size_t)y * w + x) : 0.f;
            }
        }
    }
    R sum = 0;
    int cnt = 0;
#pragma unroll
    for (int j = 1; j <= 2; ++j) {
        float2 rb = make_float2(0.f, 0.f);
        if (VEC && !rhs_zero && y0 + j < h)
            rb = *reinterpret_cast<const float2*>(b + ch * n + (size_t)(y0 + j) * w + x0 + 1);
#pragma unroll
        for (int i = 1; i <= 2; ++i) {
            const int x = x0 + i, y = y0 + j;
            if (x >= w || y >= h) continue;
            const int deg = (x > 0) + (x < w - 1) + (y > 0) + (y < h - 1);
            const R lu = (R)deg * (R)t[j][i] -
                         ((R)t[j][i - 1] + (R)t[j][i + 1] + (R)t[j - 1][i] + (R)t[j + 1][i]);
            const R rhs = rhs_zero ? (R)0
                          : VEC ? (R)(i == 1 ? rb.x : rb.y)
                                : (R)ldf(b + ch * n + (size_t)y * w + x);
            sum += rhs - lu;
            ++cnt;
        }
    }
    // 4 sum / cnt with cnt in {1, 2, 4} (children inside the image): an exact
    // power-of-two scaling, so a multiplication gives the quotient bit for bit
    stf(rH + ch * nH + P, (float)(sum * (R)(4 >> (cnt >> 1))));
}

template <bool VEC, class TU, class TB, class TO, bool F64>
__global__ void __launch_bounds__(256)
k_restrict(const TU* __restrict__ u, const TB* __restrict__ b, int rhs_zero,
           int w, int h, const uint8_t* __restrict__ cH, TO* __restrict__ rH, int wH,
           int hH) {
    restrict_body<VEC, TU, TB, TO, F64>(u, b, rhs_zero, w, h, cH, rH, wH, hH, blockIdx.x, blockIdx.y,
                                        blockIdx.z);
}

// Cell-centred bilinear prolongation.  A fine pixel takes 9/16 of its parent
// coarse cell, 3/16 of each of the two edge neighbours of the parent on the
// child's side and 1/16 of the diagonal one (coarse indices clamped at the
// border).  One thread per coarse cell (X, Y) and its up to 2x2 children:
// for the child row y = 2Y + dy the row blend takes coarse row Y three times
// and its neighbour on the child's side (Y - 1 for dy = 0, Y + 1 for dy = 1)
// once, the column blend the same with X - 1 (left child) or X + 1.
// mode 0: u = c ? b : P uH;  mode 1: u += c ? 0 : P uH (largest |P uH| over
// the updated pixels into *maxupd).  VEC: each child pair is one 8-byte word
// of u and b and one 2-byte word of c (w even, aligned base pointers; FP32 u).
// uH is stored as TC and u as TF (FP16/BF16 on the coarse levels in the
// 16-bit precision modes); b is FP32.
// The bilinear weights of one fine pixel: cc its parent coarse cell, cn the
// parent's vertical neighbour on the child's side, cs the horizontal one and
// csn the diagonal one; (3 (3 cc + cn) + (3 cs + csn)) / 16 with every
// rounding explicit, so that each kernel that prolongs gets the same bits.
__device__ __forceinline__ float prolong_blend(float cc, float cn, float cs, float csn) {
    const float vc = __fmaf_rn(3.f, cc, cn);
    const float vs = __fmaf_rn(3.f, cs, csn);
    return __fmul_rn(__fmaf_rn(3.f, vc, vs), 0.0625f);
}

template <bool VEC, class TC, class TF>
__device__ __forceinline__ void prolong_body(const TC* __restrict__ uH, int wH, int hH, const float* __restrict__ b,
          const uint8_t* __restrict__ c, int w, int h, TF* __restrict__ u, int mode,
          unsigned* __restrict__ maxupd, int bx, int by, int bz) {
    const int X = bx * blockDim.x + threadIdx.x;
    const int Y = by * blockDim.y + threadIdx.y;
    const int ch = bz;
    float amax = 0.f;
    if (X < wH && Y < hH) {
        const size_t n = (size_t)w * h, nH = (size_t)wH * hH;
        const TC* e = uH + ch * nH;
        const int Xl = max(X - 1, 0), Xr = min(X + 1, wH - 1);
        const TC* rc = e + (size_t)Y * wH;
        const TC* ru = e + (size_t)max(Y - 1, 0) * wH;
        const TC* rd = e + (size_t)min(Y + 1, hH - 1) * wH;
        const float cl = ldf(rc + Xl), cc = ldf(rc + X), cr = ldf(rc + Xr);
        const float ul = ldf(ru + Xl), uc = ldf(ru + X), ur = ldf(ru + Xr);
        const float dl = ldf(rd + Xl), dc = ldf(rd + X), dr = ldf(rd + Xr);
        const int x = 2 * X;
        TF* ucn = u + ch * n;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int y = 2 * Y + dy;
            if (y >= h) break;
            const float a0 = prolong_blend(cc, dy ? dc : uc, cl, dy ? dl : ul);
            const float a1 = prolong_blend(cc, dy ? dc : uc, cr, dy ? dr : ur);
            const size_t p = (size_t)y * w + x;
            if (VEC) {
                const uchar2 cm = *reinterpret_cast<const uchar2*>(c + p);
                float2* up = reinterpret_cast<float2*>(ucn + p);
                if (mode == 0) {
                    float2 bv = make_float2(0.f, 0.f);
                    if (cm.x | cm.y) bv = *reinterpret_cast<const float2*>(b + ch * n + p);
                    *up = make_float2(cm.x ? bv.x : a0, cm.y ? bv.y : a1);
                } else {
                    float2 uv = *up;
                    if (!cm.x) { uv.x = __fadd_rn(uv.x, a0); amax = fmaxf(amax, fabsf(a0)); }
                    if (!cm.y) { uv.y = __fadd_rn(uv.y, a1); amax = fmaxf(amax, fabsf(a1)); }
                    *up = uv;
                }
            } else {
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    if (x + dx >= w) break;
                    const float v = dx ? a1 : a0;
                    if (c[p + dx]) {
                        if (mode == 0) stf(ucn + p + dx, b[ch * n + p + dx]);
                    } else if (mode == 0) {
                        stf(ucn + p + dx, v);
                    } else {
                        stf(ucn + p + dx, __fadd_rn(ldf(ucn + p + dx), v));
                        amax = fmaxf(amax, fabsf(v));
                    }
                }
            }
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
            // most CTAs see a maximum already at least as large: skip their atomic
            if (m > __uint_as_float(*(volatile unsigned*)maxupd))
                atomicMax(maxupd, __float_as_uint(m));
        }
    }
}

template <bool VEC, class TC, class TF>
__global__ void __launch_bounds__(256)
k_prolong(const TC* __restrict__ uH, int wH, int hH, const float* __restrict__ b,
          const uint8_t* __restrict__ c, int w, int h, TF* __restrict__ u, int mode,
          unsigned* __restrict__ maxupd) {
    prolong_body<VEC, TC, TF>(uH, wH, hH, b, c, w, h, u, mode, maxupd, blockIdx.x, blockIdx.y,
                              blockIdx.z);
}

// keep == 0: u = c ? b : 0;  keep == 1: u = c ? b : u (a given iterate).
// u is stored as TU.
template <class TU>
__device__ __forceinline__ void select_body(const float* __restrict__ b, const uint8_t* __restrict__ c, size_t n,
                         TU* __restrict__ u, int keep, int bx, int nbx, int ch_) {
    const int ch = ch_;
    for (size_t i = (size_t)bx * blockDim.x + threadIdx.x; i < n;
         i += (size_t)nbx * blockDim.x) {
        if (c[i]) stf(u + ch * n + i, b[ch * n + i]);
        else if (!keep) stf(u + ch * n + i, 0.f);
    }
}

template <class TU>
__global__ void k_select(const float* __restrict__ b, const uint8_t* __restrict__ c, size_t n,
                         TU* __restrict__ u, int keep) {
    select_body<TU>(b, c, n, u, keep, blockIdx.x, gridDim.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// ORAS (Algorithm 2)
// ---------------------------------------------------------------------------

// ---- packed FP32 pairs (Blackwell f32x2 arithmetic) -------------------------
// A pair holds two horizontally adjacent pixels of one row (lo = even column).
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float lo2(f2 a) { return __uint_as_float((unsigned)(a & 0xffffffffull)); }
__device__ __forceinline__ float hi2(f2 a) { return __uint_as_float((unsigned)(a >> 32)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// r = b - ((deg) u_c - (up + down + left + right)) at one pixel; F64: in FP64
// (the finest-grid refinement residual), rounded once to FP32.
template <bool F64>
__device__ __forceinline__ float res_stencil(float b, float deg, float c, float up, float dn,
                                             float l, float r) {
    if (F64)
        return (float)((double)b - ((double)deg * (double)c -
                                    ((double)up + (double)dn + (double)l + (double)r)));
    return b - (deg * c - (up + dn + l + r));
}

// Partition-of-unity weight of block k (of nb along an axis, stride s,
// overlap o) at local coordinate l (Section 3.1): 0 at the block's outermost
// overlap pixel, 1 at its innermost one, linear in between (1/2 for o = 1).
// The ramp end points are exact so that "weight == 1" and "weight == 0"
// agree with the integer classification of the combine pass.
__device__ __forceinline__ float ramp_weight(int l, int k, int nb, int s, int o, float inv_o1) {
    float wgt = 1.f;
    if (k > 0 && l < o)
        wgt *= (o == 1) ? 0.5f : (l == o - 1 ? 1.f : (float)l * inv_o1);
    if (k < nb - 1 && l >= s) {
        const int jj = l - s;
        wgt *= (o == 1) ? 0.5f : (jj == 0 ? 1.f : (jj == o - 1 ? 0.f : 1.f - (float)jj * inv_o1));
    }
    return wgt;
}

// Pixels shared by two blocks along one axis are the open interior of each
// overlap: local offsets 1 .. o-2 after the seam (o >= 3), or the single
// overlap pixel when o = 1.  nsh is their count per seam.
__host__ __device__ __forceinline__ int shared_per_seam(int o) { return o == 1 ? 1 : (o > 2 ? o - 2 : 0); }
__host__ __device__ __forceinline__ int shared_first(int o) { return o == 1 ? 0 : 1; }

// ---- asynchronous global -> shared copies (4-byte, zero fill) ----------------
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    const int nbytes = ok ? 4 : 0;  // 0: nothing is read, the word is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(src), "r"(nbytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Bit-packed mask: row y, word k covers columns [32k, 32k + 32); bit set =
// known pixel or a column beyond the image.  wpr = words per row, including
// one padding word so that two consecutive words can always be read.  One
// warp per word (lane = column), four words in flight per warp, persistent
// warps; *unknown (nullable) gains the number of unknown pixels, with one
// atomic per CTA.
__device__ __forceinline__ void pack_mask_body(const uint8_t* __restrict__ c, int w, int h, uint32_t* __restrict__ bits, int wpr,
            unsigned long long* __restrict__ unknown, int bx, int nbx) {
    const int lane = threadIdx.x & 31;
    const int total = h * wpr;
    const int nwarps = (int)nbx * (int)(blockDim.x >> 5);
    unsigned unk = 0;
    for (int wid = (int)bx * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
         wid < total; wid += 4 * nwarps) {
        bool known[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int wk = wid + k * nwarps;
            known[k] = true;
            if (wk < total) {
                const int y = wk / wpr;
                const int x = 32 * (wk - y * wpr) + lane;
                known[k] = x >= w || c[(size_t)y * w + x] != 0;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int wk = wid + k * nwarps;
            const unsigned word = __ballot_sync(kFull, known[k]);
            if (wk < total) {  // warp-uniform
                if (lane == 0) bits[wk] = word;
                unk += (unsigned)__popc(~word);
            }
        }
    }
    if (unknown) {
        __shared__ unsigned s_u[8];
        if (lane == 0) s_u[threadIdx.x >> 5] = unk;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += s_u[i];
            if (a) atomicAdd(unknown, a);
        }
    }
}

__global__ void __launch_bounds__(256)
k_pack_mask(const uint8_t* __restrict__ c, int w, int h, uint32_t* __restrict__ bits, int wpr,
            unsigned long long* __restrict__ unknown) {
    pack_mask_body(c, w, h, bits, wpr, unknown, blockIdx.x, gridDim.x);
}

// One ORAS iteration, one warp per (block, channel) task.
//
// Lane layout: lane = (g, col), col = lane % B the block column and g the row
// group of R = B*B/32 rows; every CG vector is kept in registers as NP = R/2
// packed pairs, pair k = (row gR + k, row gR + k + NP) of the lane's column.
// Vertical neighbours of a pair are the neighbouring pairs (the first and the
// last pair swap one half with the other end of the column, and with the
// neighbouring row group through a shuffle); horizontal neighbours are the
// same pair of the neighbouring lanes (one 64-bit shuffle each way), with the
// block's outer columns cut by a 0/1 factor.  No shared memory and no barrier
// inside the CG loop.  Warps are persistent over a contiguous range of tasks
// (channel fastest, so the channels of one block are consecutive and share
// its mask bits and local operator); the next task's halo tile is fetched with
// cp.async while the current one is solved.
//
// Local problem (Section 3, Algorithm 2 step 2): plain CG on A_i v = R_i r
// from v = 0, A_i the rows of A for the block's unknown pixels with couplings
// to in-block neighbours only and alpha added to the diagonal for every
// in-image neighbour across the block edge (Robin), image edges reflecting.
// Vectors vanish on known pixels and outside the image, so the stencil reads
// neighbours unconditionally and only its result is masked.
template <int B>
struct WarpTile {
    static constexpr int G = 32 / B;       // row groups
    static constexpr int R = B / G;        // rows per lane
    static constexpr int NP = R / 2;       // packed pairs per lane
    static constexpr int TH = B + 2;       // tile side with the one-pixel halo
    static constexpr int P = B == 8 ? 12 : B + 2;  // tile pitch: row groups hit distinct banks
    static constexpr int TILE = TH * P;
    // per-warp shared memory (floats): two halo tiles, the 0/1 keep factors of
    // every pair (NP x 32 lanes x 2), the row weights (B), then optionally
    // two right-hand-side tiles (2 x B x B)
    static constexpr int KEEP = NP * 32 * 2;
    static constexpr int FIXED = 2 * TILE + KEEP + B;
};

template <int B>
__global__ void __launch_bounds__(32)
k_oras_warp(const float* __restrict__ u_in, int zero_in, const float* __restrict__ rhs,
            int rhs_zero, const uint32_t* __restrict__ mbits, int wpr, int w, int h, int C,
            int o, int nbx, int nby, float alpha, int iters, float rtol2,
            float* __restrict__ u_out, float* __restrict__ planes, unsigned* __restrict__ maxupd,
            int chan_inner, unsigned long long* __restrict__ step_count) {
    using WT = WarpTile<B>;
    constexpr int G = WT::G, R = WT::R, NP = WT::NP, TH = WT::TH, P = WT::P, TILE = WT::TILE;
    static_assert(G * B == 32 && R * G == B && NP * 2 == R, "warp shape");

    extern __shared__ float smem[];
    float* const s_u = smem;                                 // [2][TH][P]
    f2* const s_keep = reinterpret_cast<f2*>(smem + 2 * TILE);  // [NP][32] keep factors
    float* const s_wy = smem + 2 * TILE + WT::KEEP;          // [B] row weights of the block
    float* const s_b = smem + WT::FIXED;                     // [2][B][B], only when rhs_zero == 0

    const int lane = threadIdx.x;
    const int col = lane % B, g = lane / B;
    const int s = B - o;
    const size_t n = (size_t)w * h;
    const float inv_o1 = o > 1 ? 1.f / (float)(o - 1) : 0.f;

    // Task sequence of this warp.  chan_inner: blocks blockIdx.x, +gridDim.x,
    // ... each with all channels back to back (warps running together cover a
    // contiguous band of blocks, so halo re-reads hit L2, and a block's mask
    // bits and operator serve all its channels); otherwise (fewer blocks than
    // warps) tasks blockIdx.x, +gridDim.x, ... of the (block, channel) list.
    const int nblk = nbx * nby;
    auto task_of = [&](int i, int& blk, int& ch) {
        if (chan_inner) {
            blk = (int)blockIdx.x + (i / C) * (int)gridDim.x;
            ch = i % C;
        } else {
            const int t = (int)blockIdx.x + i * (int)gridDim.x;
            blk = t / C;
            ch = t - blk * C;
        }
        return blk < nblk;
    };

    // Issue the copies of task t into buffer `bs` (and the mask words of its
    // block into nlo/nhi when the block differs from `have_blk`).
    uint32_t nlo = 0xffffffffu, nhi = 0xffffffffu;
    auto prefetch = [&](int blk, int ch, int bs, int have_blk) {
        const int px0 = (blk % nbx) * s, py0 = (blk / nbx) * s;
        if (!zero_in) {
            // lane l copies tile column l of every row (and column 32 + l for
            // l < TH - 32); addresses advance by one image row per tile row
            const float* src = u_in + ch * n;
            float* dst = s_u + bs * TILE;
            const int gxa = px0 - 1 + lane, gxb = gxa + 32;
            const bool oka = lane < TH && gxa >= 0 && gxa < w;
            const bool okb = lane + 32 < TH && gxb < w;
            const float* row = src + (ptrdiff_t)(py0 - 1) * w;
#pragma unroll 2
            for (int ty = 0; ty < TH; ++ty, row += w) {
                const int gy = py0 - 1 + ty;
                const bool rok = gy >= 0 && gy < h;
                if (lane < TH) cp_async4(dst + ty * P + lane, (rok && oka) ? row + gxa : src, rok && oka);
                if (lane + 32 < TH) cp_async4(dst + ty * P + lane + 32, (rok && okb) ? row + gxb : src,
                                              rok && okb);
            }
        }
        if (!rhs_zero) {
            const float* src = rhs + ch * n;
            float* dst = s_b + bs * B * B;
#pragma unroll 4
            for (int e = lane; e < B * B; e += 32) {
                const int ly = e / B, lx = e - ly * B;
                const int gy = py0 + ly, gx = px0 + lx;
                const bool ok = gx < w && gy < h;
                cp_async4(dst + e, ok ? src + (size_t)gy * w + gx : src, ok);
            }
        }
        cp_async_commit();
        if (blk != have_blk && lane < B) {
            const int gy = py0 + lane;
            if (gy < h) {
                const uint32_t* row = mbits + (size_t)gy * wpr + (px0 >> 5);
                nlo = __ldg(row);
                nhi = __ldg(row + 1);
            } else {
                nlo = nhi = 0xffffffffu;
            }
        }
    };

    int blk, ch;
    if (!task_of(0, blk, ch)) return;  // warp-uniform
    prefetch(blk, ch, 0, -1);
    int buf = 0, cur_blk = -1;
    // per-block state
    uint32_t mb = 0;   // bit k: row gR + k of this lane's column is known or outside
    f2 ndg[NP];        // -(diagonal of A_i) per pair
    f2 ml2 = 0ull, mr2 = 0ull;  // 0/1: the left / right neighbour column is in the block
    float wx = 0.f, dh = 0.f;
    int x0 = 0, y0 = 0, bh = 0, kx = 0, ky = 0;
    float vmax = 0.f;
    unsigned nsteps = 0;  // completed local CG steps of this thread's tasks

    for (int i = 0;; ++i) {
        cp_async_wait_all();
        __syncwarp();
        const uint32_t mlo = nlo, mhi = nhi;
        int nblk_, nch;
        const bool more = task_of(i + 1, nblk_, nch);
        if (more) prefetch(nblk_, nch, buf ^ 1, blk);

        if (blk != cur_blk) {
            cur_blk = blk;
            kx = blk % nbx;
            ky = blk / nbx;
            x0 = kx * s;
            y0 = ky * s;
            const int bw = min(B, w - x0);
            bh = min(B, h - y0);
            // lane l < B holds the mask bits of block row l, columns x0 .. x0+31
            const uint32_t rowm = __funnelshift_r(mlo, mhi, x0 & 31);
            mb = 0;
#pragma unroll
            for (int rr = 0; rr < B; ++rr) {
                const uint32_t v = __shfl_sync(kFull, rowm, rr);
                const int k = rr - g * R;
                if (k >= 0 && k < R) mb |= ((v >> col) & 1u) << k;
            }
            const int gx = x0 + col;
            const float hc = (col > 0 ? 1.f : (gx > 0 ? alpha : 0.f)) +
                             (col + 1 < bw ? 1.f : (gx < w - 1 ? alpha : 0.f));
            dh = (float)((gx > 0) + (gx < w - 1));
            const float ml = col > 0 ? 1.f : 0.f, mr = col < B - 1 ? 1.f : 0.f;
            ml2 = pk(ml, ml);
            mr2 = pk(mr, mr);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                float vc[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ly = g * R + k + e * NP, gy = y0 + ly;
                    vc[e] = (ly > 0 ? 1.f : (gy > 0 ? alpha : 0.f)) +
                            (ly + 1 < bh ? 1.f : (gy < h - 1 ? alpha : 0.f));
                }
                ndg[k] = pk(-(hc + vc[0]), -(hc + vc[1]));
            }
            wx = ramp_weight(col, kx, nbx, s, o, inv_o1);
#pragma unroll
            for (int k = 0; k < NP; ++k)
                s_keep[k * 32 + lane] = pk(((mb >> k) & 1u) ? 0.f : 1.f,
                                          ((mb >> (k + NP)) & 1u) ? 0.f : 1.f);
            if (lane < B) s_wy[lane] = ramp_weight(lane, ky, nby, s, o, inv_o1);
            __syncwarp();
        }

        const float* tu = s_u + buf * TILE;
        const float* tb = s_b + buf * B * B;

        // initial residual r = R_i (b - A u), zero on known pixels
        f2 x[NP], r[NP], p[NP], q[NP];
        f2 acc0 = 0ull, acc1 = 0ull;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float rv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int ly = g * R + k + e * NP, gy = y0 + ly;
                float v = rhs_zero ? 0.f : tb[ly * B + col];
                if (!zero_in) {
                    const float* c0 = tu + (ly + 1) * P + col + 1;
                    const float dv = (float)((gy > 0) + (gy < h - 1));
                    v -= (dh + dv) * c0[0] - (c0[-P] + c0[P] + c0[-1] + c0[1]);
                }
                rv[e] = v;
            }
            r[k] = mul2(pk(rv[0], rv[1]), s_keep[k * 32 + lane]);
            p[k] = r[k];
            x[k] = 0ull;
            if (k & 1) acc1 = fma2(r[k], r[k], acc1);
            else acc0 = fma2(r[k], r[k], acc0);
        }
        acc0 = add2(acc0, acc1);
        float rr = warp_sum(lo2(acc0) + hi2(acc0));
        // rtol2 >= 0: relative stop (r.r <= max(rtol2, 1e-14) (r.r)_0); rtol2 < 0:
        // also stop once r.r <= -rtol2 (an absolute level, or the FP32 floor)
        const float rr_stop = rtol2 >= 0.f ? fmaxf(rtol2, 1e-14f) * rr
                                           : fmaxf(1e-14f * rr, -rtol2);

        for (int it = 0; it < iters; ++it) {
            if (!(rr > rr_stop)) break;  // rr is warp-uniform
            // the rows just above / below this lane's row group
            const float gu = __shfl_up_sync(kFull, hi2(p[NP - 1]), B);
            const float gd = __shfl_down_sync(kFull, lo2(p[0]), B);
            const f2 pu = pk(g > 0 ? gu : 0.f, lo2(p[NP - 1]));
            const f2 pd = pk(hi2(p[0]), g < G - 1 ? gd : 0.f);
            acc0 = 0ull;
            acc1 = 0ull;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const f2 left = __shfl_up_sync(kFull, p[k], 1, B);
                const f2 right = __shfl_down_sync(kFull, p[k], 1, B);
                const f2 up = k > 0 ? p[k - 1] : pu;
                const f2 dn = k < NP - 1 ? p[k + 1] : pd;
                f2 nbs = add2(up, dn);
                nbs = fma2(ml2, left, nbs);
                nbs = fma2(mr2, right, nbs);
                // -(A_i p), zero on known pixels
                const f2 qk = mul2(fma2(ndg[k], p[k], nbs), s_keep[k * 32 + lane]);
                q[k] = qk;
                if (k & 1) acc1 = fma2(p[k], qk, acc1);
                else acc0 = fma2(p[k], qk, acc0);
            }
            acc0 = add2(acc0, acc1);
            const float pq = -warp_sum(lo2(acc0) + hi2(acc0));
            if (!(pq > 0.f) || pq == INFINITY) break;
            const float a = __fdividef(rr, pq);
            const f2 a2 = pk(a, a);
            acc0 = 0ull;
            acc1 = 0ull;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                x[k] = fma2(a2, p[k], x[k]);
                r[k] = fma2(a2, q[k], r[k]);  // r - a A p
                if (k & 1) acc1 = fma2(r[k], r[k], acc1);
                else acc0 = fma2(r[k], r[k], acc0);
            }
            acc0 = add2(acc0, acc1);
            const float rrn = warp_sum(lo2(acc0) + hi2(acc0));
            const float beta = __fdividef(rrn, rr);
            rr = rrn;
            const f2 b2 = pk(beta, beta);
#pragma unroll
            for (int k = 0; k < NP; ++k) p[k] = fma2(b2, p[k], r[k]);
            ++nsteps;
        }

        // u_out = u_in + sum_i R_i^T D_i v_i: weight-1 pixels directly, shared
        // pixels through the parity planes.
        // x-only shared pixels go to the compact seam strips that follow the
        // four parity planes: strip[side][ch][seam - 1][y][j], side 0 = left block
        const int nsh = shared_per_seam(o), first = shared_first(o);
        int sx_seam = -1, sx_side = 0, sx_j = 0;
        if (kx > 0 && col >= first && col < first + nsh) {
            sx_seam = kx; sx_side = 1; sx_j = col - first;
        } else if (kx < nbx - 1 && col - s >= first && col - s < first + nsh) {
            sx_seam = kx + 1; sx_side = 0; sx_j = col - s - first;
        }
        float* strip = sx_seam > 0
                           ? planes + 4 * (size_t)C * n +
                                 (((size_t)(sx_side * C + ch) * (nbx - 1) + (sx_seam - 1)) * h) *
                                     nsh + sx_j
                           : planes;
        const int par = (kx & 1) | ((ky & 1) << 1);
        float* plane = planes + ((size_t)par * C + ch) * n;
        float* uo = u_out + ch * n;
        const bool colok = x0 + col < w;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int ly = g * R + k + e * NP;
                if (ly >= bh || !colok) continue;
                const float v = e ? hi2(x[k]) : lo2(x[k]);
                const float d = wx * s_wy[ly];
                const size_t gp = (size_t)(y0 + ly) * w + x0 + col;
                // the first contributor of a shared pixel (smallest block
                // index along each shared axis) also carries u_in, so the
                // combine passes only add parked values
                const float uold = zero_in ? 0.f : tu[(ly + 1) * P + col + 1];
                if (d == 1.f) {
                    uo[gp] = uold + v;
                } else if (d > 0.f) {
                    const float wyr = s_wy[ly];
                    const bool xfirst = sx_seam < 0 || sx_side == 0;  // no left partner on x
                    if (wyr < 1.f) {
                        const bool yfirst = ly >= s;  // upper block of its row overlap
                        plane[gp] = (xfirst && yfirst) ? uold + d * v : d * v;
                    } else {
                        strip[(size_t)(y0 + ly) * nsh] = xfirst ? uold + d * v : d * v;
                    }
                }
                if (d > 0.f) vmax = fmaxf(vmax, fabsf(v));
            }
        }
        if (!more) break;
        blk = nblk_;
        ch = nch;
        buf ^= 1;
    }
    if (step_count && lane == 0) atomicAdd(step_count, (unsigned long long)nsteps);
    if (maxupd) {
        vmax = warp_max(vmax);
        if (lane == 0 && vmax > 0.f) atomicMax(maxupd, __float_as_uint(vmax));
    }
}

// One ORAS iteration for 32x32 blocks with two warps per block (one per half
// of the rows), so every lane keeps 8 packed pairs per CG vector instead of
// 16 and twice as many warps fit on an SM.  Warp wi owns rows 16wi .. 16wi+15
// of every column; pair k of a lane = rows (16wi + k, 16wi + k + 8).  The row
// pair at the seam (15 | 16) is exchanged through shared memory: each warp
// publishes its seam row of r with the r.r partial sum, and rebuilds the
// partner's seam row of p = r + beta p from it.  Two 64-thread barriers per CG
// step (p.Ap and r.r).  Everything else as in k_oras_warp.
struct Tile2W {
    static constexpr int B = 32, TH = 34, P = 34, TILE = TH * P;
    // shared floats: two halo tiles, row weights, two rhs tiles (optional)
    static constexpr int FIXED = 2 * TILE + B;
};

// Shared-memory layout of the FP32 kernel (floats, from a 128-byte aligned
// base): two u tiles of TH rows with pitch PU (a 40-wide TMA box, or the
// 34-wide cp.async copy at column 0), the row weights, with a prolongation
// two patches of 18 x 18 coarse cells, then two right-hand side tiles of B
// rows with pitch PB (36-wide TMA box).  Tile strides are multiples of 128
// bytes, the alignment of a TMA destination.
struct Smem2W {
    static constexpr int B = 32, TH = 34, PU = 40, PB = 36;
    static constexpr int USTRIDE = 1376;            // >= TH * PU, 128-byte multiple
    static constexpr int BSTRIDE = B * PB;          // 1152 floats = 4608 bytes
    static constexpr int WY = 2 * USTRIDE;          // row weights (32 floats)
    static constexpr int RHS = WY + 32;             // 128-byte aligned
    static constexpr int EP = WY + 32;              // coarse patches (prolongation only)
    static constexpr int EW = 18, ES = EW * EW;     // patch side and cells
    static constexpr int EPW = 24, EH = 18;         // patch pitch (a 24-wide TMA box) and rows
    static constexpr int ESTRIDE = 448;             // >= EH * EPW, 128-byte multiple
    static constexpr int RHS_PRO = EP + 2 * ESTRIDE;
    static constexpr int TMA_E_BYTES = EH * EPW * 4;  // 1728
    static constexpr int TMA_U_BYTES = TH * PU * 4; // 5440
    static constexpr int TMA_B_BYTES = B * PB * 4;  // 4608
    static size_t bytes(bool rhs, bool pro = false) {
        return 128 + 4 * (size_t)((pro ? RHS_PRO : RHS) + (rhs ? 2 * BSTRIDE : 0));
    }
};

// The start of an iteration formed by prolongation inside a 32x32 block's
// tile (Section 4.4's cell-centred weights): the block pixels of this
// thread's column (x0 and y0 + row0 are even, so row row0 + k has parent
// patch row 1 + row0 / 2 + k / 2 and takes the coarse row above it for even
// k, below it for odd k; the column likewise), then the halo pixels the
// residual reads: warp 0 the row above the block and the column left of it,
// warp 1 the row below and the column right of it, one pixel of each per
// lane (block pixels of a neighbouring block, which counts them in the
// maximum).  pe: the block's coarse patch (cell (r, q) = coarse row
// y0 / 2 - 1 + r, column x0 / 2 - 1 + q, pitch Smem2W::EPW, clamped to the
// level); mbk: the known bits of the thread's block pixels, hk: of its two
// halo pixels (known or off the image).  ADD: u + P e at unknown pixels
// (a correction), else P e there (an interpolated solution); known pixels
// keep their tile value.  pmax gains the largest |P e| over the unknown
// block pixels.  Branch-free (every patch index stays inside the patch); the
// ten patch rows of both columns and the sixteen tile values are read before
// anything is stored (the stores could alias them otherwise), so the loads
// are in flight together.
template <bool ADD>
__device__ __forceinline__ void prolong_into_tile(float* tw, const float* pe, int row0, int col,
                                                  int lane, int wi, int x0, int y0, uint32_t mbk,
                                                  uint32_t hk, float& pmax) {
    constexpr int EW = Smem2W::EPW, P = Smem2W::PU, B = 32;
    {
        const int q = 1 + (col >> 1), qn = (col & 1) ? q + 1 : q - 1;
        const float* pr = pe + (row0 >> 1) * EW;  // patch row of coarse row Yb - 1
        float* tc = tw + (row0 + 1) * P + col + 1;
        float ec[10], es[10], tv[16];
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            ec[j] = pr[j * EW + q];
            es[j] = pr[j * EW + qn];
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) tv[k] = tc[k * P];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int jc = (k >> 1) + 1, jn = (k & 1) ? jc + 1 : jc - 1;
            const float a = prolong_blend(ec[jc], ec[jn], es[jc], es[jn]);
            const bool kn = (mbk >> k) & 1u;
            tc[k * P] = kn ? tv[k] : (ADD ? __fadd_rn(tv[k], a) : a);
            pmax = fmaxf(pmax, kn ? 0.f : fabsf(a));
        }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int hy = side == 0 ? (wi == 0 ? y0 - 1 : y0 + B) : y0 + lane;
        const int hx = side == 0 ? x0 + lane : (wi == 0 ? x0 - 1 : x0 + B);
        const int r = (hy >> 1) - (y0 >> 1) + 1, q = (hx >> 1) - (x0 >> 1) + 1;
        const int rn = (hy & 1) ? r + 1 : r - 1, qn = (hx & 1) ? q + 1 : q - 1;
        const float a = prolong_blend(pe[r * EW + q], pe[rn * EW + q], pe[r * EW + qn],
                                      pe[rn * EW + qn]);
        float* tp = tw + (hy - y0 + 1) * P + (hx - x0 + 1);
        const bool kn = (hk >> side) & 1u;  // known or off the image
        const float old = *tp;
        *tp = kn ? old : (ADD ? __fadd_rn(old, a) : a);
    }
}

// The coarse cells a task's prolongation reads, by 4-byte cp.async (all 64
// threads): rows (py0 >> 1) - 1 + r and columns (px0 >> 1) - 1 + q, r, q <
// 18, each clamped to the level as the prolongation clamps its indices,
// into dst with pitch Smem2W::EPW.  The caller commits the group.
__device__ __forceinline__ void copy_patch_clamped(float* dst, const float* e, int px0, int py0,
                                                   int wH, int hH, int t) {
    const int Ys = (py0 >> 1) - 1, Xs = (px0 >> 1) - 1;
    for (int i = t; i < Smem2W::ES; i += 64) {
        const int r = i / Smem2W::EW, q = i - r * Smem2W::EW;
        const int Y = min(max(Ys + r, 0), hH - 1), X = min(max(Xs + q, 0), wH - 1);
        cp_async4(dst + r * Smem2W::EPW + q, e + (size_t)Y * wH + X, true);
    }
}

// Known bits of a thread's two halo pixels for prolong_into_tile (bit set:
// known or off the image).
__device__ __forceinline__ uint32_t halo_known_bits(const uint32_t* __restrict__ mbits, int wpr,
                                                    int w, int h, int px0, int py0, int wi,
                                                    int lane) {
    constexpr int B = 32;
    const int hy0 = wi == 0 ? py0 - 1 : py0 + B, hx0 = px0 + lane;
    const int hy1 = py0 + lane, hx1 = wi == 0 ? px0 - 1 : px0 + B;
    uint32_t k = 3u;
    if (hx0 >= 0 && hx0 < w && hy0 >= 0 && hy0 < h &&
        !((__ldg(mbits + (size_t)hy0 * wpr + (hx0 >> 5)) >> (hx0 & 31)) & 1u))
        k &= ~1u;
    if (hx1 >= 0 && hx1 < w && hy1 >= 0 && hy1 < h &&
        !((__ldg(mbits + (size_t)hy1 * wpr + (hx1 >> 5)) >> (hx1 & 31)) & 1u))
        k &= ~2u;
    return k;
}

// Bounded wait for phase `parity` of the mbarrier at shared address `bar`;
// false if it did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int limit = 1 << 20) {
    for (int n = 0; n < limit; ++n) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Self test of the bounded wait: one CTA waits on an mbarrier that no thread
// and no copy ever completes.  *flag = 1 when the wait runs out (the expected
// outcome; the CTA then leaves normally, nothing is in flight), 2 if it
// completed.
__global__ void k_bounded_wait_selftest(unsigned* __restrict__ flag, int limit) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned a = (unsigned)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(a, 0u, limit);
    const int any_out = __syncthreads_or(!ok);
    if (threadIdx.x == 0) *flag = any_out ? 1u : 2u;
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];"
        :
        : "r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
          "r"(bar)
        : "memory");
}

// use_tma: the tiles come by TMA (tm_u over u_in, tm_b over rhs, both FP32
// [C][h][w] with w a multiple of 4); otherwise by 4-byte cp.async.  errflag:
// set to 1 if a TMA wait ran out (the CTA then stops).  use_tma_e (only with
// use_tma): the coarse patches of PRO come by TMA too (tm_e over eH).
// PRO = 1: the iteration starts from u_in + P eH instead of u_in, the coarse
// correction eH [C][hH][wH] prolonged as prolong_body does in mode 1 (added
// at unknown pixels only), so that the V-cycle's correction step needs no
// launch and no pass over the fine iterate of its own; the largest |P eH|
// over the unknown pixels goes to *maxpro.  PRO = 2: the start is u_in at
// the known pixels and P eH at the unknown ones (prolong_body's mode 0 with
// u_in as b: the cascade's interpolation of the coarser level's solution).
// Each block forms the start in its tile (block pixels and halo) before the
// residual.  Needs u_in (not zero_in) and an even block stride, so that the
// parity of a block pixel is that of its tile index.
template <bool F64, int PRO>
__global__ void __launch_bounds__(64, 8)
k_oras_2w(const float* __restrict__ u_in, int zero_in, const float* __restrict__ rhs,
          int rhs_zero, const uint32_t* __restrict__ mbits, int wpr, int w, int h, int C, int o,
          int nbx, int nby, float alpha, int iters, float rtol2, float* __restrict__ u_out,
          float* __restrict__ planes, unsigned* __restrict__ maxupd, int chan_inner,
          const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_b,
          int use_tma, unsigned* __restrict__ errflag,
          unsigned long long* __restrict__ step_count, const float* __restrict__ eH, int wH,
          int hH, unsigned* __restrict__ maxpro, const __grid_constant__ CUtensorMap tm_e,
          int use_tma_e) {
    constexpr int B = 32, NP = 8, TH = Smem2W::TH, P = Smem2W::PU, PB = Smem2W::PB;
    constexpr int TILE = Smem2W::USTRIDE;
    extern __shared__ float smem_raw[];
    float* const smem = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    float* const s_u = smem;                     // [2][USTRIDE]
    float* const s_wy = smem + Smem2W::WY;       // [B]
    float* const s_e = smem + Smem2W::EP;        // [2][ES] if PRO
    float* const s_b = smem + (PRO ? Smem2W::RHS_PRO : Smem2W::RHS);  // [2][BSTRIDE] if rhs_zero == 0
    __shared__ float s_red1[2], s_red2[2], s_seam[2][32];
    __shared__ __align__(8) unsigned long long s_bar[2];

    const int t = threadIdx.x;
    const int lane = t & 31, wi = t >> 5;
    const int col = lane;
    const int row0 = 16 * wi;
    const int s = B - o;
    const size_t n = (size_t)w * h;
    const float inv_o1 = o > 1 ? 1.f / (float)(o - 1) : 0.f;
    // Task sequence of this CTA.  chan_inner: blocks blockIdx.x, +gridDim.x,
    // ... each with all channels back to back (the CTAs running together cover
    // a contiguous band of blocks, so halo re-reads hit L2, and a block's mask
    // bits and operator serve all its channels); otherwise (fewer blocks than
    // CTA slots) tasks blockIdx.x, +gridDim.x, ... of the (block, channel) list.
    const int nblk = nbx * nby;
    // the task after (blk, ch) in this CTA's sequence (no division on the
    // channel-inner path, which the large levels take)
    auto next_task = [&](int& blk, int& ch) {
        if (chan_inner) {
            if (++ch == C) { ch = 0; blk += (int)gridDim.x; }
        } else {
            const int tt = blk * C + ch + (int)gridDim.x;
            blk = tt / C;
            ch = tt - blk * C;
        }
        return blk < nblk;
    };
    uint32_t nlo = 0xffffffffu, nhi = 0xffffffffu;
    uint32_t nhk = 3u;  // PRO: bit i = halo pixel i of this thread (next block) is known or off the image
    auto prefetch = [&](int blk, int ch, int bs, int have_blk) {
        const int px0 = (blk % nbx) * s, py0 = (blk / nbx) * s;
        if constexpr (PRO != 0) {
            // the coarse cells the task's prolongation reads: rows
            // (py0 >> 1) - 1 + r and columns (px0 >> 1) - 1 + q, r, q < 18
            // (with TMA, the box issued below; here each cell is clamped to
            // the level as the prolongation clamps its indices)
            if (!use_tma_e) {
                copy_patch_clamped(s_e + bs * Smem2W::ESTRIDE, eH + (size_t)ch * wH * hH, px0,
                                   py0, wH, hH, t);
                cp_async_commit();
            }
            // this thread's two halo pixels (see the prolongation below)
            if (blk != have_blk) nhk = halo_known_bits(mbits, wpr, w, h, px0, py0, wi, lane);
        }
        if (use_tma) {
            if (t == 0) {
                const unsigned bar =
                    (unsigned)__cvta_generic_to_shared(&s_bar[bs]);
                const unsigned bytes = (zero_in ? 0u : (unsigned)Smem2W::TMA_U_BYTES) +
                                       (rhs_zero ? 0u : (unsigned)Smem2W::TMA_B_BYTES) +
                                       (PRO != 0 && use_tma_e ? (unsigned)Smem2W::TMA_E_BYTES
                                                              : 0u);
                // the buffer's previous contents were read before the loop-top barrier
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             :: "r"(bar), "r"(bytes) : "memory");
                // x must be a multiple of 4 elements (16 bytes): round the
                // halo column down; the tile is indexed from the remainder
                if (!zero_in)
                    tma_load_3d((unsigned)__cvta_generic_to_shared(s_u + bs * TILE), &tm_u,
                                (px0 - 1) & ~3, py0 - 1, ch, bar);
                if (!rhs_zero)
                    tma_load_3d((unsigned)__cvta_generic_to_shared(s_b + bs * Smem2W::BSTRIDE),
                                &tm_b, px0 & ~3, py0, ch, bar);
                // the coarse patch from the 4-aligned column at or below its
                // first one (cells off the level read 0 and are fixed up
                // where the task starts)
                if (PRO != 0 && use_tma_e)
                    tma_load_3d((unsigned)__cvta_generic_to_shared(s_e + bs * Smem2W::ESTRIDE),
                                &tm_e, ((px0 >> 1) - 1) & ~3, (py0 >> 1) - 1, ch, bar);
            }
        } else if (!zero_in) {
            // thread t copies tile column lane of the rows ty = wi, wi + 2, ...
            // (and column 32 + lane for lane < 2)
            const float* src = u_in + ch * n;
            float* dst = s_u + bs * TILE;
            const int gxa = px0 - 1 + lane, gxb = gxa + 32;
            const bool oka = gxa >= 0 && gxa < w;
            const bool okb = lane < TH - 32 && gxb < w;
#pragma unroll 2
            for (int ty = wi; ty < TH; ty += 2) {
                const int gy = py0 - 1 + ty;
                const bool rok = gy >= 0 && gy < h;
                const float* row = src + (ptrdiff_t)gy * w;
                cp_async4(dst + ty * P + lane, (rok && oka) ? row + gxa : src, rok && oka);
                if (lane < TH - 32)
                    cp_async4(dst + ty * P + lane + 32, (rok && okb) ? row + gxb : src, rok && okb);
            }
        }
        if (!use_tma && !rhs_zero) {
            const float* src = rhs + ch * n;
            float* dst = s_b + bs * Smem2W::BSTRIDE;
            const int gx = px0 + lane;
#pragma unroll 4
            for (int ly = wi; ly < B; ly += 2) {
                const int gy = py0 + ly;
                const bool ok = gx < w && gy < h;
                cp_async4(dst + ly * PB + lane, ok ? src + (size_t)gy * w + gx : src, ok);
            }
        }
        if (!use_tma) cp_async_commit();
        if (blk != have_blk && lane < 16) {
            const int gy = py0 + row0 + lane;
            if (gy < h) {
                const uint32_t* row = mbits + (size_t)gy * wpr + (px0 >> 5);
                nlo = __ldg(row);
                nhi = __ldg(row + 1);
            } else {
                nlo = nhi = 0xffffffffu;
            }
        }
    };

    int blk = chan_inner ? (int)blockIdx.x : (int)blockIdx.x / C;
    int ch = chan_inner ? 0 : (int)blockIdx.x - blk * C;
    if (blk >= nblk) return;  // block-uniform
    if (use_tma) {
        if (t == 0) {
            for (int b = 0; b < 2; ++b)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;"
                             :: "r"((unsigned)__cvta_generic_to_shared(&s_bar[b])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        // no thread may probe a barrier before it is initialised (the shared
        // memory still holds whatever an earlier CTA left there)
        __syncthreads();
    }
    unsigned phase = 0;  // bit b: parity of the next completion of s_bar[b]
    prefetch(blk, ch, 0, -1);
    int buf = 0, cur_blk = -1;
    f2 ndg[NP], keep[NP];
    f2 ml2 = 0ull, mr2 = 0ull;
    float wx = 0.f, dh = 0.f;
    int x0 = 0, y0 = 0, bh = 0, kx = 0, ky = 0;
    uint32_t rows_w = 0;  // bit ly: row ly of the block is in the image with weight > 0
    uint32_t mbk = 0;     // bit k: pixel (row0 + k, col) of the block is known or off the image
    float vmax = 0.f, pmax = 0.f;
    unsigned nsteps = 0;  // completed local CG steps of this thread's tasks

    for (;;) {
        if (use_tma) {
            const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[buf]);
            bool ok = mbar_wait(bar, (phase >> buf) & 1u);
            phase ^= 1u << buf;
            if constexpr (PRO != 0) cp_async_wait_all();  // the coarse patch
            if (__syncthreads_or(!ok)) {
                // give the copy one more bounded wait before the CTA leaves
                if (!ok) mbar_wait(bar, ((phase >> buf) & 1u) ^ 1u);
                if (t == 0 && errflag) atomicExch(errflag, 1u);
                return;
            }
        } else {
            cp_async_wait_all();
            __syncthreads();
        }
        const uint32_t mlo = nlo, mhi = nhi, hk = nhk;
        int nb2 = blk, nc2 = ch;
        const bool more = next_task(nb2, nc2);
        if (more) prefetch(nb2, nc2, buf ^ 1, blk);

        if (blk != cur_blk) {
            cur_blk = blk;
            kx = blk % nbx;
            ky = blk / nbx;
            x0 = kx * s;
            y0 = ky * s;
            const int bw = min(B, w - x0);
            bh = min(B, h - y0);
            const uint32_t rowm = __funnelshift_r(mlo, mhi, x0 & 31);  // lane < 16: row row0+lane
            uint32_t mb = 0;
#pragma unroll
            for (int rr = 0; rr < 16; ++rr) {
                const uint32_t v = __shfl_sync(kFull, rowm, rr);
                mb |= ((v >> col) & 1u) << rr;
            }
            const int gx = x0 + col;
            const float hc = (col > 0 ? 1.f : (gx > 0 ? alpha : 0.f)) +
                             (col + 1 < bw ? 1.f : (gx < w - 1 ? alpha : 0.f));
            dh = (float)((gx > 0) + (gx < w - 1));
            const float ml = col > 0 ? 1.f : 0.f, mr = col < B - 1 ? 1.f : 0.f;
            ml2 = pk(ml, ml);
            mr2 = pk(mr, mr);
            if (bh == B) {
                // full height: vertical coupling count 2 except in rows 0 and 31
                const float d2 = -(hc + 2.f);
                const float vt = (y0 > 0 ? alpha : 0.f) + 1.f;
                const float vb = 1.f + (y0 + B < h ? alpha : 0.f);
#pragma unroll
                for (int k = 0; k < NP; ++k) ndg[k] = pk(d2, d2);
                if (wi == 0) ndg[0] = pk(-(hc + vt), d2);
                else ndg[NP - 1] = pk(d2, -(hc + vb));
            } else {
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    float vc[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int ly = row0 + k + 8 * e, gy = y0 + ly;
                        vc[e] = (ly > 0 ? 1.f : (gy > 0 ? alpha : 0.f)) +
                                (ly + 1 < bh ? 1.f : (gy < h - 1 ? alpha : 0.f));
                    }
                    ndg[k] = pk(-(hc + vc[0]), -(hc + vc[1]));
                }
            }
#pragma unroll
            for (int k = 0; k < NP; ++k)
                keep[k] = pk(((mb >> k) & 1u) ? 0.f : 1.f, ((mb >> (k + 8)) & 1u) ? 0.f : 1.f);
            mbk = mb;
            wx = ramp_weight(col, kx, nbx, s, o, inv_o1);
            const float wyl = ramp_weight(lane, ky, nby, s, o, inv_o1);  // row lane
            if (t < B) s_wy[t] = wyl;
            // s_wy is read only after the barriers of the CG below
            rows_w = __ballot_sync(kFull, wyl > 0.f && lane < bh);
        }

        // TMA tiles start at the 4-aligned column below the halo column
        const int du = use_tma ? ((x0 - 1) & 3) : 0;
        const int db = use_tma ? (x0 & 3) : 0;
        const float* tu = s_u + buf * TILE + du;
        const float* tb = s_b + buf * Smem2W::BSTRIDE + db;
        if constexpr (PRO != 0) {
            // the start of the iteration in the tile (prolong_into_tile)
            constexpr int EW = Smem2W::EPW;  // patch pitch
            float* tw = s_u + buf * TILE + du;
            const int Ys = (y0 >> 1) - 1, Xs = (x0 >> 1) - 1;
            // TMA patches start at the 4-aligned column at or below Xs
            const int dqe = use_tma_e ? Xs - (Xs & ~3) : 0;
            float* const pw = s_e + buf * Smem2W::ESTRIDE + dqe;
            if (use_tma_e && (Ys < 0 || Xs < 0 || Ys + Smem2W::EW > hH || Xs + Smem2W::EW > wH)) {
                // a block at the level's border: the cells off the level
                // (read as 0) take the value of their clamped cell, which is
                // on the level and not itself rewritten
                for (int i = t; i < Smem2W::ES; i += 64) {
                    const int r = i / Smem2W::EW, q = i - r * Smem2W::EW;
                    const int Yc = min(max(Ys + r, 0), hH - 1), Xc = min(max(Xs + q, 0), wH - 1);
                    if (Yc != Ys + r || Xc != Xs + q) pw[r * EW + q] = pw[(Yc - Ys) * EW + (Xc - Xs)];
                }
                __syncthreads();  // block-uniform branch
            }
            prolong_into_tile<PRO == 1>(tw, pw, row0, col, lane, wi, x0, y0, mbk, hk, pmax);
            __syncthreads();  // the residual reads the other threads' columns
        }

        f2 x[NP], r[NP], p[NP], q[NP];
        f2 acc0 = 0ull, acc1 = 0ull;
        // r = b - A u on the block (0 on the mask).  The variants: rows off the
        // image's top and bottom rows (vertical degree 2), and b = 0 off the mask.
        // Each run of eight rows walks down the lane's column, so a row's centre
        // is the next row's upper neighbour (one tile load per row for the
        // vertical neighbours instead of three).
        auto residual = [&](auto interior, auto rhs0) {
            float rv[2 * NP];  // rows row0 .. row0 + 15
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float* cb = tu + (row0 + 8 * e + 1) * P + col + 1;  // centre of row 8e
                float up = 0.f, cen = 0.f;
                if (!zero_in) {
                    up = cb[-P];
                    cen = cb[0];
                }
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const int ly = row0 + k + 8 * e, gy = y0 + ly;
                    float v = decltype(rhs0)::value ? 0.f : tb[ly * PB + col];
                    if (!zero_in) {
                        const float* c0 = cb + k * P;
                        const float dn = c0[P];
                        const float dv = decltype(interior)::value
                                             ? 2.f : (float)((gy > 0) + (gy < h - 1));
                        v = res_stencil<F64>(v, dh + dv, cen, up, dn, c0[-1], c0[1]);
                        up = cen;
                        cen = dn;
                    }
                    rv[k + NP * e] = v;
                }
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                r[k] = mul2(pk(rv[k], rv[k + NP]), keep[k]);
                p[k] = r[k];
                x[k] = 0ull;
                if (k & 1) acc1 = fma2(r[k], r[k], acc1);
                else acc0 = fma2(r[k], r[k], acc0);
            }
        };
        if (y0 > 0 && y0 + B < h) {
            if (rhs_zero) residual(std::true_type{}, std::true_type{});
            else residual(std::true_type{}, std::false_type{});
        } else {
            if (rhs_zero) residual(std::false_type{}, std::true_type{});
            else residual(std::false_type{}, std::false_type{});
        }
        acc0 = add2(acc0, acc1);
        // seam rows: warp 0 publishes its row 15 (hi of pair 7), warp 1 its row 16 (lo of pair 0)
        s_seam[wi][lane] = wi == 0 ? hi2(r[NP - 1]) : lo2(r[0]);
        float part = warp_sum(lo2(acc0) + hi2(acc0));
        if (lane == 0) s_red2[wi] = part;
        __syncthreads();
        float rr = s_red2[0] + s_red2[1];
        float pb = s_seam[wi ^ 1][lane];  // partner's seam row of p
        // rtol2 >= 0: relative stop (r.r <= max(rtol2, 1e-14) (r.r)_0); rtol2 < 0:
        // also stop once r.r <= -rtol2 (an absolute level, or the FP32 floor)
        const float rr_stop = rtol2 >= 0.f ? fmaxf(rtol2, 1e-14f) * rr
                                           : fmaxf(1e-14f * rr, -rtol2);

        for (int it = 0; it < iters; ++it) {
            if (!(rr > rr_stop)) break;  // rr is identical in both warps
            const f2 pu = wi == 0 ? pk(0.f, lo2(p[NP - 1])) : pk(pb, lo2(p[NP - 1]));
            const f2 pd = wi == 0 ? pk(hi2(p[0]), pb) : pk(hi2(p[0]), 0.f);
            acc0 = 0ull;
            acc1 = 0ull;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const f2 left = __shfl_up_sync(kFull, p[k], 1);
                const f2 right = __shfl_down_sync(kFull, p[k], 1);
                const f2 up = k > 0 ? p[k - 1] : pu;
                const f2 dn = k < NP - 1 ? p[k + 1] : pd;
                f2 nbs = add2(up, dn);
                nbs = fma2(ml2, left, nbs);
                nbs = fma2(mr2, right, nbs);
                const f2 qk = mul2(fma2(ndg[k], p[k], nbs), keep[k]);  // -(A_i p), 0 on the mask
                q[k] = qk;
                if (k & 1) acc1 = fma2(p[k], qk, acc1);
                else acc0 = fma2(p[k], qk, acc0);
            }
            acc0 = add2(acc0, acc1);
            part = warp_sum(lo2(acc0) + hi2(acc0));
            if (lane == 0) s_red1[wi] = part;
            __syncthreads();
            const float pq = -(s_red1[0] + s_red1[1]);
            if (!(pq > 0.f) || pq == INFINITY) break;
            const float a = __fdividef(rr, pq);
            const f2 a2 = pk(a, a);
            acc0 = 0ull;
            acc1 = 0ull;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                x[k] = fma2(a2, p[k], x[k]);
                r[k] = fma2(a2, q[k], r[k]);
                if (k & 1) acc1 = fma2(r[k], r[k], acc1);
                else acc0 = fma2(r[k], r[k], acc0);
            }
            acc0 = add2(acc0, acc1);
            s_seam[wi][lane] = wi == 0 ? hi2(r[NP - 1]) : lo2(r[0]);
            part = warp_sum(lo2(acc0) + hi2(acc0));
            if (lane == 0) s_red2[wi] = part;
            __syncthreads();
            const float rrn = s_red2[0] + s_red2[1];
            const float beta = __fdividef(rrn, rr);
            rr = rrn;
            const f2 b2 = pk(beta, beta);
#pragma unroll
            for (int k = 0; k < NP; ++k) p[k] = fma2(b2, p[k], r[k]);
            pb = fmaf(beta, pb, s_seam[wi ^ 1][lane]);
            ++nsteps;
        }

        const int nsh = shared_per_seam(o);
        float* uo = u_out + ch * n;
        const bool colok = x0 + col < w;
        if (nsh == 0) {
            // 0/1 weights (overlap 2): each pixel is written by the one block
            // whose weight is 1 there, with u_in added
            if (colok && wx > 0.f) {
                float* uol = uo + (size_t)(y0 + row0) * w + x0 + col;
                const float* tol = tu + (row0 + 1) * P + col + 1;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const int j = k + 8 * e;
                        if (!((rows_w >> (row0 + j)) & 1u)) continue;
                        const float v = e ? hi2(x[k]) : lo2(x[k]);
                        uol[j * w] = (zero_in ? 0.f : tol[j * P]) + v;
                        vmax = fmaxf(vmax, fabsf(v));
                    }
                }
            }
        } else {
            // x-only shared pixels go to the compact seam strips that follow the
            // four parity planes: strip[side][ch][seam - 1][y][j], side 0 = left block
            const int first = shared_first(o);
            int sx_seam = -1, sx_side = 0, sx_j = 0;
            if (kx > 0 && col >= first && col < first + nsh) {
                sx_seam = kx; sx_side = 1; sx_j = col - first;
            } else if (kx < nbx - 1 && col - s >= first && col - s < first + nsh) {
                sx_seam = kx + 1; sx_side = 0; sx_j = col - s - first;
            }
            const size_t strip_row0 =
                ((size_t)(sx_side * C + ch) * (nbx - 1) + (sx_seam - 1)) * h;
            float* strip = sx_seam > 0 ? planes + 4 * (size_t)C * n + strip_row0 * nsh + sx_j
                                       : planes;
            const int par = (kx & 1) | ((ky & 1) << 1);
            float* plane = planes + ((size_t)par * C + ch) * n;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ly = row0 + k + 8 * e;
                    if (ly >= bh || !colok) continue;
                    const float v = e ? hi2(x[k]) : lo2(x[k]);
                    const float d = wx * s_wy[ly];
                    const size_t gp = (size_t)(y0 + ly) * w + x0 + col;
                    // the first contributor of a shared pixel (smallest block
                    // index along each shared axis) also carries u_in, so the
                    // combine passes only add parked values
                    const float uold = zero_in ? 0.f : tu[(ly + 1) * P + col + 1];
                    if (d == 1.f) {
                        uo[gp] = uold + v;
                    } else if (d > 0.f) {
                        const float wyr = s_wy[ly];
                        const bool xfirst = sx_seam < 0 || sx_side == 0;  // no left partner on x
                        if (wyr < 1.f) {
                            const bool yfirst = ly >= s;  // upper block of its row overlap
                            plane[gp] = (xfirst && yfirst) ? uold + d * v : d * v;
                        } else {
                            strip[(size_t)(y0 + ly) * nsh] = xfirst ? uold + d * v : d * v;
                        }
                    }
                    if (d > 0.f) vmax = fmaxf(vmax, fabsf(v));
                }
            }
        }
        if (!more) break;
        blk = nb2;
        ch = nc2;
        buf ^= 1;
    }
    if (step_count && t == 0) atomicAdd(step_count, (unsigned long long)nsteps);
    if (maxupd) {
        vmax = warp_max(vmax);
        if (lane == 0 && vmax > 0.f) atomicMax(maxupd, __float_as_uint(vmax));
    }
    if (PRO == 1 && maxpro) {
        pmax = warp_max(pmax);
        if (lane == 0 && pmax > 0.f) atomicMax(maxpro, __float_as_uint(pmax));
    }
}


// ---- 16-bit storage variant of k_oras_2w ------------------------------------
// The CG vectors, the stencil and the vector updates of each local solve run
// in packed FP16 or BF16 (one 32-bit register per pixel pair, so half the
// registers and one shuffle per pair); the dot products accumulate in FP32,
// the residual that starts each local solve and the update of u stay FP32
// (the outer FP32 iteration refines whatever the narrow local solve leaves).
// The block residual is normalised by its maximum (times 1/64 for FP16, whose
// range is small) before it is narrowed.  A block whose narrow iterate stops
// being finite contributes no correction in this iteration.
struct HalfT {
    typedef __half2 T2;
    static constexpr float kScale = 1.f / 64.f;
    __device__ static __forceinline__ T2 make(float lo, float hi) { return __floats2half2_rn(lo, hi); }
    __device__ static __forceinline__ float lo(T2 a) { return __low2float(a); }
    __device__ static __forceinline__ float hi(T2 a) { return __high2float(a); }
    __device__ static __forceinline__ f2 wide(T2 a) {
        const float2 v = __half22float2(a);
        return pk(v.x, v.y);
    }
};
struct Bf16T {
    typedef __nv_bfloat162 T2;
    static constexpr float kScale = 1.f;
    __device__ static __forceinline__ T2 make(float lo, float hi) { return __floats2bfloat162_rn(lo, hi); }
    __device__ static __forceinline__ float lo(T2 a) { return __low2float(a); }
    __device__ static __forceinline__ float hi(T2 a) { return __high2float(a); }
    __device__ static __forceinline__ f2 wide(T2 a) {
        const float2 v = __bfloat1622float2(a);
        return pk(v.x, v.y);
    }
};

// TU: storage of u_in, rhs and u_out -- float on the finest level (tiles by
// 4-byte cp.async, prefetched while the previous task solves), FP16/BF16 on
// the coarse levels in the 16-bit precision modes (tiles read and widened to
// FP32 at the start of each task).  F64: the block residual in FP64.
template <class H, class TU, bool F64>
__global__ void __launch_bounds__(64, 10)
k_oras_2w_h(const TU* __restrict__ u_in, int zero_in, const TU* __restrict__ rhs,
            int rhs_zero, const uint32_t* __restrict__ mbits, int wpr, int w, int h, int C, int o,
            int nbx, int nby, float alpha, int iters, float rtol2, TU* __restrict__ u_out,
            float* __restrict__ planes, unsigned* __restrict__ maxupd, int chan_inner,
            unsigned long long* __restrict__ step_count) {
    constexpr bool kAsync = std::is_same<TU, float>::value;
    typedef typename H::T2 T2;
    constexpr int B = 32, NP = 8, TH = Tile2W::TH, P = Tile2W::P, TILE = Tile2W::TILE;
    extern __shared__ float smem[];
    float* const s_u = smem;
    float* const s_wy = smem + 2 * TILE;
    float* const s_b = smem + Tile2W::FIXED;
    __shared__ float s_red1[2], s_red2[2], s_seam[2][32], s_mx[2];

    const int t = threadIdx.x;
    const int lane = t & 31, wi = t >> 5;
    const int col = lane;
    const int row0 = 16 * wi;
    const int s = B - o;
    const size_t n = (size_t)w * h;
    const float inv_o1 = o > 1 ? 1.f / (float)(o - 1) : 0.f;
    const int nblk = nbx * nby;
    auto task_of = [&](int i, int& blk, int& ch) {
        if (chan_inner) {
            blk = (int)blockIdx.x + (i / C) * (int)gridDim.x;
            ch = i % C;
        } else {
            const int tt = (int)blockIdx.x + i * (int)gridDim.x;
            blk = tt / C;
            ch = tt - blk * C;
        }
        return blk < nblk;
    };
    uint32_t nlo = 0xffffffffu, nhi = 0xffffffffu;
    // the u tile (block + one-pixel halo) and the right-hand-side tile of a
    // task into buffer bs: asynchronous 4-byte copies (FP32 storage) or plain
    // loads widened to FP32 (16-bit storage)
    auto tiles = [&](int blk, int ch, int bs) {
        const int px0 = (blk % nbx) * s, py0 = (blk / nbx) * s;
        if (!zero_in) {
            const TU* src = u_in + ch * n;
            float* dst = s_u + bs * TILE;
            const int gxa = px0 - 1 + lane, gxb = gxa + 32;
            const bool oka = gxa >= 0 && gxa < w;
            const bool okb = lane < TH - 32 && gxb < w;
#pragma unroll 2
            for (int ty = wi; ty < TH; ty += 2) {
                const int gy = py0 - 1 + ty;
                const bool rok = gy >= 0 && gy < h;
                const TU* row = src + (ptrdiff_t)gy * w;
                if (kAsync) {
                    cp_async4(dst + ty * P + lane,
                              reinterpret_cast<const float*>((rok && oka) ? row + gxa : src),
                              rok && oka);
                    if (lane < TH - 32)
                        cp_async4(dst + ty * P + lane + 32,
                                  reinterpret_cast<const float*>((rok && okb) ? row + gxb : src),
                                  rok && okb);
                } else {
                    dst[ty * P + lane] = (rok && oka) ? ldf(row + gxa) : 0.f;
                    if (lane < TH - 32) dst[ty * P + lane + 32] = (rok && okb) ? ldf(row + gxb) : 0.f;
                }
            }
        }
        if (!rhs_zero) {
            const TU* src = rhs + ch * n;
            float* dst = s_b + bs * B * B;
            const int gx = px0 + lane;
#pragma unroll 4
            for (int ly = wi; ly < B; ly += 2) {
                const int gy = py0 + ly;
                const bool ok = gx < w && gy < h;
                if (kAsync)
                    cp_async4(dst + ly * B + lane,
                              reinterpret_cast<const float*>(ok ? src + (size_t)gy * w + gx : src),
                              ok);
                else
                    dst[ly * B + lane] = ok ? ldf(src + (size_t)gy * w + gx) : 0.f;
            }
        }
        if (kAsync) cp_async_commit();
    };
    auto prefetch = [&](int blk, int ch, int bs, int have_blk) {
        const int px0 = (blk % nbx) * s, py0 = (blk / nbx) * s;
        if (kAsync) tiles(blk, ch, bs);
        if (blk != have_blk && lane < 16) {
            const int gy = py0 + row0 + lane;
            if (gy < h) {
                const uint32_t* row = mbits + (size_t)gy * wpr + (px0 >> 5);
                nlo = __ldg(row);
                nhi = __ldg(row + 1);
            } else {
                nlo = nhi = 0xffffffffu;
            }
        }
    };

    int blk, ch;
    if (!task_of(0, blk, ch)) return;
    prefetch(blk, ch, 0, -1);
    int buf = 0, cur_blk = -1;
    T2 ndg[NP], keep[NP];
    T2 ml2 = H::make(0.f, 0.f), mr2 = H::make(0.f, 0.f);
    float wx = 0.f, dh = 0.f;
    int x0 = 0, y0 = 0, bh = 0, kx = 0, ky = 0;
    float vmax = 0.f;
    unsigned nsteps = 0;  // completed local CG steps of this thread's tasks

    for (int i = 0;; ++i) {
        if (kAsync) cp_async_wait_all();
        __syncthreads();
        if (!kAsync) {
            // the previous readers of this buffer finished before the barrier
            tiles(blk, ch, buf);
            __syncthreads();
        }
        const uint32_t mlo = nlo, mhi = nhi;
        int nb2, nc2;
        const bool more = task_of(i + 1, nb2, nc2);
        if (more) prefetch(nb2, nc2, buf ^ 1, blk);

        if (blk != cur_blk) {
            cur_blk = blk;
            kx = blk % nbx;
            ky = blk / nbx;
            x0 = kx * s;
            y0 = ky * s;
            const int bw = min(B, w - x0);
            bh = min(B, h - y0);
            const uint32_t rowm = __funnelshift_r(mlo, mhi, x0 & 31);
            uint32_t mb = 0;
#pragma unroll
            for (int rr = 0; rr < 16; ++rr) {
                const uint32_t v = __shfl_sync(kFull, rowm, rr);
                mb |= ((v >> col) & 1u) << rr;
            }
            const int gx = x0 + col;
            const float hc = (col > 0 ? 1.f : (gx > 0 ? alpha : 0.f)) +
                             (col + 1 < bw ? 1.f : (gx < w - 1 ? alpha : 0.f));
            dh = (float)((gx > 0) + (gx < w - 1));
            const float ml = col > 0 ? 1.f : 0.f, mr = col < B - 1 ? 1.f : 0.f;
            ml2 = H::make(ml, ml);
            mr2 = H::make(mr, mr);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                float vc[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ly = row0 + k + 8 * e, gy = y0 + ly;
                    vc[e] = (ly > 0 ? 1.f : (gy > 0 ? alpha : 0.f)) +
                            (ly + 1 < bh ? 1.f : (gy < h - 1 ? alpha : 0.f));
                }
                ndg[k] = H::make(-(hc + vc[0]), -(hc + vc[1]));
                keep[k] = H::make(((mb >> k) & 1u) ? 0.f : 1.f, ((mb >> (k + 8)) & 1u) ? 0.f : 1.f);
            }
            wx = ramp_weight(col, kx, nbx, s, o, inv_o1);
            if (t < B) s_wy[t] = ramp_weight(t, ky, nby, s, o, inv_o1);
        }

        const float* tu = s_u + buf * TILE;
        const float* tb = s_b + buf * B * B;

        // FP32 residual of the block, then its maximum for the normalisation
        float rv[NP][2];
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int ly = row0 + k + 8 * e, gy = y0 + ly;
                float v = rhs_zero ? 0.f : tb[ly * B + col];
                if (!zero_in) {
                    const float* c0 = tu + (ly + 1) * P + col + 1;
                    const float dv = (float)((gy > 0) + (gy < h - 1));
                    v = res_stencil<F64>(v, dh + dv, c0[0], c0[-P], c0[P], c0[-1], c0[1]);
                }
                v *= e ? H::hi(keep[k]) : H::lo(keep[k]);
                rv[k][e] = v;
                mx = fmaxf(mx, fabsf(v));
            }
        }
        mx = warp_max(mx);
        if (lane == 0) s_mx[wi] = mx;
        __syncthreads();
        mx = fmaxf(s_mx[0], s_mx[1]);
        const float sc = mx > 0.f ? mx / H::kScale : 1.f;  // r = sc * r_narrow
        const float isc = 1.f / sc;

        T2 x[NP], r[NP], p[NP], q[NP];
        f2 acc0 = 0ull, acc1 = 0ull;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            r[k] = H::make(rv[k][0] * isc, rv[k][1] * isc);
            p[k] = r[k];
            x[k] = H::make(0.f, 0.f);
            const f2 rw = H::wide(r[k]);
            if (k & 1) acc1 = fma2(rw, rw, acc1);
            else acc0 = fma2(rw, rw, acc0);
        }
        acc0 = add2(acc0, acc1);
        s_seam[wi][lane] = wi == 0 ? H::hi(r[NP - 1]) : H::lo(r[0]);
        float part = warp_sum(lo2(acc0) + hi2(acc0));
        if (lane == 0) s_red2[wi] = part;
        __syncthreads();
        float rr = s_red2[0] + s_red2[1];
        float pb = s_seam[wi ^ 1][lane];
        // rtol2 >= 0: relative stop (r.r <= max(rtol2, 1e-14) (r.r)_0); rtol2 < 0:
        // also stop once r.r <= -rtol2 (an absolute level, or the FP32 floor). rr is
        // the normalised residual's, so the absolute level is scaled by isc^2 too.
        const float rr_stop = rtol2 >= 0.f ? fmaxf(rtol2, 1e-14f) * rr
                                           : fmaxf(1e-14f * rr, -rtol2 * isc * isc);
        bool bad = !(rr < INFINITY);

        for (int it = 0; it < iters; ++it) {
            if (!(rr > rr_stop) || bad) break;  // identical in both warps
            const T2 pu = wi == 0 ? H::make(0.f, H::lo(p[NP - 1])) : H::make(pb, H::lo(p[NP - 1]));
            const T2 pd = wi == 0 ? H::make(H::hi(p[0]), pb) : H::make(H::hi(p[0]), 0.f);
            acc0 = 0ull;
            acc1 = 0ull;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const T2 left = __shfl_up_sync(kFull, p[k], 1);
                const T2 right = __shfl_down_sync(kFull, p[k], 1);
                const T2 up = k > 0 ? p[k - 1] : pu;
                const T2 dn = k < NP - 1 ? p[k + 1] : pd;
                T2 nbs = __hadd2(up, dn);
                nbs = __hfma2(ml2, left, nbs);
                nbs = __hfma2(mr2, right, nbs);
                const T2 qk = __hmul2(__hfma2(ndg[k], p[k], nbs), keep[k]);
                q[k] = qk;
                if (k & 1) acc1 = fma2(H::wide(p[k]), H::wide(qk), acc1);
                else acc0 = fma2(H::wide(p[k]), H::wide(qk), acc0);
            }
            acc0 = add2(acc0, acc1);
            part = warp_sum(lo2(acc0) + hi2(acc0));
            if (lane == 0) s_red1[wi] = part;
            __syncthreads();
            const float pq = -(s_red1[0] + s_red1[1]);
            if (!(pq > 0.f) || !(pq < INFINITY)) {
                bad = !(pq < INFINITY) || pq != pq;
                break;
            }
            const float a = __fdividef(rr, pq);
            const T2 a2 = H::make(a, a);
            acc0 = 0ull;
            acc1 = 0ull;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                x[k] = __hfma2(a2, p[k], x[k]);
                r[k] = __hfma2(a2, q[k], r[k]);
                const f2 rw = H::wide(r[k]);
                if (k & 1) acc1 = fma2(rw, rw, acc1);
                else acc0 = fma2(rw, rw, acc0);
            }
            acc0 = add2(acc0, acc1);
            s_seam[wi][lane] = wi == 0 ? H::hi(r[NP - 1]) : H::lo(r[0]);
            part = warp_sum(lo2(acc0) + hi2(acc0));
            if (lane == 0) s_red2[wi] = part;
            __syncthreads();
            const float rrn = s_red2[0] + s_red2[1];
            if (!(rrn < INFINITY)) { bad = true; break; }
            const float beta = __fdividef(rrn, rr);
            rr = rrn;
            const T2 b2 = H::make(beta, beta);
#pragma unroll
            for (int k = 0; k < NP; ++k) p[k] = __hfma2(b2, p[k], r[k]);
            pb = fmaf(beta, pb, s_seam[wi ^ 1][lane]);
            ++nsteps;
        }

        const int par = (kx & 1) | ((ky & 1) << 1);
        float* plane = planes + ((size_t)par * C + ch) * n;
        TU* uo = u_out + ch * n;
        const bool colok = x0 + col < w;
        const int nsh = shared_per_seam(o), first = shared_first(o);
        int sx_seam = -1, sx_side = 0, sx_j = 0;
        if (kx > 0 && col >= first && col < first + nsh) {
            sx_seam = kx; sx_side = 1; sx_j = col - first;
        } else if (kx < nbx - 1 && col - s >= first && col - s < first + nsh) {
            sx_seam = kx + 1; sx_side = 0; sx_j = col - s - first;
        }
        float* strip = sx_seam > 0
                           ? planes + 4 * (size_t)C * n +
                                 (((size_t)(sx_side * C + ch) * (nbx - 1) + (sx_seam - 1)) * h) *
                                     nsh + sx_j
                           : planes;
        const float vs = bad ? 0.f : sc;  // a non-finite narrow iterate gives no correction
#pragma unroll
        for (int k = 0; k < NP; ++k) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int ly = row0 + k + 8 * e;
                if (ly >= bh || !colok) continue;
                const float v = (e ? H::hi(x[k]) : H::lo(x[k])) * vs;
                const float d = wx * s_wy[ly];
                const size_t gp = (size_t)(y0 + ly) * w + x0 + col;
                const float uold = zero_in ? 0.f : tu[(ly + 1) * P + col + 1];
                if (d == 1.f) {
                    stf(uo + gp, uold + v);
                } else if (d > 0.f) {
                    const float wyr = s_wy[ly];
                    const bool xfirst = sx_seam < 0 || sx_side == 0;
                    if (wyr < 1.f) {
                        const bool yfirst = ly >= s;
                        plane[gp] = (xfirst && yfirst) ? uold + d * v : d * v;
                    } else {
                        strip[(size_t)(y0 + ly) * nsh] = xfirst ? uold + d * v : d * v;
                    }
                }
                if (d > 0.f) vmax = fmaxf(vmax, fabsf(v));
            }
        }
        if (!more) break;
        blk = nb2;
        ch = nc2;
        buf ^= 1;
    }
    if (step_count && t == 0) atomicAdd(step_count, (unsigned long long)nsteps);
    if (maxupd) {
        vmax = warp_max(vmax);
        if (lane == 0 && vmax > 0.f) atomicMax(maxupd, __float_as_uint(vmax));
    }
}

// Shared rows (the interior rows of every horizontal overlap), full width:
// contributions from the parity planes (two block rows; two block columns
// where the pixel is also shared along x).
template <class TU>
__global__ void __launch_bounds__(256)
k_combine_rows(const float* __restrict__ planes,
               int w, int h, int s, int o, int nbx, int nby, float inv_s,
               TU* __restrict__ u_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.z, C = gridDim.z;
    if (x >= w) return;
    const int nsh = shared_per_seam(o);
    const int seam = blockIdx.y / nsh + 1;             // lower block row of the overlap
    const int y = seam * s + shared_first(o) + (int)blockIdx.y % nsh;
    if (y >= h) return;
    int kx0, kx1;
    const int nx = axis_contrib(x, s, o, nbx, kx0, kx1, inv_s);
    const size_t n = (size_t)w * h, gp = (size_t)y * w + x;
    const size_t cs = (size_t)C * n;
    const float* pl = planes + ch * n + gp;
    const int pu = (seam - 1) & 1, pdn = seam & 1;  // y parity of the upper / lower block
    // the first term (upper-left block) already carries u_in
    float acc = pl[(size_t)((kx0 & 1) | (pu << 1)) * cs];
    if (nx == 2) acc += pl[(size_t)((kx1 & 1) | (pu << 1)) * cs];
    acc += pl[(size_t)((kx0 & 1) | (pdn << 1)) * cs];
    if (nx == 2) acc += pl[(size_t)((kx1 & 1) | (pdn << 1)) * cs];
    stf(u_out + ch * n + gp, acc);
}

// Pixels shared along x only: thread (j, row) adds the strip entries of the
// left and right block for pixel j of the seam's shared run in that row (j
// fastest, so the strip reads of a warp are contiguous).
template <class TU>
__global__ void __launch_bounds__(256)
k_combine_cols(const float* __restrict__ planes,
               int w, int h, int s, int o, int nbx, int nby, float inv_s,
               TU* __restrict__ u_out) {
    const int j = threadIdx.x;
    const int y = blockIdx.x * blockDim.y + threadIdx.y;
    const int seam = (int)blockIdx.y + 1;
    const int ch = blockIdx.z, C = gridDim.z;
    if (y >= h) return;
    const int x = seam * s + shared_first(o) + j;
    if (x >= w) return;
    int ky0, ky1;
    if (axis_contrib(y, s, o, nby, ky0, ky1, inv_s) == 2) return;  // shared row: k_combine_rows
    const int nsh = shared_per_seam(o);
    const size_t n = (size_t)w * h;
    const float* strips = planes + 4 * (size_t)C * n;
    const size_t side = (size_t)C * (nbx - 1) * h * nsh;
    const size_t at = (((size_t)ch * (nbx - 1) + (seam - 1)) * h + y) * nsh + j;
    // the left block's entry already carries u_in
    stf(u_out + ch * n + (size_t)y * w + x, strips[at] + strips[at + side]);
}

// ---------------------------------------------------------------------------
// Device-driven decode: the plan and the stop test (Section 5.2 stop criterion;
// the error-estimate rule in gray levels).  One thread each; they steer the
// conditional nodes of the decode graph.
// ---------------------------------------------------------------------------

__global__ void k_plan(const unsigned long long* __restrict__ counts, StopState* __restrict__ st,
                       PlanParams p) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int L = p.L;
    const unsigned long long unk0 = counts[1];
    // levels down to the first one without unknown pixels (max pooling keeps
    // a known pixel known, so every coarser level is fully known too)
    int Leff = L;
    for (int l = 1; l < L; ++l)
        if (counts[1 + l] == 0) { Leff = l; break; }
    if (unk0 == 0) Leff = 0;
    st->cycles = 0;
    st->converged = 0;
    st->levels_used = Leff;
    st->est = 0.f;
    st->prevU = -1.f;
    st->prevQ = -1.f;
    st->unknowns = unk0;
    for (int k = 0; k < kMaxChannels; ++k) st->rel[k] = -1.f;
    const bool empty = unk0 == p.n0;
    st->status = empty ? DI_ERR_EMPTY_MASK : DI_OK;
    if (empty) {
        cudaGraphSetConditional(p.h_sel, kSelSkip);
        return;
    }
    if (Leff == 0) st->converged = 1;  // every pixel known: u = f
    cudaGraphSetConditional(p.h_sel, (unsigned)Leff);
    if (Leff > 0) cudaGraphSetConditional(p.h_loop[Leff], p.max_cycles > 0 ? 1u : 0u);
}

// The stop test of the host loop, on the device: the same float arithmetic
// in the same order, so the decisions are identical.
__global__ void k_stop(unsigned* __restrict__ upd, StopState* __restrict__ st, StopParams p,
                       cudaGraphConditionalHandle h_loop) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int cycles = st->cycles + 1;
    st->cycles = cycles;
    bool stop = false;
    if (upd[kMaxUpdSlots]) {
        st->status = DI_ERR_TIMEOUT;
        stop = true;
    } else if (p.rule == DI_STOP_ERROR_ESTIMATE) {
        float U = 0.f;
        for (int k = 0; k < p.nslots; ++k) U += __uint_as_float(upd[k]);
        float prevU = st->prevU, prevQ = st->prevQ, est;
        if (!isfinite(U)) {
            est = INFINITY;
            prevU = -1.f;
            prevQ = -1.f;
        } else if (prevU > 0.f) {
            // decay factor: the larger of the last two measured ratios
            const float qk = __fdiv_rn(U, prevU);
            const float q = prevQ > qk ? prevQ : qk;
            prevQ = qk;
            est = q < 1.f ? __fdiv_rn(__fmul_rn(U, q), __fsub_rn(1.f, q)) : INFINITY;
        } else {
            est = U;  // first cycle: no decay measured yet
        }
        prevU = U;
        if (U == 0.f) est = 0.f;
        st->prevU = prevU;
        st->prevQ = prevQ;
        st->est = est;
        if (cycles >= p.min_cycles && est <= 0.5f * p.tol) {
            st->converged = 1;
            stop = true;
        }
    } else if (p.rule == DI_STOP_RELATIVE_RESIDUAL) {
        bool ok = true;
        for (int k = 0; k < p.C; ++k) {
            const double b2 = st->bnorm2[k];
            const double rr = b2 > 0 ? sqrt(st->norm2[k] / b2) : 0.0;
            st->rel[k] = (float)rr;
            if (!(rr <= (double)p.tol)) ok = false;
        }
        if (cycles >= p.min_cycles && ok) {
            st->converged = 1;
            stop = true;
        }
    } else if (cycles >= p.max_cycles) {  // fixed number of cycles
        st->converged = 1;
        stop = true;
    }
    if (!stop && cycles >= p.max_cycles) {
        st->status = DI_ERR_NOT_CONVERGED;
        stop = true;
    }
    for (int k = 0; k < p.nslots; ++k) upd[k] = 0u;
    cudaGraphSetConditional(h_loop, stop ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// Batched form: the step kernels over the segments of a batch (one image's
// level each).  A CTA finds its segment by binary search over the segments'
// first CTAs, skips it if the image does not take part in this step, and runs
// the single-image body on the segment's buffers.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int find_seg(const BatchSeg* __restrict__ segs, int nseg, int g) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].first <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool seg_active(int when, int img, int level, int L,
                                           const BatchState& bs) {
    switch (when) {
        case kWhenTopEq: return bs.top[img] == level;
        case kWhenCoarsestStart: return bs.leff[img] == L;
        case kWhenBelowTop: return level < bs.top[img];
        case kWhenCycle: return !bs.done[img] && level < bs.leff[img];
        default: return true;
    }
}

template <int KIND>
__global__ void __launch_bounds__(256)
k_batch_grid(const BatchSeg* __restrict__ segs, int nseg, BatchState bs) {
    const BatchSeg& sg = segs[find_seg(segs, nseg, (int)blockIdx.x)];
    if (!seg_active(sg.when, sg.img, sg.level, sg.L, bs)) return;  // uniform per CTA
    const int local = (int)blockIdx.x - sg.first;
    const int w = sg.w, h = sg.h;
    const int wH = (w + 1) / 2, hH = (h + 1) / 2;
    if (KIND == kBPack) {
        pack_mask_body(static_cast<const uint8_t*>(sg.in0), w, h, const_cast<uint32_t*>(sg.mbits),
                       sg.wpr, sg.counter, local, sg.gx);
        return;
    }
    if (KIND == kBSelect) {
        const int ch = local / sg.gx, bx = local - ch * sg.gx;
        const size_t n = (size_t)w * h;
        select_body<float>(static_cast<const float*>(sg.in1), static_cast<const uint8_t*>(sg.in2),
                           n, static_cast<float*>(sg.out0), sg.keep, bx, sg.gx, ch);
        if (sg.out1)
            select_body<float>(static_cast<const float*>(sg.in1),
                               static_cast<const uint8_t*>(sg.in2), n,
                               static_cast<float*>(sg.out1), sg.keep, bx, sg.gx, ch);
        return;
    }
    const int plane = sg.gx * sg.gy;
    const int bz = local / plane, rem = local - bz * plane;
    const int by = rem / sg.gx, bx = rem - by * sg.gx;
    if (KIND == kBPyramid)
        pyramid_level_body(static_cast<const uint8_t*>(sg.in0), static_cast<const float*>(sg.in1),
                           w, h, sg.C, static_cast<uint8_t*>(sg.out0),
                           static_cast<float*>(sg.out1), wH, hH, sg.mode, 1,
                           const_cast<uint32_t*>(sg.mbits), sg.wpr, sg.counter, bx, by, sg.gx);
    else if (KIND == kBMaskDown)
        mask_down_body(static_cast<const uint8_t*>(sg.in0), w, h, static_cast<uint8_t*>(sg.out0),
                       wH, hH, bx, by);
    else if (KIND == kBValuesDown)
        values_down_body(static_cast<const uint8_t*>(sg.in0), static_cast<const float*>(sg.in1),
                         w, h, sg.C, static_cast<const uint8_t*>(sg.in2),
                         static_cast<float*>(sg.out0), wH, hH, sg.mode, bx, by);
    else if (KIND == kBRestrict)
        restrict_body<false, float, float, float, false>(
            static_cast<const float*>(sg.in0), static_cast<const float*>(sg.in1), sg.rhs_zero, w,
            h, static_cast<const uint8_t*>(sg.in2), static_cast<float*>(sg.out0), wH, hH, bx, by,
            bz);
    else if (KIND == kBProlong)
        prolong_body<false, float, float>(static_cast<const float*>(sg.in0), wH, hH,
                                          static_cast<const float*>(sg.in1),
                                          static_cast<const uint8_t*>(sg.in2), w, h,
                                          static_cast<float*>(sg.out0), sg.mode, sg.maxupd, bx,
                                          by, bz);
}

// The block kernel over the block units of a batch: a unit is one 32x32
// block of one image's level with all its channels back to back; CTAs are
// persistent and stride over the units of every image in the launch, skipping
// the units of images that do not take part.  Tiles by TMA through each
// segment's tensor maps, or by 4-byte cp.async where an image does not allow
// TMA (prefetched while the previous task solves; a TMA wait that runs out
// sets *bs.err and the CTA leaves); 0/1 partition weights (overlap 2: each
// pixel is written by the one block whose weight is 1 there); a segment may
// form its start by prolongation (BatchSeg).  Otherwise the local problem,
// the CG and the write are those of k_oras_2w.
__global__ void __launch_bounds__(64, 8)
k_batch_oras(const BatchSeg* __restrict__ segs, int nseg, int nunits, int o, float alpha,
             BatchState bs) {
    constexpr int B = 32, NP = 8, TH = Smem2W::TH, P = Smem2W::PU, PB = Smem2W::PB;
    constexpr int TILE = Smem2W::USTRIDE;
    extern __shared__ float smem_raw[];
    float* const smem = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    float* const s_u = smem;
    float* const s_wy = smem + Smem2W::WY;
    float* const s_e = smem + Smem2W::EP;  // coarse patches of prolonging segments
    float* const s_b = smem + Smem2W::RHS_PRO;
    __shared__ float s_red1[2], s_red2[2], s_seam[2][32];
    __shared__ __align__(8) unsigned long long s_bar[2];  // TMA tiles of buffer 0, 1

    const int t = threadIdx.x;
    const int lane = t & 31, wi = t >> 5;
    const int col = lane;
    const int row0 = 16 * wi;
    const int s = B - o;
    const float inv_o1 = o > 1 ? 1.f / (float)(o - 1) : 0.f;
    // whether a segment's tasks form their start by prolongation (uniform per task)
    auto prolongs = [&](const BatchSeg& sg) {
        return sg.pro_mode != 0 && (!sg.pro_check || sg.level + 1 < bs.leff[sg.img]);
    };

    // a task: a unit's segment and block, and a channel
    struct Task {
        int seg, blk, ch;
    };
    // the next active task after (unit g, channel ch): the next channel, else
    // the next unit of this CTA whose image takes part
    auto advance = [&](int& g, Task& tk) {
        if (tk.seg >= 0 && ++tk.ch < segs[tk.seg].C) return true;
        for (g = g < 0 ? (int)blockIdx.x : g + (int)gridDim.x; g < nunits; g += (int)gridDim.x) {
            const int si = find_seg(segs, nseg, g);
            const BatchSeg& sg = segs[si];
            if (!seg_active(sg.when, sg.img, sg.level, sg.L, bs)) continue;
            tk.seg = si;
            tk.blk = g - sg.first;
            tk.ch = 0;
            return true;
        }
        return false;
    };
    uint32_t nlo = 0xffffffffu, nhi = 0xffffffffu, nhk = 3u;
    // bit b: buffer b awaits a TMA completion; parity of its next completion
    unsigned pend_tma = 0, phase = 0;
    auto prefetch = [&](const Task& tk, int bs_, bool new_blk) {
        const BatchSeg& sg = segs[tk.seg];
        const int w = sg.w, h = sg.h, nbx = sg.nbx;
        const size_t n = (size_t)w * h;
        const int px0 = (tk.blk % nbx) * s, py0 = (tk.blk / nbx) * s;
        if (prolongs(sg)) {
            const int wH = (w + 1) / 2, hH = (h + 1) / 2;
            copy_patch_clamped(s_e + bs_ * Smem2W::ESTRIDE, sg.pro_e + (size_t)tk.ch * wH * hH,
                               px0, py0, wH, hH, t);
            if (new_blk) nhk = halo_known_bits(sg.mbits, sg.wpr, w, h, px0, py0, wi, lane);
        }
        if (sg.tma) {
            // the tiles by TMA, as in k_oras_2w (x rounded down to a multiple
            // of 4; the tile is indexed from the remainder)
            if (t == 0) {
                const CUtensorMap* maps = static_cast<const CUtensorMap*>(sg.tmaps);
                const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[bs_]);
                const unsigned bytes = (sg.zero_in ? 0u : (unsigned)Smem2W::TMA_U_BYTES) +
                                       (sg.rhs_zero ? 0u : (unsigned)Smem2W::TMA_B_BYTES);
                // the buffer's previous contents were read before the loop-top barrier
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             :: "r"(bar), "r"(bytes) : "memory");
                if (!sg.zero_in)
                    tma_load_3d((unsigned)__cvta_generic_to_shared(s_u + bs_ * TILE), &maps[0],
                                (px0 - 1) & ~3, py0 - 1, tk.ch, bar);
                if (!sg.rhs_zero)
                    tma_load_3d((unsigned)__cvta_generic_to_shared(s_b + bs_ * Smem2W::BSTRIDE),
                                &maps[1], px0 & ~3, py0, tk.ch, bar);
            }
            pend_tma |= 1u << bs_;
        } else if (!sg.zero_in) {
            const float* src = static_cast<const float*>(sg.in0) + tk.ch * n;
            float* dst = s_u + bs_ * TILE;
            const int gxa = px0 - 1 + lane, gxb = gxa + 32;
            const bool oka = gxa >= 0 && gxa < w;
            const bool okb = lane < TH - 32 && gxb < w;
#pragma unroll 2
            for (int ty = wi; ty < TH; ty += 2) {
                const int gy = py0 - 1 + ty;
                const bool rok = gy >= 0 && gy < h;
                const float* row = src + (ptrdiff_t)gy * w;
                cp_async4(dst + ty * P + lane, (rok && oka) ? row + gxa : src, rok && oka);
                if (lane < TH - 32)
                    cp_async4(dst + ty * P + lane + 32, (rok && okb) ? row + gxb : src, rok && okb);
            }
        }
        if (!sg.tma && !sg.rhs_zero) {
            const float* src = static_cast<const float*>(sg.in1) + tk.ch * n;
            float* dst = s_b + bs_ * Smem2W::BSTRIDE;
            const int gx = px0 + lane;
#pragma unroll 4
            for (int ly = wi; ly < B; ly += 2) {
                const int gy = py0 + ly;
                const bool ok = gx < w && gy < h;
                cp_async4(dst + ly * PB + lane, ok ? src + (size_t)gy * w + gx : src, ok);
            }
        }
        cp_async_commit();
        if (new_blk && lane < 16) {
            const int gy = py0 + row0 + lane;
            if (gy < h) {
                const uint32_t* row = sg.mbits + (size_t)gy * sg.wpr + (px0 >> 5);
                nlo = __ldg(row);
                nhi = __ldg(row + 1);
            } else {
                nlo = nhi = 0xffffffffu;
            }
        }
    };

    int g = -1;
    Task cur{-1, 0, 0};
    if (!advance(g, cur)) return;  // block-uniform
    if (t == 0) {
        for (int k = 0; k < 2; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;"
                         :: "r"((unsigned)__cvta_generic_to_shared(&s_bar[k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // no thread may probe a barrier before it is initialised
    __syncthreads();
    prefetch(cur, 0, true);
    int buf = 0;
    int cur_seg = -1, cur_blk = -1;
    f2 ndg[NP], keep[NP];
    f2 ml2 = 0ull, mr2 = 0ull;
    float wx = 0.f, dh = 0.f;
    int x0 = 0, y0 = 0, bh = 0, kx = 0, ky = 0;
    uint32_t rows_w = 0, mbk = 0;
    float vmax = 0.f, pmax = 0.f;
    unsigned* vmax_slot = nullptr;
    unsigned* pmax_slot = nullptr;

    for (;;) {
        cp_async_wait_all();
        if ((pend_tma >> buf) & 1u) {  // uniform: the task's segment decides
            const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[buf]);
            const bool ok = mbar_wait(bar, (phase >> buf) & 1u);
            phase ^= 1u << buf;
            pend_tma &= ~(1u << buf);
            if (__syncthreads_or(!ok)) {
                // give the copy one more bounded wait before the CTA leaves
                if (!ok) mbar_wait(bar, ((phase >> buf) & 1u) ^ 1u);
                if (t == 0 && bs.err) atomicExch(bs.err, 1u);
                return;
            }
        } else {
            __syncthreads();
        }
        const uint32_t mlo = nlo, mhi = nhi, hk = nhk;
        Task nxt = cur;
        int g2 = g;
        const bool more = advance(g2, nxt);
        if (more) prefetch(nxt, buf ^ 1, nxt.seg != cur.seg || nxt.blk != cur.blk);

        const BatchSeg& sg = segs[cur.seg];
        const int w = sg.w, h = sg.h, nbx = sg.nbx, nby = sg.nby;
        const int zero_in = sg.zero_in, rhs_zero = sg.rhs_zero;
        const size_t n = (size_t)w * h;
        if (cur.seg != cur_seg) {
            // the image changes: flush the previous image's largest update
            if (vmax_slot) {
                const float m = warp_max(vmax);
                if (lane == 0 && m > 0.f) atomicMax(vmax_slot, __float_as_uint(m));
            }
            if (pmax_slot) {
                const float m = warp_max(pmax);
                if (lane == 0 && m > 0.f) atomicMax(pmax_slot, __float_as_uint(m));
            }
            vmax = 0.f;
            pmax = 0.f;
            vmax_slot = sg.maxupd;
            pmax_slot = sg.pro_mode == 1 ? sg.pro_max : nullptr;
            cur_seg = cur.seg;
            cur_blk = -1;
        }
        if (cur.blk != cur_blk) {
            cur_blk = cur.blk;
            kx = cur.blk % nbx;
            ky = cur.blk / nbx;
            x0 = kx * s;
            y0 = ky * s;
            const int bw = min(B, w - x0);
            bh = min(B, h - y0);
            const uint32_t rowm = __funnelshift_r(mlo, mhi, x0 & 31);
            uint32_t mb = 0;
#pragma unroll
            for (int rr = 0; rr < 16; ++rr) {
                const uint32_t v = __shfl_sync(kFull, rowm, rr);
                mb |= ((v >> col) & 1u) << rr;
            }
            const int gx = x0 + col;
            const float hc = (col > 0 ? 1.f : (gx > 0 ? alpha : 0.f)) +
                             (col + 1 < bw ? 1.f : (gx < w - 1 ? alpha : 0.f));
            dh = (float)((gx > 0) + (gx < w - 1));
            const float ml = col > 0 ? 1.f : 0.f, mr = col < B - 1 ? 1.f : 0.f;
            ml2 = pk(ml, ml);
            mr2 = pk(mr, mr);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                float vc[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ly = row0 + k + 8 * e, gy = y0 + ly;
                    vc[e] = (ly > 0 ? 1.f : (gy > 0 ? alpha : 0.f)) +
                            (ly + 1 < bh ? 1.f : (gy < h - 1 ? alpha : 0.f));
                }
                ndg[k] = pk(-(hc + vc[0]), -(hc + vc[1]));
                keep[k] = pk(((mb >> k) & 1u) ? 0.f : 1.f, ((mb >> (k + 8)) & 1u) ? 0.f : 1.f);
            }
            mbk = mb;
            wx = ramp_weight(col, kx, nbx, s, o, inv_o1);
            const float wyl = ramp_weight(lane, ky, nby, s, o, inv_o1);
            if (t < B) s_wy[t] = wyl;
            rows_w = __ballot_sync(kFull, wyl > 0.f && lane < bh);
        }
        // TMA tiles start at the 4-aligned column below the halo column
        const int du = sg.tma ? ((x0 - 1) & 3) : 0;
        const int db = sg.tma ? (x0 & 3) : 0;
        const float* tu = s_u + buf * TILE + du;
        const float* tb = s_b + buf * Smem2W::BSTRIDE + db;
        if (prolongs(sg)) {  // uniform per task
            const float* pe = s_e + buf * Smem2W::ESTRIDE;
            if (sg.pro_mode == 1)
                prolong_into_tile<true>(s_u + buf * TILE + du, pe, row0, col, lane, wi, x0, y0,
                                        mbk, hk, pmax);
            else
                prolong_into_tile<false>(s_u + buf * TILE + du, pe, row0, col, lane, wi, x0, y0,
                                         mbk, hk, pmax);
            __syncthreads();  // the residual reads the other threads' columns
        }

        f2 x[NP], r[NP], p[NP], q[NP];
        f2 acc0 = 0ull, acc1 = 0ull;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float rv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int ly = row0 + k + 8 * e, gy = y0 + ly;
                float v = rhs_zero ? 0.f : tb[ly * PB + col];
                if (!zero_in) {
                    const float* c0 = tu + (ly + 1) * P + col + 1;
                    const float dv = (float)((gy > 0) + (gy < h - 1));
                    v = res_stencil<false>(v, dh + dv, c0[0], c0[-P], c0[P], c0[-1], c0[1]);
                }
                rv[e] = v;
            }
            r[k] = mul2(pk(rv[0], rv[1]), keep[k]);
            p[k] = r[k];
            x[k] = 0ull;
            if (k & 1) acc1 = fma2(r[k], r[k], acc1);
            else acc0 = fma2(r[k], r[k], acc0);
        }
        acc0 = add2(acc0, acc1);
        s_seam[wi][lane] = wi == 0 ? hi2(r[NP - 1]) : lo2(r[0]);
        float part = warp_sum(lo2(acc0) + hi2(acc0));
        if (lane == 0) s_red2[wi] = part;
        __syncthreads();
        float rr = s_red2[0] + s_red2[1];
        float pb = s_seam[wi ^ 1][lane];
        const float rtol2 = sg.rtol2;
        const float rr_stop = rtol2 >= 0.f ? fmaxf(rtol2, 1e-14f) * rr
                                           : fmaxf(1e-14f * rr, -rtol2);
        const int iters = sg.iters;
        for (int it = 0; it < iters; ++it) {
            if (!(rr > rr_stop)) break;  // rr is identical in both warps
            const f2 pu = wi == 0 ? pk(0.f, lo2(p[NP - 1])) : pk(pb, lo2(p[NP - 1]));
            const f2 pd = wi == 0 ? pk(hi2(p[0]), pb) : pk(hi2(p[0]), 0.f);
            acc0 = 0ull;
            acc1 = 0ull;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const f2 left = __shfl_up_sync(kFull, p[k], 1);
                const f2 right = __shfl_down_sync(kFull, p[k], 1);
                const f2 up = k > 0 ? p[k - 1] : pu;
                const f2 dn = k < NP - 1 ? p[k + 1] : pd;
                f2 nbs = add2(up, dn);
                nbs = fma2(ml2, left, nbs);
                nbs = fma2(mr2, right, nbs);
                const f2 qk = mul2(fma2(ndg[k], p[k], nbs), keep[k]);
                q[k] = qk;
                if (k & 1) acc1 = fma2(p[k], qk, acc1);
                else acc0 = fma2(p[k], qk, acc0);
            }
            acc0 = add2(acc0, acc1);
            part = warp_sum(lo2(acc0) + hi2(acc0));
            if (lane == 0) s_red1[wi] = part;
            __syncthreads();
            const float pq = -(s_red1[0] + s_red1[1]);
            if (!(pq > 0.f) || pq == INFINITY) break;
            const float a = __fdividef(rr, pq);
            const f2 a2 = pk(a, a);
            acc0 = 0ull;
            acc1 = 0ull;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                x[k] = fma2(a2, p[k], x[k]);
                r[k] = fma2(a2, q[k], r[k]);
                if (k & 1) acc1 = fma2(r[k], r[k], acc1);
                else acc0 = fma2(r[k], r[k], acc0);
            }
            acc0 = add2(acc0, acc1);
            s_seam[wi][lane] = wi == 0 ? hi2(r[NP - 1]) : lo2(r[0]);
            part = warp_sum(lo2(acc0) + hi2(acc0));
            if (lane == 0) s_red2[wi] = part;
            __syncthreads();
            const float rrn = s_red2[0] + s_red2[1];
            const float beta = __fdividef(rrn, rr);
            rr = rrn;
            const f2 b2 = pk(beta, beta);
#pragma unroll
            for (int k = 0; k < NP; ++k) p[k] = fma2(b2, p[k], r[k]);
            pb = fmaf(beta, pb, s_seam[wi ^ 1][lane]);
        }

        // 0/1 weights: each pixel is written by the one block whose weight is
        // 1 there, with u_in added
        float* uo = static_cast<float*>(sg.out0) + cur.ch * n;
        if (x0 + col < w && wx > 0.f) {
            float* uol = uo + (size_t)(y0 + row0) * w + x0 + col;
            const float* tol = tu + (row0 + 1) * P + col + 1;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const int j = k + 8 * e;
                    if (!((rows_w >> (row0 + j)) & 1u)) continue;
                    const float v = e ? hi2(x[k]) : lo2(x[k]);
                    uol[(size_t)j * w] = (zero_in ? 0.f : tol[j * P]) + v;
                    vmax = fmaxf(vmax, fabsf(v));
                }
            }
        }
        if (!more) break;
        g = g2;
        cur = nxt;
        buf ^= 1;
    }
    if (vmax_slot) {
        vmax = warp_max(vmax);
        if (lane == 0 && vmax > 0.f) atomicMax(vmax_slot, __float_as_uint(vmax));
    }
    if (pmax_slot) {
        pmax = warp_max(pmax);
        if (lane == 0 && pmax > 0.f) atomicMax(pmax_slot, __float_as_uint(pmax));
    }
}

// Plan of every image of a batch: levels in use, the cascade's start level
// and the initial stop state (as k_plan for one image).
__global__ void k_batch_plan(int n, const int* __restrict__ Ls,
                             const unsigned long long* __restrict__ n0s, BatchState bs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int L = Ls[i];
    const unsigned long long* counts = bs.counts + (size_t)i * (kMaxLevels + 1);
    const unsigned long long unk0 = counts[1];
    int Leff = L;
    for (int l = 1; l < L; ++l)
        if (counts[1 + l] == 0) { Leff = l; break; }
    if (unk0 == 0) Leff = 0;
    StopState* st = bs.st + i;
    st->cycles = 0;
    st->converged = 0;
    st->levels_used = Leff;
    st->est = 0.f;
    st->prevU = -1.f;
    st->prevQ = -1.f;
    st->unknowns = unk0;
    for (int k = 0; k < kMaxChannels; ++k) st->rel[k] = -1.f;
    const bool empty = unk0 == n0s[i];
    st->status = empty ? DI_ERR_EMPTY_MASK : DI_OK;
    bs.leff[i] = empty ? 0 : Leff;
    bs.top[i] = empty ? -1 : (Leff == 0 ? 0 : (Leff == L ? L - 1 : Leff));
    bs.done[i] = (empty || Leff == 0) ? 1 : 0;
    if (!empty && Leff == 0) st->converged = 1;
    unsigned* upd = bs.upd + (size_t)i * (kMaxUpdSlots + 1);
    for (int k = 0; k <= kMaxUpdSlots; ++k) upd[k] = 0u;
}

// The stop test of every image still running (k_stop's rule per image); the
// loop continues while any image runs.
__global__ void k_batch_stop(int n, StopParams p, BatchState bs, cudaGraphConditionalHandle h) {
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    int running = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (bs.done[i]) continue;
        StopState* st = bs.st + i;
        unsigned* upd = bs.upd + (size_t)i * (kMaxUpdSlots + 1);
        const int cycles = st->cycles + 1;
        st->cycles = cycles;
        bool stop = false;
        if (upd[kMaxUpdSlots]) {
            st->status = DI_ERR_TIMEOUT;
            stop = true;
        } else if (p.rule == DI_STOP_ERROR_ESTIMATE) {
            float U = 0.f;
            for (int k = 0; k < p.nslots; ++k) U += __uint_as_float(upd[k]);
            float prevU = st->prevU, prevQ = st->prevQ, est;
            if (!isfinite(U)) {
                est = INFINITY;
                prevU = -1.f;
                prevQ = -1.f;
            } else if (prevU > 0.f) {
                const float qk = __fdiv_rn(U, prevU);
                const float q = prevQ > qk ? prevQ : qk;
                prevQ = qk;
                est = q < 1.f ? __fdiv_rn(__fmul_rn(U, q), __fsub_rn(1.f, q)) : INFINITY;
            } else {
                est = U;
            }
            prevU = U;
            if (U == 0.f) est = 0.f;
            st->prevU = prevU;
            st->prevQ = prevQ;
            st->est = est;
            if (cycles >= p.min_cycles && est <= 0.5f * bs.tol[i]) {
                st->converged = 1;
                stop = true;
            }
        } else if (cycles >= p.max_cycles) {  // fixed number of cycles
            st->converged = 1;
            stop = true;
        }
        if (!stop && cycles >= p.max_cycles) {
            st->status = DI_ERR_NOT_CONVERGED;
            stop = true;
        }
        for (int k = 0; k < p.nslots; ++k) upd[k] = 0u;
        if (stop) bs.done[i] = 1;
        else running = 1;
    }
    if (running) atomicOr(&s_any, 1);
    __syncthreads();
    if (threadIdx.x == 0) cudaGraphSetConditional(h, s_any ? 1u : 0u);
}

// Timing event on s; inside a stream capture it becomes an event record node
// of the graph (recorded by every replay).
void record_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

inline dim3 grid2(int w, int h, dim3 blk, int z = 1) {
    return dim3((unsigned)((w + blk.x - 1) / blk.x), (unsigned)((h + blk.y - 1) / blk.y),
                (unsigned)z);
}

cudaError_t launch_combine(float* planes, int w, int h, int C, int B, int o, int nbx, int nby,
                           float* u_out, cudaStream_t s, int stor);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of an FP32 [C][h][w] image with a (bw x bh x 1) box; false if
// the image does not meet TMA's rules (w a multiple of 4, 16-byte base).
bool make_map(CUtensorMap* m, const float* base, int w, int h, int C, int bw, int bh) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || !base || w % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)C};
    const cuuint64_t strides[2] = {(cuuint64_t)w * 4, (cuuint64_t)w * h * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Resident CTAs per SM of a kernel at a shared-memory size, and the SM count,
// cached per (device, kernel, shared-memory size): a process may drive
// several GPUs.
int cached_occupancy(const void* kern, int threads, size_t smem, size_t smem_max, int* nsm_out) {
    static std::mutex occ_mu;
    constexpr int kSlots = 64;
    static int occ_dev[kSlots];
    static const void* occ_fn[kSlots] = {};
    static size_t occ_key[kSlots] = {};
    static int occ_val[kSlots] = {};
    static int occ_nsm[kSlots] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> occ_lock(occ_mu);
    for (int i = 0; i < kSlots; ++i)
        if (occ_fn[i] == kern && occ_key[i] == smem && occ_dev[i] == dev) {
            *nsm_out = occ_nsm[i];
            return occ_val[i];
        }
    int nsm = 0, oc = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, kern, threads, smem);
    if (oc < 1) oc = 1;
    if (nsm < 1) nsm = 1;
    for (int i = 0; i < kSlots; ++i)
        if (occ_fn[i] == nullptr) {
            occ_fn[i] = kern;
            occ_key[i] = smem;
            occ_dev[i] = dev;
            occ_val[i] = oc;
            occ_nsm[i] = nsm;
            break;
        }
    *nsm_out = nsm;
    return oc;
}

// The 16-bit block kernel for iterate type H and storage TU.
template <class H, class TU, bool F64>
void run_oras_2w_h(int grid, size_t smem, cudaStream_t s, const float* u_in, int zero_in,
                   const float* rhs, int rhs_zero, const uint32_t* mbits, int wpr, int w, int h,
                   int C, int o, int nbx, int nby, float alpha, int iters, float rtol2,
                   float* u_out, float* planes, unsigned* maxupd, int chan_inner,
                   unsigned long long* step_count) {
    k_oras_2w_h<H, TU, F64><<<grid, 64, smem, s>>>(
        reinterpret_cast<const TU*>(u_in), zero_in, reinterpret_cast<const TU*>(rhs), rhs_zero,
        mbits, wpr, w, h, C, o, nbx, nby, alpha, iters, rtol2, reinterpret_cast<TU*>(u_out),
        planes, maxupd, chan_inner, step_count);
}

template <class H, class TU, bool F64>
const void* oras_2w_h_fn() {
    return (const void*)k_oras_2w_h<H, TU, F64>;
}

// precision: 0 FP32 iterates (tiles by TMA where the image allows it), 1 FP16,
// 2 BF16 iterates; stor: storage of u_in, rhs, u_out (kF32, or the iterate
// type on the coarse levels of the 16-bit modes); f64: FP64 block residual.
// pro_e: coarser level's correction (pro_mode 1) or solution (pro_mode 0)
// prolonged into the iteration's start (FP32 only; see k_oras_2w), largest
// |P e| of mode 1 into *pro_max.
cudaError_t launch_oras_2w(const float* u_in, int zero_in, const float* rhs, int rhs_zero,
                           const uint32_t* mbits, int wpr, int w, int h, int C, int o, float alpha,
                           int iters, float rtol2, float* u_out, float* planes, unsigned* maxupd,
                           cudaStream_t s, cudaEvent_t* ev, int precision, unsigned* errflag,
                           unsigned long long* step_count, int stor, bool f64,
                           const float* pro_e, unsigned* pro_max, int pro_mode) {
    constexpr int B = 32;
    if (stor != kF32 && stor != precision) return cudaErrorInvalidValue;
    if (pro_e && (!prolong_fusable(precision, o, zero_in) || (pro_mode != 0 && pro_mode != 1)))
        return cudaErrorInvalidValue;
    const int pm = pro_e ? (pro_mode == 1 ? 1 : 2) : 0;  // the kernel's PRO
    int wH = 0, hH = 0;
    coarse_dims(w, h, &wH, &hH);
    const int nbx = axis_blocks(w, B, o), nby = axis_blocks(h, B, o);
    const int ntasks = nbx * nby * C;
    const int nblk = nbx * nby;
    int nsm = 0, oc = 0;
    size_t smem = 0;
    const void* kern = nullptr;
    CUtensorMap tm_u, tm_b, tm_e;
    std::memset(&tm_u, 0, sizeof tm_u);
    std::memset(&tm_b, 0, sizeof tm_b);
    std::memset(&tm_e, 0, sizeof tm_e);
    int use_tma = 0, use_tma_e = 0;
    if (precision == 0) {
        use_tma = (!zero_in || !rhs_zero) &&
                  (zero_in || make_map(&tm_u, u_in, w, h, C, Smem2W::PU, Smem2W::TH)) &&
                  (rhs_zero || make_map(&tm_b, rhs, w, h, C, Smem2W::PB, B));
        use_tma_e = use_tma && pm != 0 &&
                    make_map(&tm_e, pro_e, wH, hH, C, Smem2W::EPW, Smem2W::EH);
        smem = Smem2W::bytes(!rhs_zero, pm != 0);
        kern = pm == 1 ? (f64 ? (const void*)k_oras_2w<true, 1> : (const void*)k_oras_2w<false, 1>)
               : pm == 2 ? (f64 ? (const void*)k_oras_2w<true, 2> : (const void*)k_oras_2w<false, 2>)
                         : (f64 ? (const void*)k_oras_2w<true, 0> : (const void*)k_oras_2w<false, 0>);
        oc = cached_occupancy(kern, 64, smem, Smem2W::bytes(true, pm != 0), &nsm);
    } else {
        smem = ((size_t)Tile2W::FIXED + (rhs_zero ? 0 : (size_t)2 * B * B)) * sizeof(float);
        if (precision == 1)
            kern = stor != kF32 ? oras_2w_h_fn<HalfT, __half, false>()
                   : f64        ? oras_2w_h_fn<HalfT, float, true>()
                                : oras_2w_h_fn<HalfT, float, false>();
        else
            kern = stor != kF32 ? oras_2w_h_fn<Bf16T, __nv_bfloat16, false>()
                   : f64        ? oras_2w_h_fn<Bf16T, float, true>()
                                : oras_2w_h_fn<Bf16T, float, false>();
        oc = cached_occupancy(kern, 64, smem, ((size_t)Tile2W::FIXED + (size_t)2 * B * B) *
                                                  sizeof(float), &nsm);
    }
    const int slots = nsm * oc;
    const int chan_inner = nblk >= slots ? 1 : 0;
    int grid = chan_inner ? slots : (ntasks < slots ? ntasks : slots);
    if (grid < 1) grid = 1;
    if (ev) record_event(ev[0], s);
    if (precision == 0) {
#define DI_ORAS_F(F, PR)                                                                         \
    k_oras_2w<F, PR><<<grid, 64, smem, s>>>(u_in, zero_in, rhs, rhs_zero, mbits, wpr, w, h, C, o, \
                                            nbx, nby, alpha, iters, rtol2, u_out, planes, maxupd, \
                                            chan_inner, tm_u, tm_b, use_tma, errflag, step_count, \
                                            pro_e, wH, hH, pro_max, tm_e, use_tma_e)
        if (pm == 1) {
            if (f64) DI_ORAS_F(true, 1);
            else DI_ORAS_F(false, 1);
        } else if (pm == 2) {
            if (f64) DI_ORAS_F(true, 2);
            else DI_ORAS_F(false, 2);
        } else {
            if (f64) DI_ORAS_F(true, 0);
            else DI_ORAS_F(false, 0);
        }
#undef DI_ORAS_F
    } else {
#define DI_ORAS_H(H, TU, F)                                                                     \
    run_oras_2w_h<H, TU, F>(grid, smem, s, u_in, zero_in, rhs, rhs_zero, mbits, wpr, w, h, C, o, \
                            nbx, nby, alpha, iters, rtol2, u_out, planes, maxupd, chan_inner,   \
                            step_count)
        if (precision == 1) {
            if (stor != kF32) DI_ORAS_H(HalfT, __half, false);
            else if (f64) DI_ORAS_H(HalfT, float, true);
            else DI_ORAS_H(HalfT, float, false);
        } else {
            if (stor != kF32) DI_ORAS_H(Bf16T, __nv_bfloat16, false);
            else if (f64) DI_ORAS_H(Bf16T, float, true);
            else DI_ORAS_H(Bf16T, float, false);
        }
#undef DI_ORAS_H
    }
    count();
    if (ev) record_event(ev[1], s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_combine(planes, w, h, C, B, o, nbx, nby, u_out, s, stor);
}

template <int B>
cudaError_t launch_oras_t(const float* u_in, int zero_in, const float* rhs, int rhs_zero,
                          const uint32_t* mbits, int wpr, int w, int h, int C, int o, float alpha,
                          int iters, float rtol2, float* u_out, float* planes, unsigned* maxupd,
                          cudaStream_t s, cudaEvent_t* ev,
                          unsigned long long* step_count) {
    const int nbx = axis_blocks(w, B, o), nby = axis_blocks(h, B, o);
    const int ntasks = nbx * nby * C;
    constexpr int FIXED = WarpTile<B>::FIXED;
    const size_t smem = (size_t)FIXED * sizeof(float) +
                        (rhs_zero ? 0 : (size_t)2 * B * B * sizeof(float));
    // persistent warps: as many as fit on the GPU at once
    int nsm = 0;
    const int oc = cached_occupancy((const void*)k_oras_warp<B>, 32, smem,
                                    FIXED * sizeof(float) + 2 * B * B * sizeof(float), &nsm);
    const int slots = nsm * oc;
    const int nblk = nbx * nby;
    const int chan_inner = nblk >= slots ? 1 : 0;
    int grid = chan_inner ? slots : (ntasks < slots ? ntasks : slots);
    if (grid < 1) grid = 1;
    if (ev) record_event(ev[0], s);
    k_oras_warp<B><<<grid, 32, smem, s>>>(u_in, zero_in, rhs, rhs_zero, mbits, wpr, w, h, C, o,
                                          nbx, nby, alpha, iters, rtol2, u_out, planes, maxupd,
                                          chan_inner, step_count);
    count();
    if (ev) record_event(ev[1], s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_combine(planes, w, h, C, B, o, nbx, nby, u_out, s, kF32);
}

template <class TU>
cudaError_t launch_combine_t(float* planes, int w, int h, int C, int B, int o, int nbx, int nby,
                             TU* u_out, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    // Overlap 2 gives 0/1 weights: no pixel is shared, the combine is empty.
    const int nsh = shared_per_seam(o);
    const int sb = B - o;
    const float inv_s = 1.f / (float)sb;
    if (nsh > 0 && nby > 1) {
        dim3 grid_r((unsigned)((w + 255) / 256), (unsigned)((nby - 1) * nsh), (unsigned)C);
        k_combine_rows<TU><<<grid_r, 256, 0, s>>>(planes, w, h, sb, o, nbx, nby, inv_s, u_out);
        count();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int nseams = nbx - 1;
    if (nsh > 0 && nbx > 1 && nseams > 0) {
        const int rows = 256 / nsh > 0 ? 256 / nsh : 1;
        dim3 blk_c((unsigned)nsh, (unsigned)rows);
        dim3 grid_c((unsigned)((h + rows - 1) / rows), (unsigned)nseams, (unsigned)C);
        k_combine_cols<TU><<<grid_c, blk_c, 0, s>>>(planes, w, h, sb, o, nbx, nby, inv_s, u_out);
        count();
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_combine(float* planes, int w, int h, int C, int B, int o, int nbx, int nby,
                           float* u_out, cudaStream_t s, int stor) {
    if (stor == kF16)
        return launch_combine_t(planes, w, h, C, B, o, nbx, nby, reinterpret_cast<__half*>(u_out), s);
    if (stor == kBF16)
        return launch_combine_t(planes, w, h, C, B, o, nbx, nby,
                                reinterpret_cast<__nv_bfloat16*>(u_out), s);
    return launch_combine_t(planes, w, h, C, B, o, nbx, nby, u_out, s);
}

}  // namespace

bool make_tile_maps(void* out, const float* u_in, int zero_in, const float* rhs, int rhs_zero,
                    int w, int h, int C) {
    CUtensorMap* m = static_cast<CUtensorMap*>(out);
    std::memset(m, 0, 2 * sizeof(CUtensorMap));
    static_assert(2 * sizeof(CUtensorMap) == kTileMapsBytes, "two tensor maps");
    return (zero_in || make_map(&m[0], u_in, w, h, C, Smem2W::PU, Smem2W::TH)) &&
           (rhs_zero || make_map(&m[1], rhs, w, h, C, Smem2W::PB, 32));
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------

cudaError_t launch_mask_down(const uint8_t* c, int w, int h, uint8_t* cH, cudaStream_t s) {
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    dim3 blk(32, 8);
    k_mask_down<<<grid2(wH, hH, blk), blk, 0, s>>>(c, w, h, cH, wH, hH);
    count();
    return cudaGetLastError();
}

cudaError_t launch_values_down(const uint8_t* c, const float* b, int w, int h, int C,
                               const uint8_t* cH, float* bH, int modified, cudaStream_t s) {
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    dim3 blk(32, 8);
    k_values_down<<<grid2(wH, hH, blk), blk, 0, s>>>(c, b, w, h, C, cH, bH, wH, hH, modified);
    count();
    return cudaGetLastError();
}

size_t residual_partials_per_channel(int w, int h) {
    return (size_t)((w + kResBX - 1) / kResBX) * (size_t)((h + kResBY - 1) / kResBY);
}

cudaError_t launch_residual(const float* u, int zero_u, const float* b, int rhs_zero,
                            const uint8_t* c, int w, int h, int C, float* r, double* partials,
                            int* nparts, cudaStream_t s, bool f64) {
    dim3 blk(kResBX, kResBY);
    dim3 grid = grid2(w, h, blk, C);
    *nparts = (int)(grid.x * grid.y);
    if (f64)
        k_residual<true><<<grid, blk, 0, s>>>(u, zero_u, b, rhs_zero, c, w, h, r, partials);
    else
        k_residual<false><<<grid, blk, 0, s>>>(u, zero_u, b, rhs_zero, c, w, h, r, partials);
    count();
    return cudaGetLastError();
}

// Fixed reduction scratch for callers that cannot allocate (see
// di_residual_norm_noalloc in di.h).  Host code must not pass the symbol
// itself to a kernel: on the host it names a stand-in, not device memory.
// Its device address is looked up once per device and context, with that
// device current: a context that is destroyed and created again (a device
// reset) loads the module anew, so the address is keyed on the context's
// process-unique id, not on the device ordinal alone.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Process-unique id of the calling thread's current context (0 if none).
unsigned long long current_context_id() {
    static std::once_flag once;
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

cudaError_t launch_residual_noalloc(const float* u, const float* b, int rhs_zero,
                                    const uint8_t* c, int w, int h, int C, float* r,
                                    double* norm2, cudaStream_t s) {
    static std::mutex mu;
    static double* addr[128] = {};
    static unsigned long long addr_ctx[128] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    double* scratch;
    {
        std::lock_guard<std::mutex> lock(mu);
        unsigned long long id = current_context_id();
        if (!addr[dev] || id == 0 || id != addr_ctx[dev]) {
            // first call on this device, or its context changed: (re)load
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess) return e;
            addr[dev] = static_cast<double*>(p);
            // the lookup makes the primary context current if none was
            if (id == 0) id = current_context_id();
            addr_ctx[dev] = id;
        }
        scratch = addr[dev];
    }
    int nparts = 0;
    e = launch_residual(u, 0, b, rhs_zero, c, w, h, C, r, scratch, &nparts, s);
    if (e != cudaSuccess) return e;
    return launch_reduce_partials(scratch, nparts, C, norm2, s);
}

cudaError_t launch_reduce_partials(const double* partials, int nparts, int C, double* out,
                                   cudaStream_t s) {
    k_reduce<<<C, 256, 0, s>>>(partials, nparts, out);
    count();
    return cudaGetLastError();
}

template <class TU, class TB, class TO, bool F64>
void run_restrict(dim3 grid, dim3 blk, cudaStream_t s, const float* u, const float* b,
                  int rhs_zero, int w, int h, const uint8_t* cH, float* rH, int wH, int hH) {
    k_restrict<false, TU, TB, TO, F64><<<grid, blk, 0, s>>>(
        reinterpret_cast<const TU*>(u), reinterpret_cast<const TB*>(b), rhs_zero, w, h, cH,
        reinterpret_cast<TO*>(rH), wH, hH);
}

cudaError_t launch_restrict(const float* u, const float* b, int rhs_zero, const uint8_t* c,
                            int w, int h, int C, const uint8_t* cH, float* rH, cudaStream_t s,
                            int su, int sb, int sr, bool f64) {
    (void)c;  // children of an unmasked coarse cell are unknown by construction
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    dim3 blk(32, 8);
    const dim3 grid = grid2(wH, hH, blk, C);
    if (rhs_zero) sb = kF32;  // b is not read
    const bool vec = su == kF32 && sb == kF32 && (w % 2 == 0) &&
                     ((reinterpret_cast<uintptr_t>(u) |
                       reinterpret_cast<uintptr_t>(rhs_zero ? nullptr : b)) % 8 == 0);
    if (su == kF32 && sb == kF32 && sr == kF32) {
        if (vec && f64)
            k_restrict<true, float, float, float, true><<<grid, blk, 0, s>>>(
                u, b, rhs_zero, w, h, cH, rH, wH, hH);
        else if (vec)
            k_restrict<true, float, float, float, false><<<grid, blk, 0, s>>>(
                u, b, rhs_zero, w, h, cH, rH, wH, hH);
        else if (f64)
            run_restrict<float, float, float, true>(grid, blk, s, u, b, rhs_zero, w, h, cH, rH, wH, hH);
        else
            run_restrict<float, float, float, false>(grid, blk, s, u, b, rhs_zero, w, h, cH, rH, wH,
                                                     hH);
    } else if (su == kF32 && sb == kF32 && sr == kF16) {  // finest level, FP16 coarse levels
        if (vec && f64)
            k_restrict<true, float, float, __half, true><<<grid, blk, 0, s>>>(
                u, b, rhs_zero, w, h, cH, reinterpret_cast<__half*>(rH), wH, hH);
        else if (vec)
            k_restrict<true, float, float, __half, false><<<grid, blk, 0, s>>>(
                u, b, rhs_zero, w, h, cH, reinterpret_cast<__half*>(rH), wH, hH);
        else if (f64)
            run_restrict<float, float, __half, true>(grid, blk, s, u, b, rhs_zero, w, h, cH, rH, wH, hH);
        else
            run_restrict<float, float, __half, false>(grid, blk, s, u, b, rhs_zero, w, h, cH, rH, wH,
                                                      hH);
    } else if (su == kF32 && sb == kF32 && sr == kBF16) {
        if (vec && f64)
            k_restrict<true, float, float, __nv_bfloat16, true><<<grid, blk, 0, s>>>(
                u, b, rhs_zero, w, h, cH, reinterpret_cast<__nv_bfloat16*>(rH), wH, hH);
        else if (vec)
            k_restrict<true, float, float, __nv_bfloat16, false><<<grid, blk, 0, s>>>(
                u, b, rhs_zero, w, h, cH, reinterpret_cast<__nv_bfloat16*>(rH), wH, hH);
        else if (f64)
            run_restrict<float, float, __nv_bfloat16, true>(grid, blk, s, u, b, rhs_zero, w, h, cH,
                                                            rH, wH, hH);
        else
            run_restrict<float, float, __nv_bfloat16, false>(grid, blk, s, u, b, rhs_zero, w, h, cH,
                                                             rH, wH, hH);
    } else if (su == kF16 && (sb == kF16 || rhs_zero) && sr == kF16) {  // coarse levels
        run_restrict<__half, __half, __half, false>(grid, blk, s, u, b, rhs_zero, w, h, cH, rH, wH,
                                                    hH);
    } else if (su == kBF16 && (sb == kBF16 || rhs_zero) && sr == kBF16) {
        run_restrict<__nv_bfloat16, __nv_bfloat16, __nv_bfloat16, false>(grid, blk, s, u, b,
                                                                         rhs_zero, w, h, cH, rH,
                                                                         wH, hH);
    } else {
        return cudaErrorInvalidValue;
    }
    count();
    return cudaGetLastError();
}

template <bool VEC, class TC, class TF>
void run_prolong(dim3 grid, dim3 blk, cudaStream_t s, const float* uH, int wH, int hH,
                 const float* b, const uint8_t* c, int w, int h, float* u, int mode,
                 unsigned* maxupd) {
    k_prolong<VEC, TC, TF><<<grid, blk, 0, s>>>(reinterpret_cast<const TC*>(uH), wH, hH, b, c, w,
                                                h, reinterpret_cast<TF*>(u), mode, maxupd);
}

cudaError_t launch_prolong(const float* uH, const float* b, const uint8_t* c, int w, int h,
                           int C, float* u, int mode, unsigned* maxupd, cudaStream_t s, int suH,
                           int su) {
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    dim3 blk(32, 8);
    const dim3 grid = grid2(wH, hH, blk, C);  // one thread per coarse cell
    const bool vec = su == kF32 && (w % 2 == 0) &&
                     ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(b)) % 8 == 0) &&
                     reinterpret_cast<uintptr_t>(c) % 2 == 0;
    unsigned* mu = mode == 1 ? maxupd : nullptr;
    if (su == kF32) {
        if (suH == kF32) {
            if (vec) run_prolong<true, float, float>(grid, blk, s, uH, wH, hH, b, c, w, h, u, mode, mu);
            else run_prolong<false, float, float>(grid, blk, s, uH, wH, hH, b, c, w, h, u, mode, mu);
        } else if (suH == kF16) {
            if (vec) run_prolong<true, __half, float>(grid, blk, s, uH, wH, hH, b, c, w, h, u, mode, mu);
            else run_prolong<false, __half, float>(grid, blk, s, uH, wH, hH, b, c, w, h, u, mode, mu);
        } else {
            if (vec)
                run_prolong<true, __nv_bfloat16, float>(grid, blk, s, uH, wH, hH, b, c, w, h, u,
                                                        mode, mu);
            else
                run_prolong<false, __nv_bfloat16, float>(grid, blk, s, uH, wH, hH, b, c, w, h, u,
                                                         mode, mu);
        }
    } else if (su == kF16 && suH == kF16) {
        run_prolong<false, __half, __half>(grid, blk, s, uH, wH, hH, b, c, w, h, u, mode, mu);
    } else if (su == kBF16 && suH == kBF16) {
        run_prolong<false, __nv_bfloat16, __nv_bfloat16>(grid, blk, s, uH, wH, hH, b, c, w, h, u,
                                                         mode, mu);
    } else {
        return cudaErrorInvalidValue;
    }
    count();
    return cudaGetLastError();
}

cudaError_t launch_select(const float* b, const uint8_t* c, int w, int h, int C, float* u,
                          cudaStream_t s, int keep, int su) {
    const size_t n = (size_t)w * h;
    size_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    const dim3 grid((unsigned)blocks, (unsigned)C);
    if (su == kF16)
        k_select<__half><<<grid, 256, 0, s>>>(b, c, n, reinterpret_cast<__half*>(u), keep);
    else if (su == kBF16)
        k_select<__nv_bfloat16><<<grid, 256, 0, s>>>(b, c, n, reinterpret_cast<__nv_bfloat16*>(u),
                                                     keep);
    else
        k_select<float><<<grid, 256, 0, s>>>(b, c, n, u, keep);
    count();
    return cudaGetLastError();
}

// Global CG smoother on one level: `steps` CG steps on A x = b - A in (known
// pixels fixed), out = in + x.  With restart == 0 the state in (r, p, sc) of
// the previous call on the same level continues (single-level CG).
cudaError_t launch_cg_smooth(const float* in, int zero_in, const float* b, int rhs_zero,
                             const uint8_t* c, int w, int h, int C, int steps, int restart,
                             float* r, float* p, float* q, float* x, double* partials, double* sc,
                             int* step_par, float* out, unsigned* maxupd, cudaStream_t s) {
    CgTiles g;
    g.w = w;
    g.h = h;
    g.tiles_x = (w + kCgBX - 1) / kCgBX;
    g.ntiles = g.tiles_x * ((h + kCgBY - 1) / kCgBY);
    int per_ch = kCgCtas / C;
    if (per_ch > g.ntiles) per_ch = g.ntiles;
    if (per_ch < 1) per_ch = 1;
    const dim3 grid((unsigned)per_ch, (unsigned)C), blk(kCgBX, kCgBY);
    const size_t n = (size_t)w * h;
    size_t nb = (n + 255) / 256;
    if (nb > 8192) nb = 8192;
    cudaError_t e;
    if (restart) {
        k_cg_init<<<grid, blk, 0, s>>>(g, in, zero_in, b, rhs_zero, c, r, p, x, partials);
        count();
        k_reduce_slot<<<C, 256, 0, s>>>(partials, per_ch, sc, 0);
        count();
        *step_par = 0;
    } else {
        // continue: the correction restarts from zero on top of the new iterate
        e = cudaMemsetAsync(x, 0, n * C * sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    for (int k = 0; k < steps; ++k) {
        const int par = *step_par;
        k_cg_matvec<<<grid, blk, 0, s>>>(g, p, c, q, partials);
        count();
        k_reduce_slot<<<C, 256, 0, s>>>(partials, per_ch, sc, 2);
        count();
        k_cg_update<<<grid, blk, 0, s>>>(g, p, q, x, r, sc, par, partials);
        count();
        k_reduce_slot<<<C, 256, 0, s>>>(partials, per_ch, sc, par ^ 1);
        count();
        k_cg_direction<<<dim3((unsigned)nb, (unsigned)C), 256, 0, s>>>(p, r, n, sc, par);
        count();
        *step_par = par ^ 1;
    }
    k_cg_finish<<<dim3((unsigned)nb, (unsigned)C), 256, 0, s>>>(in, zero_in, x, out, n, maxupd);
    count();
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned* flag, int limit, cudaStream_t s) {
    k_bounded_wait_selftest<<<1, 64, 0, s>>>(flag, limit);
    count();
    return cudaGetLastError();
}

cudaError_t launch_pack_mask(const uint8_t* c, int w, int h, uint32_t* bits,
                             unsigned long long* unknown, cudaStream_t s) {
    const int wpr = mask_words_per_row(w);
    const long long words = (long long)h * wpr;
    if (words > 0x7fffffffLL) return cudaErrorInvalidValue;
    long long blocks = (words + 31) / 32;  // 8 warps x 4 words per CTA pass
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_pack_mask<<<(unsigned)blocks, 256, 0, s>>>(c, w, h, bits, wpr, unknown);
    count();
    return cudaGetLastError();
}

cudaError_t launch_oras(const float* u_in, int zero_in, const float* rhs, int rhs_zero,
                        const uint32_t* mbits, int w, int h, int C, int B, int o, float alpha,
                        int iters, float rtol2, float* u_out, float* planes, unsigned* maxupd,
                        cudaStream_t s, cudaEvent_t* ev, int precision, unsigned* errflag,
                        unsigned long long* step_count, int stor, bool f64, const float* pro_e,
                        unsigned* pro_max, int pro_mode) {
    const int wpr = mask_words_per_row(w);
    if (B != 32 && (stor != kF32 || f64 || pro_e)) return cudaErrorInvalidValue;
    switch (B) {
        case 32:
            return launch_oras_2w(u_in, zero_in, rhs, rhs_zero, mbits, wpr, w, h, C, o, alpha,
                                  iters, rtol2, u_out, planes, maxupd, s, ev, precision, errflag,
                                  step_count, stor, f64, pro_e, pro_max, pro_mode);
        case 16:
            return launch_oras_t<16>(u_in, zero_in, rhs, rhs_zero, mbits, wpr, w, h, C, o, alpha,
                                     iters, rtol2, u_out, planes, maxupd, s, ev, step_count);
        case 8:
            return launch_oras_t<8>(u_in, zero_in, rhs, rhs_zero, mbits, wpr, w, h, C, o, alpha,
                                    iters, rtol2, u_out, planes, maxupd, s, ev, step_count);
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_plan(const unsigned long long* counts, StopState* st, const PlanParams& p,
                        cudaStream_t s) {
    k_plan<<<1, 32, 0, s>>>(counts, st, p);
    count();
    return cudaGetLastError();
}

cudaError_t launch_stop(unsigned* upd, StopState* st, const StopParams& p,
                        unsigned long long h_loop, cudaStream_t s) {
    k_stop<<<1, 32, 0, s>>>(upd, st, p, (cudaGraphConditionalHandle)h_loop);
    count();
    return cudaGetLastError();
}

void batch_grid_dims(int kind, int w, int h, int* gx, int* gy) {
    if (kind == kBPack) {  // persistent warps over the packed words
        const long long words = (long long)h * mask_words_per_row(w);
        long long b = (words + 31) / 32;
        if (b > 152) b = 152;
        *gx = (int)(b < 1 ? 1 : b);
        *gy = 1;
    } else if (kind == kBSelect) {
        size_t b = ((size_t)w * h + 255) / 256;
        if (b > 1024) b = 1024;
        *gx = (int)(b < 1 ? 1 : b);
        *gy = 1;
    } else if (kind == kBRestrict || kind == kBProlong || kind == kBMaskDown ||
               kind == kBValuesDown || kind == kBPyramid) {  // a coarse cell per thread, 32 x 8 per CTA
        const int wH = (w + 1) / 2, hH = (h + 1) / 2;
        *gx = (wH + 31) / 32;
        *gy = (hH + 7) / 8;
    } else {
        *gx = *gy = 1;
    }
}

cudaError_t launch_batch_grid(int kind, const BatchSeg* segs, int nseg, int nctas,
                              const BatchState& bs, cudaStream_t s) {
    if (nctas < 1 || nseg < 1) return cudaSuccess;
    const dim3 blk2(32, 8), blk1(256);
    switch (kind) {
        case kBMaskDown: k_batch_grid<kBMaskDown><<<nctas, blk2, 0, s>>>(segs, nseg, bs); break;
        case kBValuesDown: k_batch_grid<kBValuesDown><<<nctas, blk2, 0, s>>>(segs, nseg, bs); break;
        case kBPack: k_batch_grid<kBPack><<<nctas, blk1, 0, s>>>(segs, nseg, bs); break;
        case kBSelect: k_batch_grid<kBSelect><<<nctas, blk1, 0, s>>>(segs, nseg, bs); break;
        case kBRestrict: k_batch_grid<kBRestrict><<<nctas, blk2, 0, s>>>(segs, nseg, bs); break;
        case kBProlong: k_batch_grid<kBProlong><<<nctas, blk2, 0, s>>>(segs, nseg, bs); break;
        case kBPyramid: k_batch_grid<kBPyramid><<<nctas, blk2, 0, s>>>(segs, nseg, bs); break;
        default: return cudaErrorInvalidValue;
    }
    count();
    return cudaGetLastError();
}

cudaError_t launch_batch_oras(const BatchSeg* segs, int nseg, int nunits, int o, float alpha,
                              const BatchState& bs, cudaStream_t s) {
    if (nunits < 1 || nseg < 1) return cudaSuccess;
    if (shared_per_seam(o) != 0) return cudaErrorInvalidValue;  // 0/1 weights only
    int nsm = 0;
    const size_t smem = Smem2W::bytes(true, true);
    const int oc = cached_occupancy((const void*)k_batch_oras, 64, smem, smem, &nsm);
    int grid = nsm * oc;
    if (grid > nunits) grid = nunits;
    k_batch_oras<<<grid, 64, smem, s>>>(segs, nseg, nunits, o, alpha, bs);
    count();
    return cudaGetLastError();
}

cudaError_t launch_batch_plan(int n, const int* L, const unsigned long long* n0,
                              const BatchState& bs, cudaStream_t s) {
    k_batch_plan<<<(n + 127) / 128, 128, 0, s>>>(n, L, n0, bs);
    count();
    return cudaGetLastError();
}

cudaError_t launch_batch_stop(int n, const StopParams& p, const BatchState& bs,
                              unsigned long long h_loop, cudaStream_t s) {
    k_batch_stop<<<1, 256, 0, s>>>(n, p, bs, (cudaGraphConditionalHandle)h_loop);
    count();
    return cudaGetLastError();
}

cudaError_t launch_pyramid_level(const uint8_t* c, const float* b, int w, int h, int C,
                                 uint8_t* cH, float* bH, int modified, int values, uint32_t* bits,
                                 unsigned long long* unknown, cudaStream_t s) {
    int wH, hH;
    coarse_dims(w, h, &wH, &hH);
    const int wpr = mask_words_per_row(wH);
    // one CTA column per packed word of a coarse row but the padding word
    const dim3 grid((unsigned)(wpr - 1), (unsigned)((hH + 7) / 8));
    k_pyramid_level<<<grid, dim3(32, 8), 0, s>>>(c, b, w, h, C, cH, bH, wH, hH, modified, values,
                                                 bits, wpr, unknown);
    count();
    return cudaGetLastError();
}

}  // namespace di

// Host side of the decoder: context and device workspace, the reduced-FMG /
// V-cycle scheduler (Sections 4.2 and 4.4) and the C ABI declared in di.h.
//
// Schedule of di_inpaint for an image with L levels (level 0 finest; the
// coarsest fits one B x B block, Section 4.4):
//   1. mask pyramid c_l (max pooling) with unknown-pixel counts per level, and
//      the value pyramid b_l (modified downsampling), Section 4.3;
//   2. the cascade (one-way multigrid, Section 4.2 "reduced FMG"): on the
//      coarsest level u = b on the mask, 0 elsewhere, then one ORAS iteration
//      (one block: a local solve of the whole level); on each finer level
//      u = P u_coarse with u = b on the mask, then one ORAS iteration;
//   3. V(pre, post)-cycles on the finest level (Algorithm 3 applied
//      recursively), each followed by the stop test.
// A level whose mask covers every pixel has an identically zero correction,
// so recursion stops above the first such level and the cascade starts from
// it (u = b there); this changes no arithmetic result.
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <new>

#include "../../include/di.h"
#include "di_internal.h"

using namespace di;

namespace {

struct Level {
    int w = 0, h = 0;
    size_t n = 0;
    const uint8_t* c = nullptr;  // level 0: caller's mask
    const float* b = nullptr;    // mask values (level 0: caller's f, read only on the mask)
    float* u[2] = {nullptr, nullptr};
    float* r = nullptr;          // restricted residual (right-hand side of the error equation)
    uint32_t* mbits = nullptr;   // bit-packed mask for the block solver
    long long unknowns = 0;
};

// One whole decode as a CUDA graph (pyramid, plan, cascade, V-cycle loop with
// the stop test), valid for the buffers and sizes it was captured for.  The
// number of levels in use, which depends on the mask, selects a body of the
// graph on the device, so the graph needs no host round trip.  Kernel counts
// per body feed the launch counter.
struct DecodeGraph {
    bool valid = false;
    const float* f = nullptr;
    const uint8_t* c = nullptr;
    float* u = nullptr;
    int w = 0, h = 0, C = 0;
    float tol = 0.f;
    unsigned long long ws_gen = 0;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long k_pre = 0;                    // kernels outside the switch bodies
    long long k_sel[kMaxLevels + 1] = {};   // kernels of switch body v outside its loop
    long long k_cycle[kMaxLevels + 1] = {}; // kernels of one cycle of body v
    unsigned long long used = 0;
};

}  // namespace

struct di_ctx {
    di_config cfg;
    int device = 0;
    // workspace capacity
    int cap_w = 0, cap_h = 0, cap_c = 0;
    void* pool = nullptr;           // one allocation for every level buffer
    float* planes = nullptr;        // 4 * C * n0 floats
    double* partials = nullptr;     // residual norm partial sums
    size_t partials_cap = 0;
    double* norm2 = nullptr;        // [kMaxChannels]
    unsigned long long* counts = nullptr;  // [kMaxLevels + 1]
    unsigned* upd = nullptr;        // [kMaxUpdSlots] per-cycle max update (float bits)
    void* host = nullptr;           // pinned staging for small device->host reads
    Level lv[kMaxLevels];
    int L = 0;
    di_stats stats;
    char err[256];
    // profiling (cfg.profile): event pairs around finest-level ORAS launches
    static constexpr int kEvPairs = 64;
    cudaEvent_t ev[kEvPairs][2] = {};
    bool ev_made = false;
    int ev_used = 0;
    di_profile prof = {};
    long long launch_base = 0;
    // global-CG smoother state (cfg.smoother == DI_SMOOTH_CG): r, p, q, x
    float* cg[4] = {nullptr, nullptr, nullptr, nullptr};
    double* cg_sc = nullptr;
    int cg_par = 0;
    // CUDA graph of the finest-level V-cycle: captured on cap_stream once per
    // di_inpaint call (while the cascade runs), updated into gexec and
    // replayed once per cycle; its profiling events are gev (fixed handles)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool capturing = false;
    static constexpr int kGPairs = 16;
    cudaEvent_t gev[kGPairs][2] = {};
    int g_pairs = 0;            // event pairs recorded by one replay
    long long g_kernels = 0;    // kernels launched by one replay
    long long g_oras = 0, g_pxch = 0, g_tasks = 0, g_pro = 0;  // profile counters of one replay
    unsigned long long* dsteps = nullptr;  // device: completed finest-level local CG steps
    // device-driven decode (see DecodeGraph): stop-test state on the device,
    // its pinned host copy, the capture streams of the graph and its bodies,
    // and a cache of whole-decode graphs keyed by the call's buffers
    StopState* dstate = nullptr;
    StopState* hstate = nullptr;
    cudaEvent_t done_ev = nullptr;
    cudaStream_t cs[3] = {nullptr, nullptr, nullptr};
    static constexpr int kGraphs = 16;
    DecodeGraph graphs[kGraphs];
    unsigned long long graph_clock = 0;
    unsigned long long ws_gen = 0;     // workspace generation (graphs bake its addresses)
    DecodeGraph* pending = nullptr;    // device-driven decode whose stats are not read yet
    bool device_path_broken = false;   // a capture failed: use the host-driven loop
    // capture policy: a call whose buffers have no graph captures one while
    // the cache has room; once it is full, only buffers seen before (a recent
    // key, kept here) get a graph, so a caller that changes buffers every call
    // runs the host-driven loop instead of capturing every time
    static constexpr int kSeen = 64;
    unsigned long long seen[kSeen] = {};
    int seen_next = 0;
};

namespace {

constexpr size_t kAlign = 256;
// The single-block solve of the coarsest level iterates until its
// preconditioned residual r.z has dropped by this factor (relative residual
// about 1e-6, near the FP32 floor), capped at coarse_iters steps.
constexpr float kCoarseRtol2 = 1e-12f;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

di_config resolve(const di_config* in) {
    di_config c;
    std::memset(&c, 0, sizeof c);
    if (in) c = *in;
    if (c.block == 0) c.block = 32;
    if (c.overlap == 0) c.overlap = 6;
    if (c.local_iters == 0) c.local_iters = 8;
    if (c.coarse_iters == 0) c.coarse_iters = 2048;
    if (c.pre == 0) c.pre = 1;
    if (c.post == 0) c.post = 1;
    if (c.max_cycles == 0) c.max_cycles = 16;
    if (c.min_cycles == 0) c.min_cycles = 1;
    if (c.alpha == 0.f) c.alpha = 0.5f;
    if (c.local_stop == 0.f) c.local_stop = 0.2f;
    return c;
}

bool config_ok(const di_config& c) {
    if (c.block != 8 && c.block != 16 && c.block != 32) return false;
    if (c.overlap < 1 || 2 * c.overlap > c.block) return false;
    if (c.local_iters < 0 || c.coarse_iters < 0) return false;
    if (c.pre < 0 || c.post < 0 || c.pre + 1 + c.post > kMaxUpdSlots) return false;
    if (c.max_cycles < 0 || c.min_cycles < 0 || c.min_cycles > c.max_cycles) return false;
    if (!(c.alpha > 0.f) || !std::isfinite(c.alpha)) return false;
    if (c.downsample != 0 && c.downsample != 1) return false;
    if (c.stop_rule < 0 || c.stop_rule > 2) return false;
    if (c.profile != 0 && c.profile != 1) return false;
    if (c.precision < 0 || c.precision > 2) return false;
    if (c.schedule < 0 || c.schedule > 3) return false;
    if (c.smoother < 0 || c.smoother > 1) return false;
    if (c.graph < 0 || c.graph > 1) return false;
    if (c.start < 0 || c.start > 1) return false;
    if (c.local_iters_coarse < 0) return false;
    if (!std::isfinite(c.local_stop)) return false;
    if (c.refine_fp64 != 0 && c.refine_fp64 != 1) return false;
    if (c.local_iters_cascade < 0) return false;
    // the 16-bit modes store the coarse levels narrow: 32x32 blocks and the
    // block smoother only (the global CG smoother keeps FP32 vectors)
    if (c.precision != DI_PREC_FP32 && (c.block != 32 || c.smoother != DI_SMOOTH_ORAS))
        return false;
    return true;
}

di_status cuda_fail(di_ctx* ctx, cudaError_t e, const char* what) {
    if (ctx) std::snprintf(ctx->err, sizeof ctx->err, "%.160s: %.80s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DI_ERR_OOM : DI_ERR_CUDA;
}

// Add the durations of the recorded event pairs (the stream has been
// synchronised) to the profile and recycle the pairs.
void prof_flush(di_ctx* ctx) {
    for (int i = 0; i < ctx->ev_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[i][0], ctx->ev[i][1]) == cudaSuccess)
            ctx->prof.oras_l0_ms += ms;
        else
            cudaGetLastError();  // a missing time is not an error of the next call
    }
    ctx->ev_used = 0;
}

// Add the durations of the event pairs of the last graph replay (the stream
// has been synchronised) and that replay's counters to the profile.
void prof_flush_graph(di_ctx* ctx) {
    for (int i = 0; i < ctx->g_pairs; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->gev[i][0], ctx->gev[i][1]) == cudaSuccess)
            ctx->prof.oras_l0_ms += ms;
        else
            cudaGetLastError();
    }
}

#define DI_CUDA(ctx, call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

void drop_graph(DecodeGraph& dg) {
    if (dg.exec) cudaGraphExecDestroy(dg.exec);
    if (dg.g) cudaGraphDestroy(dg.g);
    dg = DecodeGraph();
}

void free_workspace(di_ctx* ctx) {
    // the cached decode graphs bake the workspace's addresses
    for (auto& dg : ctx->graphs) drop_graph(dg);
    ctx->pending = nullptr;
    ++ctx->ws_gen;
    for (int k = 0; k < 4; ++k) {
        if (ctx->cg[k]) cudaFree(ctx->cg[k]);
        ctx->cg[k] = nullptr;
    }
    if (ctx->pool) cudaFree(ctx->pool);
    if (ctx->planes) cudaFree(ctx->planes);
    if (ctx->partials) cudaFree(ctx->partials);
    ctx->pool = nullptr;
    ctx->planes = nullptr;
    ctx->partials = nullptr;
    ctx->partials_cap = 0;
    ctx->cap_w = ctx->cap_h = ctx->cap_c = 0;
}

// Byte size of the pooled level buffers for an image of (w, h, C); the coarse
// levels' iterates and right-hand sides are stored as `stor` (Storage).
size_t pool_bytes(int w, int h, int C, int L, int stor) {
    size_t total = 0;
    int lw = w, lh = h;
    for (int l = 0; l < L; ++l) {
        const size_t n = (size_t)lw * lh;
        total += align_up((size_t)lh * mask_words_per_row(lw) * sizeof(uint32_t));  // mbits
        if (l == 0) {
            total += align_up(n * C * sizeof(float));  // u[1]
        } else {
            total += align_up(n);                                  // c
            total += align_up(n * C * sizeof(float));             // b
            total += 3 * align_up(n * C * storage_bytes(stor));  // u[0], u[1], r
        }
        coarse_dims(lw, lh, &lw, &lh);
    }
    return total;
}

// Make sure the workspace covers (w, h, C); grows to the elementwise maximum
// of everything seen so far (level l of a smaller image is never larger).
di_status ensure_workspace(di_ctx* ctx, int w, int h, int C) {
    if (w <= ctx->cap_w && h <= ctx->cap_h && C <= ctx->cap_c) return DI_OK;
    const int nw = w > ctx->cap_w ? w : ctx->cap_w;
    const int nh = h > ctx->cap_h ? h : ctx->cap_h;
    const int nc = C > ctx->cap_c ? C : ctx->cap_c;
    free_workspace(ctx);
    const int L = num_levels(nw, nh, ctx->cfg.block);
    cudaError_t e = cudaMalloc(&ctx->pool, pool_bytes(nw, nh, nc, L, ctx->cfg.precision));
    if (e != cudaSuccess) { ctx->pool = nullptr; return cuda_fail(ctx, e, "cudaMalloc(pool)"); }
    e = cudaMalloc(&ctx->planes,
                   oras_scratch_floats(nw, nh, nc, ctx->cfg.block, ctx->cfg.overlap) * sizeof(float));
    if (e != cudaSuccess) { free_workspace(ctx); return cuda_fail(ctx, e, "cudaMalloc(planes)"); }
    ctx->partials_cap = residual_partials_per_channel(nw, nh) * nc;
    e = cudaMalloc(&ctx->partials, ctx->partials_cap * sizeof(double));
    if (e != cudaSuccess) { free_workspace(ctx); return cuda_fail(ctx, e, "cudaMalloc(partials)"); }
    if (ctx->cfg.smoother == DI_SMOOTH_CG) {
        for (int k = 0; k < 4; ++k) {
            e = cudaMalloc(&ctx->cg[k], (size_t)nw * nh * nc * sizeof(float));
            if (e != cudaSuccess) { free_workspace(ctx); return cuda_fail(ctx, e, "cudaMalloc(cg)"); }
        }
    }
    ctx->cap_w = nw;
    ctx->cap_h = nh;
    ctx->cap_c = nc;
    return DI_OK;
}

// Lay the pooled buffers out for this image.
void bind_levels(di_ctx* ctx, const float* f, const uint8_t* c, float* u, int w, int h, int C) {
    const int L = num_levels(w, h, ctx->cfg.block);
    ctx->L = L;
    char* p = static_cast<char*>(ctx->pool);
    int lw = w, lh = h;
    for (int l = 0; l < L; ++l) {
        Level& v = ctx->lv[l];
        v.w = lw;
        v.h = lh;
        v.n = (size_t)lw * lh;
        const size_t fb = align_up(v.n * C * sizeof(float));
        const size_t nb = align_up(v.n * C * storage_bytes(ctx->cfg.precision));
        v.mbits = reinterpret_cast<uint32_t*>(p);
        p += align_up((size_t)lh * mask_words_per_row(lw) * sizeof(uint32_t));
        if (l == 0) {
            v.c = c;
            v.b = f;
            v.u[0] = u;
            v.u[1] = reinterpret_cast<float*>(p); p += fb;
            v.r = nullptr;
        } else {
            v.c = reinterpret_cast<uint8_t*>(p); p += align_up(v.n);
            v.b = reinterpret_cast<float*>(p); p += fb;
            // stored as the coarse levels' Storage (the pointers are untyped there)
            v.u[0] = reinterpret_cast<float*>(p); p += nb;
            v.u[1] = reinterpret_cast<float*>(p); p += nb;
            v.r = reinterpret_cast<float*>(p); p += nb;
        }
        v.unknowns = 0;
        coarse_dims(lw, lh, &lw, &lh);
    }
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

// ---------------------------------------------------------------------------
// Scheduler
// ---------------------------------------------------------------------------

namespace {

struct Sched {
    di_ctx* ctx;
    int C;
    int Leff;   // levels that carry unknown pixels (recursion depth)
    cudaStream_t s;
    int root = 0;  // level whose own problem is being solved (the others solve A e = r)
    float abs2 = 0.f;  // absolute local stop r.r <= abs2 of the smoothing ORAS calls (0: none)

    // Storage of level l's iterates and restricted residual: FP32 on the
    // finest level, the precision's type on the coarse levels.
    int stor(int l) const { return l == 0 ? (int)kF32 : ctx->cfg.precision; }
    // FP64 residuals on the finest level (cfg.refine_fp64)
    bool f64(int l) const { return l == 0 && ctx->cfg.refine_fp64; }

    // Right-hand side of level l: the root level solves A u = b_l (level 0:
    // b = C f; coarse levels: the downsampled mask values), whose right-hand
    // side is zero at unknown pixels; the levels below it solve A e = r_l.
    const float* rhs_of(int l, int* rhs_zero) const {
        const Level& v = ctx->lv[l];
        if (l == root) { *rhs_zero = 1; return v.b; }
        *rhs_zero = 0;
        return v.r;
    }

    di_status run_oras(int l, const float* in, int zero_in, float* out, int iters,
                       unsigned* maxupd, float rtol2 = 0.f, const float* pro_e = nullptr,
                       unsigned* pro_max = nullptr, int pro_mode = 1) {
        const Level& v = ctx->lv[l];
        int rhs_zero;
        const float* rhs = rhs_of(l, &rhs_zero);
        cudaEvent_t* ev = nullptr;
        if (l == 0 && ctx->cfg.profile) {
            if (!ctx->ev_made) {
                for (int i = 0; i < di_ctx::kEvPairs; ++i)
                    for (int k = 0; k < 2; ++k) DI_CUDA(ctx, cudaEventCreate(&ctx->ev[i][k]));
                for (int i = 0; i < di_ctx::kGPairs; ++i)
                    for (int k = 0; k < 2; ++k) DI_CUDA(ctx, cudaEventCreate(&ctx->gev[i][k]));
                ctx->ev_made = true;
            }
            if (ctx->capturing) {
                // a graph node: the pair is read after every replay
                if (ctx->g_pairs < di_ctx::kGPairs) ev = ctx->gev[ctx->g_pairs++];
            } else {
                if (ctx->ev_used == di_ctx::kEvPairs) {
                    DI_CUDA(ctx, cudaStreamSynchronize(s));
                    prof_flush(ctx);
                }
                ev = ctx->ev[ctx->ev_used++];
            }
            ctx->prof.oras_l0_launches += 1;
            if (pro_e) ctx->prof.oras_l0_prolong += 1;
            ctx->prof.oras_l0_pixel_channels += (long long)v.n * C;
            ctx->prof.oras_l0_tasks += (long long)axis_blocks(v.w, ctx->cfg.block, ctx->cfg.overlap) *
                                       axis_blocks(v.h, ctx->cfg.block, ctx->cfg.overlap) * C;
        }
        DI_CUDA(ctx, launch_oras(in, zero_in, rhs, rhs_zero, v.mbits, v.w, v.h, C, ctx->cfg.block,
                                 ctx->cfg.overlap, ctx->cfg.alpha, iters, rtol2, out,
                                 ctx->planes, maxupd, s, ev, ctx->cfg.precision,
                                 ctx->upd + kMaxUpdSlots,
                                 l == 0 && ctx->cfg.profile ? ctx->dsteps : nullptr, stor(l),
                                 f64(l), pro_e, pro_max, pro_mode));
        return DI_OK;
    }

    // Whether a prolongation from level l + 1 to level l can run inside the
    // ORAS iteration that follows it on level l (the V-cycle's correction
    // step before the first post-smoothing, the cascade's interpolation
    // before its smoothing step).
    bool fuse_prolong(int l) const {
        const di_config& cfg = ctx->cfg;
        return cfg.smoother == DI_SMOOTH_ORAS && cfg.block == 32 && stor(l + 1) == kF32 &&
               prolong_fusable(cfg.precision, cfg.overlap, 0);
    }

    // One smoothing call on level l (in -> out): an ORAS iteration, or
    // local_iters steps of global CG (restart = false continues the previous
    // CG call on the same level).
    // pro_e, pro_max, pro_mode: a coarser field prolonged into the start
    // (fuse_prolong; mode 1 adds a correction, mode 0 interpolates a solution
    // with in = b).
    // cascade: the cascade's smoothing step (cfg.local_iters_cascade on level 0).
    di_status smooth(int l, const float* in, int zero_in, float* out, unsigned* maxupd,
                     bool restart = true, const float* pro_e = nullptr,
                     unsigned* pro_max = nullptr, int pro_mode = 1, bool cascade = false) {
        const di_config& cfg = ctx->cfg;
        if (cfg.smoother == DI_SMOOTH_ORAS)
            return run_oras(l, in, zero_in, out,
                            l == 0 && cascade && cfg.local_iters_cascade > 0
                                ? cfg.local_iters_cascade
                            : l > 0 && cfg.local_iters_coarse > 0 ? cfg.local_iters_coarse
                                                                  : cfg.local_iters,
                            maxupd, abs2 > 0.f ? -abs2 : 0.f, pro_e, pro_max, pro_mode);
        const Level& v = ctx->lv[l];
        int rhs_zero;
        const float* rhs = rhs_of(l, &rhs_zero);
        DI_CUDA(ctx, launch_cg_smooth(in, zero_in, rhs, rhs_zero, v.c, v.w, v.h, C,
                                      cfg.local_iters, restart ? 1 : 0, ctx->cg[0], ctx->cg[1],
                                      ctx->cg[2], ctx->cg[3], ctx->partials, ctx->cg_sc,
                                      &ctx->cg_par, out, maxupd, s));
        return DI_OK;
    }

    // V-cycle on level l.  The iterate starts in lv[l].u[0] (or is zero) and
    // ends in lv[l].u[*which].  upd: per-step max-update slots (level 0 only).
    di_status vcycle(int l, bool zero_init, int* which, unsigned* upd) {
        const di_config& cfg = ctx->cfg;
        Level& v = ctx->lv[l];
        const bool coarsest = (l == ctx->L - 1);
        int cur = 0;
        di_status st;
        if (coarsest) {
            // one block covers the level: one ORAS iteration is a local solve
            st = run_oras(l, v.u[0], zero_init ? 1 : 0, v.u[1], cfg.coarse_iters,
                          upd ? &upd[0] : nullptr, kCoarseRtol2);
            if (st) return st;
            *which = 1;
            return DI_OK;
        }
        int slot = 0;
        bool zero = zero_init;
        for (int k = 0; k < cfg.pre; ++k) {
            st = smooth(l, v.u[cur], zero ? 1 : 0, v.u[cur ^ 1], upd ? &upd[slot] : nullptr);
            if (st) return st;
            ++slot;
            cur ^= 1;
            zero = false;
        }
        if (zero) {  // pre = 0 on a zero start: materialise the zero iterate
            DI_CUDA(ctx, cudaMemsetAsync(v.u[cur], 0, v.n * C * storage_bytes(stor(l)), s));
            zero = false;
        }
        const float* pro_e = nullptr;  // correction prolonged inside the first post-smoothing
        unsigned* pro_max = nullptr;
        if (l + 1 < Leff) {
            Level& cv = ctx->lv[l + 1];
            int rz;
            const float* rhs = rhs_of(l, &rz);
            DI_CUDA(ctx, launch_restrict(v.u[cur], rhs, rz, v.c, v.w, v.h, C, cv.c, cv.r, s, stor(l),
                                         rz ? (int)kF32 : stor(l), stor(l + 1), f64(l)));
            int cw = 0;
            st = vcycle(l + 1, true, &cw, nullptr);
            if (st) return st;
            if (cfg.post >= 1 && fuse_prolong(l)) {
                pro_e = cv.u[cw];
                pro_max = upd ? &upd[slot] : nullptr;
            } else {
                DI_CUDA(ctx, launch_prolong(cv.u[cw], nullptr, v.c, v.w, v.h, C, v.u[cur], 1,
                                            upd ? &upd[slot] : nullptr, s, stor(l + 1), stor(l)));
            }
        }
        ++slot;
        for (int k = 0; k < cfg.post; ++k) {
            st = smooth(l, v.u[cur], 0, v.u[cur ^ 1], upd ? &upd[slot] : nullptr, true,
                        k == 0 ? pro_e : nullptr, k == 0 ? pro_max : nullptr);
            if (st) return st;
            ++slot;
            cur ^= 1;
        }
        *which = cur;
        return DI_OK;
    }
};

// Capture one finest-level V-cycle (with the reset of the update slots) as a
// CUDA graph and make ctx->gexec replay it.  The cycle must leave the iterate
// in lv[0].u[0] (pre + post even).  Nothing runs during the capture; on any
// failure the caller falls back to launching the cycle kernel by kernel.
bool capture_vcycle(di_ctx* ctx, Sched& S) {
    if (!ctx->cap_stream &&
        cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const di_profile p0 = ctx->prof;
    const long long k0 = thread_launch_count();
    cudaStream_t s = S.s;
    ctx->g_pairs = 0;
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ctx->capturing = true;
    S.s = ctx->cap_stream;
    int which = -1;
    di_status st = DI_OK;
    if (cudaMemsetAsync(ctx->upd, 0, kMaxUpdSlots * sizeof(unsigned), ctx->cap_stream) !=
        cudaSuccess)
        st = DI_ERR_CUDA;
    if (st == DI_OK) st = S.vcycle(0, false, &which, ctx->upd);
    S.s = s;
    ctx->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->g_kernels = thread_launch_count() - k0;
    add_launches(-ctx->g_kernels);  // captured, not launched
    ctx->g_oras = ctx->prof.oras_l0_launches - p0.oras_l0_launches;
    ctx->g_pxch = ctx->prof.oras_l0_pixel_channels - p0.oras_l0_pixel_channels;
    ctx->g_tasks = ctx->prof.oras_l0_tasks - p0.oras_l0_tasks;
    ctx->g_pro = ctx->prof.oras_l0_prolong - p0.oras_l0_prolong;
    ctx->prof = p0;
    if (st != DI_OK || e != cudaSuccess || g == nullptr || which != 0) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        ctx->err[0] = 0;
        return false;
    }
    bool ok = true;
    if (ctx->gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ctx->gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
    }
    if (!ctx->gexec && cudaGraphInstantiate(&ctx->gexec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        ctx->gexec = nullptr;
        ok = false;
    }
    cudaGraphDestroy(g);
    return ok;
}

di_status timeout(di_ctx* ctx) {
    std::snprintf(ctx->err, sizeof ctx->err,
                  "a bounded device-side wait of the block kernel ran out (tile copies missing)");
    return DI_ERR_TIMEOUT;
}

unsigned bits_of(float f) {
    unsigned b;
    std::memcpy(&b, &f, sizeof b);
    return b;
}

float bits_to_float(unsigned b) {
    float f;
    std::memcpy(&f, &b, sizeof f);
    return f;
}

// ---------------------------------------------------------------------------
// Device-driven decode
//
// The whole decode of one image is captured once (per buffers, size and
// tolerance) into a CUDA graph and replayed: the pyramid with the unknown
// counts, the plan kernel, then one SWITCH node over the number of levels in
// use (the levels down to the first one without unknown pixels, as the
// host-driven loop finds them after the pyramid).  Body v holds the cascade
// for v levels and a WHILE node whose body is one V-cycle recursing through v
// levels followed by the stop test (k_stop, which ends the loop).  What
// depends on the mask is thus decided on the device with one conditional node
// per decode and one loop iteration per cycle, and the graph needs no host
// round trip.  Results equal the host-driven loop bit for bit.
// ---------------------------------------------------------------------------

// Note why the whole-decode graph could not be built (di_last_error); the
// decode then runs the host-driven loop.
void capture_error(di_ctx* ctx, const char* step) {
    const cudaError_t e = cudaGetLastError();
    std::snprintf(ctx->err, sizeof ctx->err, "device-driven decode unavailable (%s: %s)", step,
                  cudaGetErrorString(e));
}

// Add a conditional node after everything captured so far on `s` (which must
// be capturing) and return its body graphs.
bool add_conditional(cudaStream_t s, cudaGraphConditionalHandle h,
                     cudaGraphConditionalNodeType type, unsigned size, cudaGraph_t** bodies) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
        return false;
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = size;
    cudaGraphNode_t node = nullptr;
    if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &p) != cudaSuccess) return false;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies) != cudaSuccess)
        return false;
    *bodies = p.conditional.phGraph_out;
    return true;
}

// Capture into `body` on stream s whatever fn enqueues on it; the kernels it
// launched (counted, then taken back from the launch counter) go to *kern.
template <class Fn>
bool capture_body(cudaStream_t s, cudaGraph_t body, long long* kern, Fn&& fn) {
    if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return false;
    const long long k0 = thread_launch_count();
    const bool ok = fn();
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &out);
    const long long k = thread_launch_count() - k0;
    add_launches(-k);
    if (kern) *kern += k;
    return ok && e == cudaSuccess;
}

// Device address of a norm array of the stop state.
enum { kBnorm2, kNorm2 };
double* state_field(di_ctx* ctx, int which) {
    char* base = reinterpret_cast<char*>(ctx->dstate);
    return reinterpret_cast<double*>(
        base + (which == kBnorm2 ? offsetof(StopState, bnorm2) : offsetof(StopState, norm2)));
}

// The cascade of the reduced FMG for `Leff` levels in use (Leff >= 1), on
// S.s: the start on the coarsest level (a single-block solve) or on the first
// fully known level (u = b there), then prolongation and one smoothing step
// per level up to the finest.  The host-driven loop runs the same sequence.
bool capture_cascade(di_ctx* ctx, Sched& S, int Leff) {
    const di_config& cfg = ctx->cfg;
    const int L = ctx->L, C = S.C;
    Level* lv = ctx->lv;
    int top;
    if (Leff == L) {
        top = L - 1;
        Level& v = lv[top];
        S.root = top;
        if (launch_select(v.b, v.c, v.w, v.h, C, v.u[1], S.s, 0, S.stor(top))) return false;
        if (S.run_oras(top, v.u[1], 0, v.u[0], cfg.coarse_iters, nullptr, kCoarseRtol2))
            return false;
    } else {
        top = Leff;
        Level& v = lv[top];
        if (launch_select(v.b, v.c, v.w, v.h, C, v.u[0], S.s, 0, S.stor(top))) return false;
    }
    for (int l = top - 1; l >= 0; --l) {
        Level& v = lv[l];
        Level& cv = lv[l + 1];
        S.root = l;
        if (S.fuse_prolong(l)) {
            if (S.smooth(l, v.b, 0, v.u[0], nullptr, true, cv.u[0], nullptr, 0, true)) return false;
            continue;
        }
        if (launch_prolong(cv.u[0], v.b, v.c, v.w, v.h, C, v.u[1], 0, nullptr, S.s, S.stor(l + 1),
                           S.stor(l)))
            return false;
        if (S.smooth(l, v.u[1], 0, v.u[0], nullptr, true, nullptr, nullptr, 1, true)) return false;
    }
    S.root = 0;
    return true;
}

bool capture_decode(di_ctx* ctx, Sched& S, const float* f, const uint8_t* c, float* u, int w,
                    int h, int C, float tol, DecodeGraph& dg) {
    const di_config& cfg = ctx->cfg;
    const int L = ctx->L;
    for (int k = 0; k < 3; ++k)
        if (!ctx->cs[k] && cudaStreamCreateWithFlags(&ctx->cs[k], cudaStreamNonBlocking) != cudaSuccess)
            return false;
    cudaStream_t s0 = ctx->cs[0], s1 = ctx->cs[1], s2 = ctx->cs[2];
    cudaStream_t caller = S.s;
    cudaGraph_t g = nullptr;
    const char* step = "graph";
    if (cudaGraphCreate(&g, 0) != cudaSuccess) {
        capture_error(ctx, step);
        return false;
    }
    PlanParams pp;
    std::memset(&pp, 0, sizeof pp);
    pp.L = L;
    pp.max_cycles = cfg.max_cycles;
    pp.n0 = (unsigned long long)w * h;
    const bool cascade = cfg.start != DI_START_GIVEN;
    step = "conditional handles";
    bool ok = cudaGraphConditionalHandleCreate(&pp.h_sel, g, kSelSkip,
                                               cudaGraphCondAssignDefault) == cudaSuccess;
    for (int v = 1; v <= L && ok; ++v)
        ok = cudaGraphConditionalHandleCreate(&pp.h_loop[v], g, 0, cudaGraphCondAssignDefault) ==
             cudaSuccess;
    if (!ok) {
        capture_error(ctx, step);
        cudaGraphDestroy(g);
        return false;
    }
    dg = DecodeGraph();
    const long long k0 = thread_launch_count();
    StopParams sp;
    sp.rule = cfg.stop_rule;
    sp.nslots = cfg.pre + 1 + cfg.post;
    sp.min_cycles = cfg.min_cycles;
    sp.max_cycles = cfg.max_cycles;
    sp.C = C;
    sp.tol = tol;
    Level* lv = ctx->lv;
    int nparts = 0;
    unsigned long long* cnt = ctx->counts;

    ok = cudaStreamBeginCaptureToGraph(s0, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
         cudaSuccess;
    if (ok) {
        S.s = s0;
        auto run = [&]() -> bool {
            // 1. pyramids with the unknown counts, then the plan
            step = "pyramid";
            if (cudaMemsetAsync(cnt, 0, (kMaxLevels + 1) * sizeof(unsigned long long), s0) ||
                cudaMemsetAsync(ctx->upd, 0, (kMaxUpdSlots + 1) * sizeof(unsigned), s0))
                return false;
            if (launch_pack_mask(c, w, h, lv[0].mbits, cnt + 1, s0)) return false;
            for (int l = 1; l < L; ++l) {
                Level& fl = lv[l - 1];
                Level& cl = lv[l];
                if (launch_pyramid_level(fl.c, fl.b, fl.w, fl.h, C, const_cast<uint8_t*>(cl.c),
                                         const_cast<float*>(cl.b), cfg.downsample == 0 ? 1 : 0,
                                         cascade ? 1 : 0, cl.mbits, cnt + 1 + l, s0))
                    return false;
            }
            if (launch_plan(cnt, ctx->dstate, pp, s0)) return false;
            // 2. the given start, and the reference norm of the relative-residual rule
            if (!cascade && launch_select(f, c, w, h, C, u, s0, 1)) return false;
            step = "reference norm";
            if (cfg.stop_rule == DI_STOP_RELATIVE_RESIDUAL &&
                (launch_residual(nullptr, 1, f, 1, c, w, h, C, nullptr, ctx->partials, &nparts,
                                 s0, cfg.refine_fp64 != 0) ||
                 launch_reduce_partials(ctx->partials, nparts, C, state_field(ctx, kBnorm2), s0)))
                return false;
            // 3. one body per number of levels in use: the cascade, then the
            // V-cycle loop recursing through those levels
            cudaGraph_t* b = nullptr;
            step = "switch node";
            if (!add_conditional(s0, pp.h_sel, cudaGraphCondTypeSwitch, L + 1, &b)) return false;
            S.s = s1;
            step = "all-known body";
            if (!capture_body(s1, b[0], &dg.k_sel[0], [&] {
                    return launch_select(f, c, w, h, C, u, s1) == cudaSuccess;
                }))
                return false;
            for (int v = 1; v <= L; ++v) {
                step = "level body";
                const bool bok = capture_body(s1, b[v], &dg.k_sel[v], [&] {
                    S.Leff = v;
                    if (cascade && !capture_cascade(ctx, S, v)) return false;
                    cudaGraph_t* wb = nullptr;
                    step = "while node";
                    if (!add_conditional(s1, pp.h_loop[v], cudaGraphCondTypeWhile, 1, &wb))
                        return false;
                    step = "cycle body";
                    S.s = s2;
                    const bool cok = capture_body(s2, wb[0], &dg.k_cycle[v], [&] {
                        int which = -1;
                        if (S.vcycle(0, false, &which, ctx->upd) || which != 0) return false;
                        if (cfg.stop_rule == DI_STOP_RELATIVE_RESIDUAL &&
                            (launch_residual(lv[0].u[0], 0, f, 1, c, w, h, C, nullptr,
                                             ctx->partials, &nparts, s2,
                                             cfg.refine_fp64 != 0) ||
                             launch_reduce_partials(ctx->partials, nparts, C,
                                                    state_field(ctx, kNorm2), s2)))
                            return false;
                        return launch_stop(ctx->upd, ctx->dstate, sp, pp.h_loop[v], s2) ==
                               cudaSuccess;
                    });
                    S.s = s1;
                    return cok;
                });
                if (!bok) return false;
            }
            S.s = s0;
            return true;
        };
        ok = run();
        if (ok) step = "end of capture";
        cudaGraph_t out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s0, &out);
        ok = ok && e == cudaSuccess;
    } else {
        step = "begin capture";
    }
    S.s = caller;
    S.root = 0;
    S.Leff = L;
    // everything left after the bodies took theirs is the fixed part
    dg.k_pre = thread_launch_count() - k0;
    add_launches(-dg.k_pre);
    if (ok) {
        step = "instantiate";
        ok = cudaGraphInstantiate(&dg.exec, g, 0) == cudaSuccess;
    }
    if (!ok) {
        capture_error(ctx, step);
        if (dg.exec) cudaGraphExecDestroy(dg.exec);
        cudaGraphDestroy(g);
        dg = DecodeGraph();
        return false;
    }
    dg.g = g;
    dg.valid = true;
    dg.f = f;
    dg.c = c;
    dg.u = u;
    dg.w = w;
    dg.h = h;
    dg.C = C;
    dg.tol = tol;
    dg.ws_gen = ctx->ws_gen;
    return true;
}

// Fill the statistics from the read-back stop state of a device-driven
// decode (its stream has completed) and count its kernels.
di_status finish_device(di_ctx* ctx) {
    DecodeGraph* dg = ctx->pending;
    ctx->pending = nullptr;
    const StopState& hs = *ctx->hstate;
    const int L = ctx->L;
    const int Leff = hs.levels_used;
    std::memset(&ctx->stats, 0, sizeof ctx->stats);
    for (int k = 0; k < 4; ++k) ctx->stats.rel_residual[k] = -1.f;
    if (hs.status == DI_ERR_EMPTY_MASK) {  // as the host-driven loop reports it
        if (dg && dg->valid) add_launches(dg->k_pre);
        return DI_ERR_EMPTY_MASK;
    }
    ctx->stats.levels = L;
    ctx->stats.levels_used = Leff;
    ctx->stats.cycles = hs.cycles;
    ctx->stats.converged = hs.converged;
    ctx->stats.est_error = ctx->cfg.stop_rule == DI_STOP_ERROR_ESTIMATE ? hs.est : 0.f;
    for (int k = 0; k < 4; ++k) ctx->stats.rel_residual[k] = hs.rel[k];
    ctx->stats.unknowns = (long long)hs.unknowns;
    if (dg && dg->valid) {
        long long k = dg->k_pre;  // the empty-mask case runs nothing else
        if (hs.status != DI_ERR_EMPTY_MASK && Leff >= 0 && Leff <= L)
            k += dg->k_sel[Leff] + dg->k_cycle[Leff] * hs.cycles;
        add_launches(k);
    }
    if (hs.status == DI_ERR_TIMEOUT) return timeout(ctx);
    if (hs.status == DI_ERR_EMPTY_MASK) return DI_ERR_EMPTY_MASK;
    return hs.status == DI_OK ? DI_OK : DI_ERR_NOT_CONVERGED;
}

// Run a decode through its cached (or newly captured) graph.  Returns false
// if the graph could not be built (the caller then runs the host-driven
// loop); otherwise *st is the status (DI_OK while the work is still running
// when wait is false).
bool device_decode(di_ctx* ctx, Sched& S, const float* f, const uint8_t* c, float* u, int w,
                   int h, int C, float tol, bool wait, di_status* st) {
    DecodeGraph* hit = nullptr;
    DecodeGraph* victim = &ctx->graphs[0];
    for (auto& dg : ctx->graphs) {
        if (dg.valid && dg.f == f && dg.c == c && dg.u == u && dg.w == w && dg.h == h &&
            dg.C == C && dg.tol == tol && dg.ws_gen == ctx->ws_gen) {
            hit = &dg;
            break;
        }
        if (!dg.valid || dg.used < victim->used) victim = &dg;
    }
    if (!hit) {
        // capture while the cache has room; then only for buffers seen before
        // (the others run the host-driven loop, which captures no more than
        // one V-cycle per call)
        unsigned long long key = 1469598103934665603ull;
        for (unsigned long long v :
             {(unsigned long long)(uintptr_t)f, (unsigned long long)(uintptr_t)c,
              (unsigned long long)(uintptr_t)u, (unsigned long long)w, (unsigned long long)h,
              (unsigned long long)C, (unsigned long long)bits_of(tol), ctx->ws_gen})
            key = (key ^ v) * 1099511628211ull;
        bool seen = false;
        for (unsigned long long k : ctx->seen) seen = seen || (k == key);
        if (!seen) {
            ctx->seen[ctx->seen_next] = key;
            ctx->seen_next = (ctx->seen_next + 1) % di_ctx::kSeen;
        }
        if (victim->valid && !seen) return false;  // the cache is full
        drop_graph(*victim);
        if (!capture_decode(ctx, S, f, c, u, w, h, C, tol, *victim)) {
            ctx->device_path_broken = true;
            return false;
        }
        hit = victim;
    }
    hit->used = ++ctx->graph_clock;
    cudaStream_t s = S.s;
    cudaError_t e = cudaGraphLaunch(hit->exec, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(StopState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->done_ev, s);
    if (e != cudaSuccess) {
        *st = cuda_fail(ctx, e, "device-driven decode");
        return true;
    }
    ctx->pending = hit;
    ctx->prof.device_decodes += 1;
    if (!wait) {
        *st = DI_OK;
        return true;
    }
    e = cudaEventSynchronize(ctx->done_ev);
    if (e != cudaSuccess) {
        ctx->pending = nullptr;
        *st = cuda_fail(ctx, e, "cudaEventSynchronize");
        return true;
    }
    *st = finish_device(ctx);
    return true;
}

}  // namespace

extern "C" {

di_status di_plan(const di_config* cfg, int width, int height, int channels,
                  di_plan_info* out) {
    if (!out || width < 1 || height < 1 || channels < 1 || channels > kMaxChannels)
        return DI_ERR_INVALID_ARG;
    di_config c = resolve(cfg);
    if (!config_ok(c)) return DI_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof *out);
    const int L = num_levels(width, height, c.block);
    if (L > kMaxLevels) return DI_ERR_INVALID_ARG;
    out->levels = L;
    int lw = width, lh = height;
    for (int l = 0; l < L; ++l) {
        out->width[l] = lw;
        out->height[l] = lh;
        out->blocks_x[l] = axis_blocks(lw, c.block, c.overlap);
        out->blocks_y[l] = axis_blocks(lh, c.block, c.overlap);
        coarse_dims(lw, lh, &lw, &lh);
    }
    out->local_problems = (long long)out->blocks_x[0] * out->blocks_y[0] * channels;
    out->workspace_bytes = (long long)(pool_bytes(width, height, channels, L, c.precision) +
                                       oras_scratch_floats(width, height, channels, c.block,
                                                           c.overlap) * sizeof(float) +
                                       residual_partials_per_channel(width, height) * channels *
                                           sizeof(double));
    if (c.smoother == DI_SMOOTH_CG)  // r, p, q, x of the global CG smoother
        out->workspace_bytes += 4LL * width * height * channels * (long long)sizeof(float);
    return DI_OK;
}

di_status di_create(const di_config* cfg, int device, di_ctx** out) {
    if (!out) return DI_ERR_INVALID_ARG;
    *out = nullptr;
    di_config c = resolve(cfg);
    if (!config_ok(c)) return DI_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return DI_ERR_INVALID_ARG;
    di_ctx* ctx = new (std::nothrow) di_ctx();
    if (!ctx) return DI_ERR_OOM;
    ctx->cfg = c;
    ctx->launch_base = launch_count();
    ctx->device = device;
    std::memset(&ctx->stats, 0, sizeof ctx->stats);
    ctx->err[0] = 0;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->norm2, kMaxChannels * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->counts, (kMaxLevels + 1) * sizeof(unsigned long long));
    // update slots, then one word: the device-side error flag (timed-out waits)
    if (e == cudaSuccess) e = cudaMalloc(&ctx->upd, (kMaxUpdSlots + 1) * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->upd, 0, (kMaxUpdSlots + 1) * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->cg_sc, 4 * kMaxChannels * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dsteps, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->dsteps, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->host, 4096);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dstate, sizeof(StopState));
    if (e == cudaSuccess) e = cudaMemset(ctx->dstate, 0, sizeof(StopState));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->hstate, sizeof(StopState));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        di_status st = cuda_fail(ctx, e, "di_create");
        di_destroy(ctx);
        return st;
    }
    *out = ctx;
    return DI_OK;
}

void di_destroy(di_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    free_workspace(ctx);
    if (ctx->ev_made) {
        for (int i = 0; i < di_ctx::kEvPairs; ++i)
            for (int k = 0; k < 2; ++k) cudaEventDestroy(ctx->ev[i][k]);
        for (int i = 0; i < di_ctx::kGPairs; ++i)
            for (int k = 0; k < 2; ++k) cudaEventDestroy(ctx->gev[i][k]);
    }
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (int k = 0; k < 3; ++k)
        if (ctx->cs[k]) cudaStreamDestroy(ctx->cs[k]);
    if (ctx->dstate) cudaFree(ctx->dstate);
    if (ctx->hstate) cudaFreeHost(ctx->hstate);
    if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
    if (ctx->norm2) cudaFree(ctx->norm2);
    if (ctx->counts) cudaFree(ctx->counts);
    if (ctx->upd) cudaFree(ctx->upd);
    if (ctx->cg_sc) cudaFree(ctx->cg_sc);
    if (ctx->dsteps) cudaFree(ctx->dsteps);
    if (ctx->host) cudaFreeHost(ctx->host);
    delete ctx;
}

const char* di_status_string(di_status s) {
    switch (s) {
        case DI_OK: return "ok";
        case DI_ERR_INVALID_ARG: return "invalid argument";
        case DI_ERR_EMPTY_MASK: return "empty mask";
        case DI_ERR_OOM: return "out of device memory";
        case DI_ERR_NOT_CONVERGED: return "not converged";
        case DI_ERR_CUDA: return "CUDA error";
        case DI_ERR_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char* di_last_error(const di_ctx* ctx) { return ctx ? ctx->err : ""; }

di_status di_get_profile(const di_ctx* ctx, di_profile* out) {
    if (!ctx || !out) return DI_ERR_INVALID_ARG;
    *out = ctx->prof;
    out->launches = launch_count() - ctx->launch_base;
    unsigned long long steps = 0;
    if (cudaSetDevice(ctx->device) != cudaSuccess ||
        cudaMemcpy(&steps, ctx->dsteps, sizeof steps, cudaMemcpyDeviceToHost) != cudaSuccess)
        return DI_ERR_CUDA;
    out->oras_l0_cg_steps = (long long)steps;
    return DI_OK;
}

di_status di_reset_profile(di_ctx* ctx) {
    if (!ctx) return DI_ERR_INVALID_ARG;
    std::memset(&ctx->prof, 0, sizeof ctx->prof);
    ctx->launch_base = launch_count();
    if (cudaSetDevice(ctx->device) != cudaSuccess ||
        cudaMemset(ctx->dsteps, 0, sizeof(unsigned long long)) != cudaSuccess)
        return DI_ERR_CUDA;
    return DI_OK;
}

di_status di_get_stats(const di_ctx* cctx, di_stats* out) {
    if (!cctx || !out) return DI_ERR_INVALID_ARG;
    di_ctx* ctx = const_cast<di_ctx*>(cctx);
    if (ctx->pending) {
        // the last call was enqueued without waiting: wait for its work and
        // read its statistics now
        if (cudaSetDevice(ctx->device) != cudaSuccess ||
            cudaEventSynchronize(ctx->done_ev) != cudaSuccess) {
            ctx->pending = nullptr;
            return DI_ERR_CUDA;
        }
        ctx->stats.status = finish_device(ctx);
    }
    *out = ctx->stats;
    return DI_OK;
}

}  // extern "C"

namespace {

// The decode of di_inpaint / di_inpaint_async.  The device-driven graph runs
// it when the configuration allows (V-cycle schedule of the reduced FMG,
// graph replay on, no profiling events, an even number of smoothing steps
// per cycle, at least two levels); otherwise the host-driven loop below runs
// it, synchronously.
di_status inpaint_impl(di_ctx* ctx, const float* f, const uint8_t* c, int width, int height,
                       int channels, float tol, float* u, void* stream, bool wait) {
    if (!ctx || !f || !c || !u || width < 1 || height < 1 || channels < 1 ||
        channels > kMaxChannels || !(tol > 0.f) || !std::isfinite(tol))
        return DI_ERR_INVALID_ARG;
    const size_t n0 = (size_t)width * height;
    const size_t img_bytes = n0 * channels * sizeof(float);
    if (overlaps(f, img_bytes, u, img_bytes) || overlaps(c, n0, u, img_bytes))
        return DI_ERR_INVALID_ARG;
    if (num_levels(width, height, ctx->cfg.block) > kMaxLevels - 1) return DI_ERR_INVALID_ARG;
    std::memset(&ctx->stats, 0, sizeof ctx->stats);
    for (int k = 0; k < 4; ++k) ctx->stats.rel_residual[k] = -1.f;
    ctx->pending = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DI_CUDA(ctx, cudaSetDevice(ctx->device));
    di_status st = ensure_workspace(ctx, width, height, channels);
    if (st) return st;
    bind_levels(ctx, f, c, u, width, height, channels);
    const di_config& cfg = ctx->cfg;
    const int L = ctx->L;
    const int C = channels;

    if (cfg.graph == DI_GRAPH_ON && !cfg.profile && cfg.schedule == DI_SCHED_REDUCED_FMG &&
        (cfg.pre + cfg.post) % 2 == 0 && L >= 2 && !ctx->device_path_broken) {
        Sched S{ctx, C, L, s};
        if (cfg.stop_rule == DI_STOP_ERROR_ESTIMATE && cfg.local_stop > 0.f)
            S.abs2 = (cfg.local_stop * tol) * (cfg.local_stop * tol);
        if (device_decode(ctx, S, f, c, u, width, height, C, tol, wait, &st)) return st;
        // the graph could not be built: the host-driven loop below
        bind_levels(ctx, f, c, u, width, height, channels);
    }

    // 1. pyramids and unknown counts
    unsigned long long* cnt = ctx->counts;
    DI_CUDA(ctx, cudaMemsetAsync(cnt, 0, (kMaxLevels + 1) * sizeof(unsigned long long), s));
    DI_CUDA(ctx, cudaMemsetAsync(ctx->upd + kMaxUpdSlots, 0, sizeof(unsigned), s));
    // cnt[1 + l]: unknown pixels of level l
    DI_CUDA(ctx, launch_pack_mask(c, width, height, ctx->lv[0].mbits, cnt + 1, s));
    for (int l = 1; l < L; ++l) {
        Level& f_ = ctx->lv[l - 1];
        Level& cv = ctx->lv[l];
        // the coarse values feed the cascade only
        DI_CUDA(ctx, launch_pyramid_level(f_.c, f_.b, f_.w, f_.h, C, const_cast<uint8_t*>(cv.c),
                                          const_cast<float*>(cv.b), cfg.downsample == 0 ? 1 : 0,
                                          cfg.start != DI_START_GIVEN ? 1 : 0, cv.mbits,
                                          cnt + 1 + l, s));
    }
    unsigned long long* hcnt = static_cast<unsigned long long*>(ctx->host);
    DI_CUDA(ctx, cudaMemcpyAsync(hcnt, cnt, (L + 1) * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
    DI_CUDA(ctx, cudaStreamSynchronize(s));
    if (hcnt[1] == (unsigned long long)n0) return DI_ERR_EMPTY_MASK;
    ctx->lv[0].unknowns = (long long)hcnt[1];
    int Leff = L;
    for (int l = 1; l < L; ++l) {
        ctx->lv[l].unknowns = (long long)hcnt[1 + l];
        if (ctx->lv[l].unknowns == 0) { Leff = l; break; }
    }
    if (ctx->lv[0].unknowns == 0) Leff = 0;
    ctx->stats.levels = L;
    ctx->stats.levels_used = Leff;
    ctx->stats.unknowns = ctx->lv[0].unknowns;

    if (Leff == 0) {  // every pixel is known
        DI_CUDA(ctx, launch_select(f, c, width, height, C, u, s));
        DI_CUDA(ctx, cudaStreamSynchronize(s));
        ctx->stats.converged = 1;
        return DI_OK;
    }

    Sched S{ctx, C, Leff, s};
    if (cfg.stop_rule == DI_STOP_ERROR_ESTIMATE && cfg.local_stop > 0.f)
        S.abs2 = (cfg.local_stop * tol) * (cfg.local_stop * tol);
    Level& v0 = ctx->lv[0];
    float* const caller_u = v0.u[0];
    if (cfg.start == DI_START_GIVEN) {
        // the caller's u is the initial iterate (e.g. the previous video
        // frame's result): u = f on the mask, the given values elsewhere
        DI_CUDA(ctx, launch_select(f, c, width, height, C, v0.u[0], s, 1));
    } else if (cfg.schedule == DI_SCHED_SINGLE) {
        // no hierarchy: u = f on the mask, 0 elsewhere, then smoothing on level 0
        DI_CUDA(ctx, launch_select(f, c, width, height, C, v0.u[0], s));
    } else {
        // 2. cascade (one-way multigrid from the coarsest level)
        int top;
        if (Leff == L) {
            top = L - 1;
            Level& v = ctx->lv[top];
            S.root = top;
            DI_CUDA(ctx, launch_select(v.b, v.c, v.w, v.h, C, v.u[1], s, 0, S.stor(top)));
            st = S.run_oras(top, v.u[1], 0, v.u[0], cfg.coarse_iters, nullptr, kCoarseRtol2);
            if (st) return st;
        } else {
            top = Leff;  // fully known level: u = b there
            Level& v = ctx->lv[top];
            DI_CUDA(ctx, launch_select(v.b, v.c, v.w, v.h, C, v.u[0], s, 0, S.stor(top)));
        }
        for (int l = top - 1; l >= 0; --l) {
            Level& v = ctx->lv[l];
            Level& cv = ctx->lv[l + 1];
            S.root = l;
            if (cfg.schedule == DI_SCHED_FULL_FMG) {
                // full FMG: a V-cycle on every level of the cascade
                DI_CUDA(ctx, launch_prolong(cv.u[0], v.b, v.c, v.w, v.h, C, v.u[0], 0, nullptr, s,
                                            S.stor(l + 1), S.stor(l)));
                int which = 0;
                st = S.vcycle(l, false, &which, nullptr);
                if (st) return st;
                if (which != 0) std::swap(v.u[0], v.u[1]);
            } else if (S.fuse_prolong(l)) {
                // reduced FMG and multilevel: one smoothing step per level,
                // from b on the mask and the interpolated coarser solution
                st = S.smooth(l, v.b, 0, v.u[0], nullptr, true, cv.u[0], nullptr, 0, true);
                if (st) return st;
            } else {
                DI_CUDA(ctx, launch_prolong(cv.u[0], v.b, v.c, v.w, v.h, C, v.u[1], 0, nullptr, s,
                                            S.stor(l + 1), S.stor(l)));
                st = S.smooth(l, v.u[1], 0, v.u[0], nullptr, true, nullptr, nullptr, 1, true);
                if (st) return st;
            }
        }
    }

    // 3. cycles on the finest level with the stop test: V-cycles (FMG
    // schedules) or single smoothing steps (multilevel, single level)
    S.root = 0;
    const bool vcycles = cfg.schedule == DI_SCHED_REDUCED_FMG || cfg.schedule == DI_SCHED_FULL_FMG;
    // replay the finest-level V-cycle as a CUDA graph, captured while the
    // cascade (already queued) runs
    const bool graph = vcycles && cfg.graph == DI_GRAPH_ON && (cfg.pre + cfg.post) % 2 == 0 &&
                       cfg.max_cycles > 0 && capture_vcycle(ctx, S);
    // CG smoothing on the finest level continues one CG run across the steps
    // of the multilevel and single-level schedules (multilevel: from the
    // cascade's level-0 call, which solves the same system)
    bool cg_continue = cfg.schedule == DI_SCHED_MULTILEVEL;
    const int nslots = vcycles ? cfg.pre + 1 + cfg.post : 1;
    float prevU = -1.f, prevQ = -1.f;
    int cycles = 0;
    bool converged = false;
    float est = INFINITY;
    float* hupd = static_cast<float*>(ctx->host);
    double* hnorm = reinterpret_cast<double*>(static_cast<char*>(ctx->host) + 256);
    double bnorm2[kMaxChannels] = {0, 0, 0, 0};
    int nparts = 0;
    if (cfg.stop_rule == DI_STOP_RELATIVE_RESIDUAL) {
        DI_CUDA(ctx, launch_residual(nullptr, 1, f, 1, c, width, height, C, nullptr,
                                     ctx->partials, &nparts, s, cfg.refine_fp64 != 0));
        DI_CUDA(ctx, launch_reduce_partials(ctx->partials, nparts, C, ctx->norm2, s));
        DI_CUDA(ctx, cudaMemcpyAsync(hnorm, ctx->norm2, C * sizeof(double), cudaMemcpyDeviceToHost, s));
        DI_CUDA(ctx, cudaStreamSynchronize(s));
        for (int k = 0; k < C; ++k) bnorm2[k] = hnorm[k];
    }
    while (cycles < cfg.max_cycles) {
        int which = 0;
        if (graph) {
            DI_CUDA(ctx, cudaGraphLaunch(ctx->gexec, s));
            add_launches(ctx->g_kernels);
            ctx->prof.oras_l0_launches += ctx->g_oras;
            ctx->prof.oras_l0_pixel_channels += ctx->g_pxch;
            ctx->prof.oras_l0_tasks += ctx->g_tasks;
            ctx->prof.oras_l0_prolong += ctx->g_pro;
            if (cfg.profile && cfg.stop_rule == DI_STOP_FIXED_CYCLES) {
                // the replay's event pairs are re-recorded by the next one
                DI_CUDA(ctx, cudaStreamSynchronize(s));
                prof_flush_graph(ctx);
            }
            ++cycles;
            if (cfg.stop_rule == DI_STOP_FIXED_CYCLES) continue;
            goto stop_test;
        }
        DI_CUDA(ctx, cudaMemsetAsync(ctx->upd, 0, kMaxUpdSlots * sizeof(unsigned), s));
        // the iterate lives in v0.u[0] between cycles (buffers swap by pointer)
        if (vcycles) {
            st = S.vcycle(0, false, &which, ctx->upd);
        } else {
            st = S.smooth(0, v0.u[0], 0, v0.u[1], ctx->upd, !cg_continue);
            cg_continue = true;
            which = 1;
        }
        if (st) return st;
        if (which != 0) std::swap(v0.u[0], v0.u[1]);
        ++cycles;
        if (cfg.stop_rule == DI_STOP_FIXED_CYCLES) continue;
    stop_test:
        if (cfg.stop_rule == DI_STOP_ERROR_ESTIMATE) {
            DI_CUDA(ctx, cudaMemcpyAsync(hupd, ctx->upd, (kMaxUpdSlots + 1) * sizeof(unsigned),
                                         cudaMemcpyDeviceToHost, s));
            DI_CUDA(ctx, cudaStreamSynchronize(s));
            prof_flush(ctx);
            if (graph) prof_flush_graph(ctx);
            if (reinterpret_cast<unsigned*>(hupd)[kMaxUpdSlots]) return timeout(ctx);
            float U = 0.f;
            for (int k = 0; k < nslots; ++k) U += bits_to_float(reinterpret_cast<unsigned*>(hupd)[k]);
            if (!std::isfinite(U)) { est = INFINITY; prevU = -1.f; prevQ = -1.f; }
            else if (prevU > 0.f) {
                // decay factor: the larger of the last two measured ratios
                const float qk = U / prevU;
                const float q = prevQ > qk ? prevQ : qk;
                prevQ = qk;
                est = q < 1.f ? U * q / (1.f - q) : INFINITY;
            } else {
                est = U;  // first cycle: no decay measured yet (factor 1/2 assumed)
            }
            prevU = U;
            if (U == 0.f) est = 0.f;
            ctx->stats.est_error = est;
            if (cycles >= cfg.min_cycles && est <= 0.5f * tol) { converged = true; break; }
        } else {
            DI_CUDA(ctx, launch_residual(v0.u[0], 0, f, 1, c, width, height, C, nullptr,
                                         ctx->partials, &nparts, s, cfg.refine_fp64 != 0));
            DI_CUDA(ctx, launch_reduce_partials(ctx->partials, nparts, C, ctx->norm2, s));
            DI_CUDA(ctx, cudaMemcpyAsync(hnorm, ctx->norm2, C * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
            DI_CUDA(ctx, cudaStreamSynchronize(s));
            prof_flush(ctx);
            if (graph) prof_flush_graph(ctx);
            bool ok = true;
            for (int k = 0; k < C; ++k) {
                const double rr = bnorm2[k] > 0 ? std::sqrt(hnorm[k] / bnorm2[k]) : 0.0;
                ctx->stats.rel_residual[k] = (float)rr;
                if (!(rr <= tol)) ok = false;
            }
            if (cycles >= cfg.min_cycles && ok) { converged = true; break; }
        }
    }
    if (cfg.stop_rule == DI_STOP_FIXED_CYCLES) {
        DI_CUDA(ctx, cudaStreamSynchronize(s));
        converged = true;
    }
    if (v0.u[0] != caller_u)
        DI_CUDA(ctx, cudaMemcpyAsync(caller_u, v0.u[0], v0.n * C * sizeof(float),
                                     cudaMemcpyDeviceToDevice, s));
    if (cfg.stop_rule != DI_STOP_ERROR_ESTIMATE || v0.u[0] != caller_u) {
        unsigned* hflag = static_cast<unsigned*>(ctx->host) + 1000;
        DI_CUDA(ctx, cudaMemcpyAsync(hflag, ctx->upd + kMaxUpdSlots, sizeof(unsigned),
                                     cudaMemcpyDeviceToHost, s));
        DI_CUDA(ctx, cudaStreamSynchronize(s));
        if (*hflag) return timeout(ctx);
    }
    prof_flush(ctx);
    ctx->stats.cycles = cycles;
    ctx->stats.converged = converged ? 1 : 0;
    return converged ? DI_OK : DI_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" {

di_status di_inpaint(di_ctx* ctx, const float* f, const uint8_t* c, int width, int height,
                     int channels, float tol, float* u, void* stream) {
    const di_status st = inpaint_impl(ctx, f, c, width, height, channels, tol, u, stream, true);
    if (ctx) ctx->stats.status = st;
    return st;
}

di_status di_inpaint_async(di_ctx* ctx, const float* f, const uint8_t* c, int width, int height,
                           int channels, float tol, float* u, void* stream) {
    const di_status st = inpaint_impl(ctx, f, c, width, height, channels, tol, u, stream, false);
    if (ctx && !ctx->pending) ctx->stats.status = st;
    return st;
}

// ---------------------------------------------------------------------------
// Single steps
// ---------------------------------------------------------------------------

di_status di_mask_downsample(const uint8_t* c, int width, int height, uint8_t* cH,
                             void* stream) {
    if (!c || !cH || width < 1 || height < 1) return DI_ERR_INVALID_ARG;
    cudaError_t e = launch_mask_down(c, width, height, cH, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DI_OK : DI_ERR_CUDA;
}

di_status di_values_downsample(const uint8_t* c, const float* b, int width, int height,
                               int channels, const uint8_t* cH, float* bH, int modified,
                               void* stream) {
    if (!c || !b || !cH || !bH || width < 1 || height < 1 || channels < 1 ||
        channels > kMaxChannels || (modified != 0 && modified != 1))
        return DI_ERR_INVALID_ARG;
    cudaError_t e = launch_values_down(c, b, width, height, channels, cH, bH, modified,
                                       static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DI_OK : DI_ERR_CUDA;
}

di_status di_pyramid_level(const uint8_t* c, const float* b, int width, int height, int channels,
                           uint8_t* cH, float* bH, uint32_t* bits, int modified,
                           unsigned long long* unknown, void* stream) {
    if (!c || !cH || !bits || width < 1 || height < 1 || channels < 1 ||
        channels > kMaxChannels || (modified != 0 && modified != 1) || (!b) != (!bH))
        return DI_ERR_INVALID_ARG;
    cudaError_t e = launch_pyramid_level(c, b, width, height, channels, cH, bH, modified,
                                         b ? 1 : 0, bits, unknown,
                                         static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DI_OK : DI_ERR_CUDA;
}

di_status di_residual_norm(di_ctx* ctx, const float* u, const float* b, int rhs_zero,
                           const uint8_t* c, int width, int height, int channels, float* r,
                           double* norm2, void* stream) {
    if (!ctx || !u || !b || !c || !norm2 || width < 1 || height < 1 || channels < 1 ||
        channels > kMaxChannels)
        return DI_ERR_INVALID_ARG;
    DI_CUDA(ctx, cudaSetDevice(ctx->device));
    di_status st = ensure_workspace(ctx, width, height, channels);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int nparts = 0;
    DI_CUDA(ctx, launch_residual(u, 0, b, rhs_zero ? 1 : 0, c, width, height, channels, r,
                                 ctx->partials, &nparts, s));
    DI_CUDA(ctx, launch_reduce_partials(ctx->partials, nparts, channels, norm2, s));
    return DI_OK;
}

di_status di_residual_norm_noalloc(const float* u, const float* b, int rhs_zero,
                                   const uint8_t* c, int width, int height, int channels,
                                   float* r, double* norm2, void* stream) {
    if (!u || !b || !c || !norm2 || width < 1 || height < 1 || channels < 1 ||
        channels > kMaxChannels)
        return DI_ERR_INVALID_ARG;
    const long long need = (long long)residual_partials_per_channel(width, height) * channels;
    if (need > kNoAllocPartials || need > DI_NOALLOC_PARTIALS) return DI_ERR_INVALID_ARG;
    cudaError_t e = launch_residual_noalloc(u, b, rhs_zero ? 1 : 0, c, width, height, channels, r,
                                            norm2, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DI_OK : DI_ERR_CUDA;
}

di_status di_restrict_residual(const float* u, const float* b, int rhs_zero, const uint8_t* c,
                               int width, int height, int channels, const uint8_t* cH,
                               float* rH, int fp64, void* stream) {
    if (!u || !b || !c || !cH || !rH || width < 1 || height < 1 || channels < 1 ||
        channels > kMaxChannels || (fp64 != 0 && fp64 != 1))
        return DI_ERR_INVALID_ARG;
    cudaError_t e = launch_restrict(u, b, rhs_zero ? 1 : 0, c, width, height, channels, cH, rH,
                                    static_cast<cudaStream_t>(stream), kF32, kF32, kF32,
                                    fp64 != 0);
    return e == cudaSuccess ? DI_OK : DI_ERR_CUDA;
}

di_status di_prolong(const float* uH, const float* b, const uint8_t* c, int width, int height,
                     int channels, float* u, int mode, void* stream) {
    if (!uH || !c || !u || width < 1 || height < 1 || channels < 1 || channels > kMaxChannels ||
        (mode != 0 && mode != 1) || (mode == 0 && !b))
        return DI_ERR_INVALID_ARG;
    cudaError_t e = launch_prolong(uH, b, c, width, height, channels, u, mode, nullptr,
                                   static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DI_OK : DI_ERR_CUDA;
}

di_status di_oras_iteration(di_ctx* ctx, const float* u_in, const float* b, int rhs_zero,
                            const uint8_t* c, int width, int height, int channels,
                            int local_iters, float* u_out, void* stream) {
    if (!ctx || !u_in || !b || !c || !u_out || width < 1 || height < 1 || channels < 1 ||
        channels > kMaxChannels || local_iters < 0)
        return DI_ERR_INVALID_ARG;
    const size_t bytes = (size_t)width * height * channels * sizeof(float);
    if (overlaps(u_in, bytes, u_out, bytes)) return DI_ERR_INVALID_ARG;
    DI_CUDA(ctx, cudaSetDevice(ctx->device));
    di_status st = ensure_workspace(ctx, width, height, channels);
    if (st) return st;
    // the single-step call uses the finest level's packed-mask buffer of the pool
    bind_levels(ctx, b, c, u_out, width, height, channels);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* bits = ctx->lv[0].mbits;
    DI_CUDA(ctx, launch_pack_mask(c, width, height, bits, nullptr, s));
    DI_CUDA(ctx, launch_oras(u_in, 0, b, rhs_zero ? 1 : 0, bits, width, height, channels,
                             ctx->cfg.block, ctx->cfg.overlap, ctx->cfg.alpha, local_iters, 0.f,
                             u_out, ctx->planes, nullptr, s, nullptr, ctx->cfg.precision,
                             ctx->upd + kMaxUpdSlots, nullptr, kF32,
                             ctx->cfg.refine_fp64 != 0));
    return DI_OK;
}

di_status di_prolong_oras_iteration(di_ctx* ctx, const float* uH, int mode, const float* u_in,
                                    const float* b, int rhs_zero, const uint8_t* c, int width,
                                    int height, int channels, int local_iters, float* u_out,
                                    void* stream) {
    if (!ctx || !uH || !u_in || !b || !c || !u_out || width < 1 || height < 1 || channels < 1 ||
        channels > kMaxChannels || local_iters < 0 || (mode != 0 && mode != 1) ||
        ctx->cfg.block != 32 ||
        !prolong_fusable(ctx->cfg.precision, ctx->cfg.overlap, 0))
        return DI_ERR_INVALID_ARG;
    const size_t bytes = (size_t)width * height * channels * sizeof(float);
    int wH, hH;
    coarse_dims(width, height, &wH, &hH);
    const size_t bytesH = (size_t)wH * hH * channels * sizeof(float);
    if (overlaps(u_in, bytes, u_out, bytes) || overlaps(uH, bytesH, u_out, bytes))
        return DI_ERR_INVALID_ARG;
    DI_CUDA(ctx, cudaSetDevice(ctx->device));
    di_status st = ensure_workspace(ctx, width, height, channels);
    if (st) return st;
    bind_levels(ctx, b, c, u_out, width, height, channels);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* bits = ctx->lv[0].mbits;
    DI_CUDA(ctx, launch_pack_mask(c, width, height, bits, nullptr, s));
    DI_CUDA(ctx, launch_oras(u_in, 0, b, rhs_zero ? 1 : 0, bits, width, height, channels, 32,
                             ctx->cfg.overlap, ctx->cfg.alpha, local_iters, 0.f, u_out,
                             ctx->planes, nullptr, s, nullptr, ctx->cfg.precision,
                             ctx->upd + kMaxUpdSlots, nullptr, kF32, ctx->cfg.refine_fp64 != 0,
                             uH, nullptr, mode));
    return DI_OK;
}

di_status di_selftest_bounded_wait(int device, int limit, void* stream) {
    if (limit < 1) return DI_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DI_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned* flag = nullptr;
    unsigned h = 0;
    di_status st = DI_OK;
    if (cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess) return DI_ERR_OOM;
    if (cudaMemsetAsync(flag, 0, sizeof(unsigned), s) != cudaSuccess ||
        launch_wait_selftest(flag, limit, s) != cudaSuccess ||
        cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        st = DI_ERR_CUDA;
    cudaFree(flag);
    if (st != DI_OK) return st;
    return h == 1 ? DI_ERR_TIMEOUT : h == 2 ? DI_OK : DI_ERR_CUDA;
}

}  // extern "C"

// The batched form of the decoder: many images of uneven sizes decoded
// together, with one launch per step of the method over every image of the
// batch and the whole batch captured once as one CUDA graph.
//
// The steps run in lockstep over the levels (level 0 the finest of every
// image): the pyramid (mask downsampling, value downsampling, packed masks
// and unknown counts, Section 4.3) one launch per level; the plan kernel (per
// image: levels in use, the cascade's start level); the cascade of the
// reduced FMG (Section 4.2) from the deepest level up, per level one start
// (select), one prolongation and one block-kernel launch; then a WHILE node
// whose body is one V(1,1)-cycle (Algorithm 3 applied recursively; per level
// a restriction and a block-kernel launch down, a block-kernel launch and a
// prolongation up) followed by the stop test of every image.  An image takes
// part in a step according to its own levels in use and pyramid depth, and
// drops out of the cycles once its stop rule holds; the loop ends when no
// image runs.  Each image's arithmetic is that of its single-image decode
// (the same kernels' bodies and the same order), so a result does not
// depend on what else is in the batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/di.h"
#include "di_internal.h"

using namespace di;

namespace {

constexpr float kCoarseRtol2B = 1e-12f;  // the coarsest single-block solve (as di_inpaint)
constexpr size_t kAlignB = 256;
size_t align_b(size_t x) { return (x + kAlignB - 1) / kAlignB * kAlignB; }

struct BLevel {
    int w = 0, h = 0;
    size_t n = 0;
    const uint8_t* c = nullptr;
    const float* b = nullptr;
    float* u[2] = {nullptr, nullptr};
    float* r = nullptr;
    uint32_t* mbits = nullptr;
};

struct BImage {
    int w = 0, h = 0, C = 0, L = 0;
    float tol = 0.f;
    const float* f = nullptr;
    const uint8_t* c = nullptr;
    float* u = nullptr;
    BLevel lv[kMaxLevels];
};

// One launch of the graph: its kind and its segments' range in the table.
struct Launch {
    int kind;  // BatchKind, or -1 for the block kernel
    int seg0, nseg, nwork;
};

}  // namespace

struct di_batch {
    di_config cfg;
    int device = 0;
    int n = 0;
    std::vector<BImage> im;
    void* pool = nullptr;      // level buffers of every image
    void* state = nullptr;     // per-image device state
    BatchSeg* dsegs = nullptr; // every launch's segments
    void* dmaps = nullptr;     // tensor maps of the block-kernel segments (kTileMapsBytes each)
    int* dL = nullptr;
    unsigned long long* dn0 = nullptr;
    BatchState bs;
    StopState* hstate = nullptr;  // pinned read-back
    cudaStream_t cap = nullptr;
    cudaStream_t cap2 = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long k_fixed = 0, k_cycle = 0;  // kernels outside the loop, and per loop iteration
};

namespace {

bool batch_config_ok(const di_config& c) {
    return c.block == 32 && c.overlap == 2 && c.precision == DI_PREC_FP32 && !c.refine_fp64 &&
           c.smoother == DI_SMOOTH_ORAS && c.schedule == DI_SCHED_REDUCED_FMG &&
           c.start == DI_START_CASCADE && c.pre == 1 && c.post == 1 &&
           (c.stop_rule == DI_STOP_ERROR_ESTIMATE || c.stop_rule == DI_STOP_FIXED_CYCLES) &&
           c.graph == DI_GRAPH_ON && !c.profile && c.max_cycles > 0;
}

void free_batch(di_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->g) cudaGraphDestroy(b->g);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->cap2) cudaStreamDestroy(b->cap2);
    if (b->pool) cudaFree(b->pool);
    if (b->state) cudaFree(b->state);
    if (b->dsegs) cudaFree(b->dsegs);
    if (b->dmaps) cudaFree(b->dmaps);
    if (b->hstate) cudaFreeHost(b->hstate);
    delete b;
}

// Lay out every image's level buffers in one allocation.
bool alloc_levels(di_batch* b) {
    size_t total = 0;
    for (int pass = 0; pass < 2; ++pass) {
        char* p = static_cast<char*>(b->pool);
        size_t off = 0;
        auto take = [&](size_t bytes) -> char* {
            char* q = pass ? p + off : nullptr;
            off += align_b(bytes);
            return q;
        };
        for (auto& I : b->im) {
            int lw = I.w, lh = I.h;
            for (int l = 0; l < I.L; ++l) {
                BLevel& v = I.lv[l];
                v.w = lw;
                v.h = lh;
                v.n = (size_t)lw * lh;
                const size_t fb = v.n * I.C * sizeof(float);
                v.mbits = reinterpret_cast<uint32_t*>(take((size_t)lh * mask_words_per_row(lw) * 4));
                if (l == 0) {
                    v.c = I.c;
                    v.b = I.f;
                    v.u[0] = I.u;
                    v.u[1] = reinterpret_cast<float*>(take(fb));
                    v.r = nullptr;
                } else {
                    v.c = reinterpret_cast<uint8_t*>(take(v.n));
                    v.b = reinterpret_cast<float*>(take(fb));
                    v.u[0] = reinterpret_cast<float*>(take(fb));
                    v.u[1] = reinterpret_cast<float*>(take(fb));
                    v.r = reinterpret_cast<float*>(take(fb));
                }
                coarse_dims(lw, lh, &lw, &lh);
            }
        }
        if (pass == 0) {
            total = off;
            if (cudaMalloc(&b->pool, total > 0 ? total : 1) != cudaSuccess) return false;
        }
    }
    return true;
}

// The segment tables of every launch, in graph order, and the graph.
struct alignas(64) TileMaps {
    unsigned char bytes[kTileMapsBytes];
};

struct Builder {
    di_batch* b;
    std::vector<BatchSeg> segs;
    std::vector<Launch> launches;
    std::vector<TileMaps> maps;  // a block segment with tma = 1 holds its index in tmaps
    int Lmax = 0;

    BatchSeg base(int img, int level, int when) const {
        BatchSeg s;
        std::memset(&s, 0, sizeof s);
        s.img = img;
        s.level = level;
        s.when = when;
        s.L = b->im[img].L;
        return s;
    }
    // a grid-kernel segment over the level of size (w, h) with `planes` planes
    void add_grid(std::vector<BatchSeg>& v, BatchSeg s, int kind, int w, int h, int planes,
                  int* cta) {
        batch_grid_dims(kind, w, h, &s.gx, &s.gy);
        s.w = w;
        s.h = h;
        s.first = *cta;
        *cta += s.gx * s.gy * planes;
        v.push_back(s);
    }
    void push(int kind, std::vector<BatchSeg>& v, int nwork) {
        if (v.empty() || nwork < 1) return;
        launches.push_back({kind, (int)segs.size(), (int)v.size(), nwork});
        segs.insert(segs.end(), v.begin(), v.end());
    }
    // a block-kernel segment of image i on level l (in -> out)
    // pro_e, pro_mode, pro_max, pro_check: the start prolonged from level
    // l + 1 inside the block kernel (BatchSeg)
    void add_oras(std::vector<BatchSeg>& v, int i, int l, int when, const float* in, int zero_in,
                  const float* rhs, int rhs_zero, float* out, int iters, float rtol2,
                  unsigned* maxupd, int* units, const float* pro_e = nullptr, int pro_mode = 0,
                  unsigned* pro_max = nullptr, int pro_check = 0) {
        const BLevel& lv = b->im[i].lv[l];
        BatchSeg s = base(i, l, when);
        s.w = lv.w;
        s.h = lv.h;
        s.C = b->im[i].C;
        s.in0 = in;
        s.in1 = rhs;
        s.out0 = out;
        s.zero_in = zero_in;
        s.rhs_zero = rhs_zero;
        s.iters = iters;
        s.rtol2 = rtol2;
        s.maxupd = maxupd;
        s.mbits = lv.mbits;
        s.wpr = mask_words_per_row(lv.w);
        s.nbx = axis_blocks(lv.w, 32, b->cfg.overlap);
        s.nby = axis_blocks(lv.h, 32, b->cfg.overlap);
        s.pro_e = pro_e;
        s.pro_mode = pro_e ? pro_mode : 0;
        s.pro_max = pro_max;
        s.pro_check = pro_check;
        TileMaps tm;
        if (make_tile_maps(&tm, in, zero_in, rhs, rhs_zero, lv.w, lv.h, s.C)) {
            s.tma = 1;
            s.tmaps = reinterpret_cast<const void*>(static_cast<uintptr_t>(maps.size()));
            maps.push_back(tm);
        }
        s.first = *units;
        *units += s.nbx * s.nby;
        v.push_back(s);
    }
    unsigned* upd(int i, int slot) const {
        return b->bs.upd + (size_t)i * (kMaxUpdSlots + 1) + slot;
    }
    float abs2(int i) const {
        const di_config& c = b->cfg;
        if (c.stop_rule != DI_STOP_ERROR_ESTIMATE || !(c.local_stop > 0.f)) return 0.f;
        const float a = c.local_stop * b->im[i].tol;
        return -(a * a);
    }
    int K(int l) const {
        const di_config& c = b->cfg;
        return l > 0 && c.local_iters_coarse > 0 ? c.local_iters_coarse : c.local_iters;
    }
    // the cascade's smoothing step on level l
    int Kc(int l) const {
        const di_config& c = b->cfg;
        return l == 0 && c.local_iters_cascade > 0 ? c.local_iters_cascade : K(l);
    }

    void build_tables() {
        const di_config& cfg = b->cfg;
        const int n = b->n;
        for (auto& I : b->im) Lmax = std::max(Lmax, I.L);
        // 1. pyramid: packed finest masks, then per level
        {
            std::vector<BatchSeg> v;
            int cta = 0;
            for (int i = 0; i < n; ++i) {
                const BLevel& l0 = b->im[i].lv[0];
                BatchSeg s = base(i, 0, kWhenAlways);
                s.in0 = l0.c;
                s.mbits = l0.mbits;
                s.wpr = mask_words_per_row(l0.w);
                s.counter = b->bs.counts + (size_t)i * (kMaxLevels + 1) + 1;
                add_grid(v, s, kBPack, l0.w, l0.h, 1, &cta);
            }
            push(kBPack, v, cta);
        }
        for (int l = 1; l < Lmax; ++l) {
            // level l in one pass: mask, mask values, packed words, unknown count
            std::vector<BatchSeg> v;
            int cta = 0;
            for (int i = 0; i < n; ++i) {
                const BImage& I = b->im[i];
                if (l >= I.L) continue;
                const BLevel& fl = I.lv[l - 1];
                const BLevel& cl = I.lv[l];
                BatchSeg s = base(i, l, kWhenAlways);
                s.in0 = fl.c;
                s.in1 = fl.b;
                s.out0 = const_cast<uint8_t*>(cl.c);
                s.out1 = const_cast<float*>(cl.b);
                s.C = I.C;
                s.mode = cfg.downsample == 0 ? 1 : 0;
                s.mbits = cl.mbits;
                s.wpr = mask_words_per_row(cl.w);
                s.counter = b->bs.counts + (size_t)i * (kMaxLevels + 1) + 1 + l;
                add_grid(v, s, kBPyramid, fl.w, fl.h, 1, &cta);
            }
            push(kBPyramid, v, cta);
        }
    }

    // the cascade and the cycle body, as (kind, segments) lists
    void build_cascade() {
        const int n = b->n;
        for (int l = Lmax - 1; l >= 0; --l) {
            std::vector<BatchSeg> sel, ora;
            int c1 = 0, units = 0;
            for (int i = 0; i < n; ++i) {
                const BImage& I = b->im[i];
                if (l >= I.L) continue;
                const BLevel& v = I.lv[l];
                // the start on this level: u = b in both buffers
                BatchSeg s = base(i, l, kWhenTopEq);
                s.in1 = v.b;
                s.in2 = v.c;
                s.out0 = v.u[0];
                s.out1 = v.u[1];
                s.C = I.C;
                add_grid(sel, s, kBSelect, v.w, v.h, I.C, &c1);
                if (l + 1 < I.L) {
                    // the coarser level's solution interpolated inside the
                    // smoothing step: b on the mask, P u_{l+1} elsewhere
                    const BLevel& cv = I.lv[l + 1];
                    add_oras(ora, i, l, kWhenBelowTop, v.b, 0, v.b, 1, v.u[0], Kc(l), abs2(i),
                             nullptr, &units, cv.u[0], 2);
                } else {  // the coarsest level: the single-block solve of the start
                    add_oras(ora, i, l, kWhenCoarsestStart, v.u[1], 0, v.b, 1, v.u[0],
                             b->cfg.coarse_iters, kCoarseRtol2B, nullptr, &units);
                }
            }
            push(kBSelect, sel, c1);
            push(-1, ora, units);
        }
    }

    void build_cycle() {
        const int n = b->n;
        // level 0 pre-smoothing: u[0] -> u[1]
        {
            std::vector<BatchSeg> ora;
            int units = 0;
            for (int i = 0; i < n; ++i) {
                const BLevel& v = b->im[i].lv[0];
                add_oras(ora, i, 0, kWhenCycle, v.u[0], 0, v.b, 1, v.u[1], K(0), abs2(i),
                         upd(i, 0), &units);
            }
            push(-1, ora, units);
        }
        // down: restriction into level l, then its pre-smoothing (or the
        // coarsest solve), both from zero
        for (int l = 1; l < Lmax; ++l) {
            std::vector<BatchSeg> res, ora;
            int c1 = 0, units = 0;
            for (int i = 0; i < n; ++i) {
                const BImage& I = b->im[i];
                if (l >= I.L) continue;
                const BLevel& fl = I.lv[l - 1];
                const BLevel& v = I.lv[l];
                BatchSeg s = base(i, l, kWhenCycle);
                s.in0 = fl.u[1];
                s.in1 = l - 1 == 0 ? fl.b : fl.r;
                s.rhs_zero = l - 1 == 0 ? 1 : 0;
                s.in2 = v.c;
                s.out0 = v.r;
                s.C = I.C;
                add_grid(res, s, kBRestrict, fl.w, fl.h, I.C, &c1);
                if (l == I.L - 1)
                    add_oras(ora, i, l, kWhenCycle, v.u[0], 1, v.r, 0, v.u[1],
                             b->cfg.coarse_iters, kCoarseRtol2B, nullptr, &units);
                else
                    add_oras(ora, i, l, kWhenCycle, v.u[0], 1, v.r, 0, v.u[1], K(l), abs2(i),
                             nullptr, &units);
            }
            push(kBRestrict, res, c1);
            push(-1, ora, units);
        }
        // up: the post-smoothing of every level that has a coarser one, with
        // that level's correction prolonged into its start inside the block
        // kernel (while the coarser level is in use for the image); level 0
        // of an image without coarser levels smooths plainly
        for (int l = Lmax - 2; l >= 0; --l) {
            std::vector<BatchSeg> ora;
            int units = 0;
            for (int i = 0; i < n; ++i) {
                const BImage& I = b->im[i];
                const BLevel& v = I.lv[std::min(l, I.L - 1)];
                if (l + 1 < I.L) {
                    const BLevel& cv = I.lv[l + 1];
                    const float* e = l + 1 == I.L - 1 ? cv.u[1] : cv.u[0];
                    if (l == 0)
                        add_oras(ora, i, 0, kWhenCycle, v.u[1], 0, v.b, 1, v.u[0], K(0), abs2(i),
                                 upd(i, 2), &units, e, 1, upd(i, 1), 1);
                    else
                        add_oras(ora, i, l, kWhenCycle, v.u[1], 0, v.r, 0, v.u[0], K(l), abs2(i),
                                 nullptr, &units, e, 1, nullptr, 1);
                } else if (l == 0) {
                    add_oras(ora, i, 0, kWhenCycle, v.u[1], 0, v.b, 1, v.u[0], K(0), abs2(i),
                             upd(i, 2), &units);
                }
            }
            push(-1, ora, units);
        }
        if (Lmax == 1) {  // every image has one level: its post-smoothing alone
            std::vector<BatchSeg> ora;
            int units = 0;
            for (int i = 0; i < n; ++i) {
                const BLevel& v = b->im[i].lv[0];
                add_oras(ora, i, 0, kWhenCycle, v.u[1], 0, v.b, 1, v.u[0], K(0), abs2(i),
                         upd(i, 2), &units);
            }
            push(-1, ora, units);
        }
    }

    cudaError_t run(const Launch& L, cudaStream_t s) {
        const BatchSeg* d = b->dsegs + L.seg0;
        if (L.kind < 0)
            return launch_batch_oras(d, L.nseg, L.nwork, b->cfg.overlap, b->cfg.alpha, b->bs, s);
        return launch_batch_grid(L.kind, d, L.nseg, L.nwork, b->bs, s);
    }
};

}  // namespace

extern "C" di_status di_batch_create(const di_config* cfg, int device, const di_image* imgs,
                                     int n, di_batch** out) {
    if (!out || !imgs || n < 1) return DI_ERR_INVALID_ARG;
    *out = nullptr;
    di_config c;
    std::memset(&c, 0, sizeof c);
    if (cfg) c = *cfg;
    di_plan_info plan;
    if (di_plan(&c, 1, 1, 1, &plan) != DI_OK) return DI_ERR_INVALID_ARG;
    // the defaults of a zero field, as di_create resolves them
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
    if (!batch_config_ok(c)) return DI_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const di_image& m = imgs[i];
        if (!m.f || !m.c || !m.u || m.width < 1 || m.height < 1 || m.channels < 1 ||
            m.channels > kMaxChannels || !(m.tol > 0.f) || !std::isfinite(m.tol))
            return DI_ERR_INVALID_ARG;
        const int L = num_levels(m.width, m.height, 32);
        if (L < 2 || L > kMaxLevels - 1) return DI_ERR_INVALID_ARG;  // one block: di_inpaint
    }
    if (cudaSetDevice(device) != cudaSuccess) return DI_ERR_CUDA;
    di_batch* b = new (std::nothrow) di_batch();
    if (!b) return DI_ERR_OOM;
    b->cfg = c;
    b->device = device;
    b->n = n;
    b->im.resize(n);
    std::vector<int> Ls(n);
    std::vector<unsigned long long> n0s(n);
    std::vector<float> tols(n);
    for (int i = 0; i < n; ++i) {
        BImage& I = b->im[i];
        I.w = imgs[i].width;
        I.h = imgs[i].height;
        I.C = imgs[i].channels;
        I.L = num_levels(I.w, I.h, 32);
        I.tol = imgs[i].tol;
        I.f = imgs[i].f;
        I.c = imgs[i].c;
        I.u = imgs[i].u;
        Ls[i] = I.L;
        n0s[i] = (unsigned long long)I.w * I.h;
        tols[i] = I.tol;
    }
    // per-image state: leff, top, done, L, tol | n0 | StopState | upd | counts | err
    const size_t ints = (size_t)5 * n * sizeof(int);
    const size_t o_n0 = align_b(ints);
    const size_t o_st = o_n0 + align_b((size_t)n * sizeof(unsigned long long));
    const size_t o_upd = o_st + align_b((size_t)n * sizeof(StopState));
    const size_t o_cnt = o_upd + align_b((size_t)n * (kMaxUpdSlots + 1) * sizeof(unsigned));
    const size_t o_err = o_cnt + align_b((size_t)n * (kMaxLevels + 1) * sizeof(unsigned long long));
    const size_t state_bytes = o_err + sizeof(unsigned);
    if (!alloc_levels(b) || cudaMalloc(&b->state, state_bytes) != cudaSuccess ||
        cudaMallocHost(&b->hstate, (size_t)n * sizeof(StopState)) != cudaSuccess) {
        free_batch(b);
        return DI_ERR_OOM;
    }
    char* sp = static_cast<char*>(b->state);
    b->bs.leff = reinterpret_cast<int*>(sp);
    b->bs.top = b->bs.leff + n;
    b->bs.done = b->bs.top + n;
    b->dL = b->bs.done + n;
    float* dtol = reinterpret_cast<float*>(b->dL + n);
    b->bs.tol = dtol;
    b->dn0 = reinterpret_cast<unsigned long long*>(sp + o_n0);
    b->bs.st = reinterpret_cast<StopState*>(sp + o_st);
    b->bs.upd = reinterpret_cast<unsigned*>(sp + o_upd);
    b->bs.counts = reinterpret_cast<unsigned long long*>(sp + o_cnt);
    b->bs.err = reinterpret_cast<unsigned*>(sp + o_err);
    if (cudaMemcpy(b->dL, Ls.data(), n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dtol, tols.data(), n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dn0, n0s.data(), n * sizeof(unsigned long long), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        free_batch(b);
        return DI_ERR_CUDA;
    }
    // segment tables of every launch
    Builder B{b};
    B.build_tables();
    const size_t n_pyr = B.launches.size();
    B.build_cascade();
    const size_t n_casc = B.launches.size();
    B.build_cycle();
    // the block segments' tensor maps, then their device addresses in the tables
    if (!B.maps.empty()) {
        if (cudaMalloc(&b->dmaps, B.maps.size() * sizeof(TileMaps)) != cudaSuccess ||
            cudaMemcpy(b->dmaps, B.maps.data(), B.maps.size() * sizeof(TileMaps),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            free_batch(b);
            return DI_ERR_OOM;
        }
        for (auto& sg : B.segs)
            if (sg.tma)
                sg.tmaps = static_cast<const TileMaps*>(b->dmaps) +
                           reinterpret_cast<uintptr_t>(sg.tmaps);
    }
    if (cudaMalloc(&b->dsegs, B.segs.size() * sizeof(BatchSeg)) != cudaSuccess ||
        cudaMemcpy(b->dsegs, B.segs.data(), B.segs.size() * sizeof(BatchSeg),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        free_batch(b);
        return DI_ERR_OOM;
    }
    // the graph: pyramid, plan, cascade, then the cycle loop
    StopParams sp_;
    sp_.rule = c.stop_rule;
    sp_.nslots = c.pre + 1 + c.post;
    sp_.min_cycles = c.min_cycles;
    sp_.max_cycles = c.max_cycles;
    sp_.C = 0;
    sp_.tol = 0.f;
    cudaGraphConditionalHandle h = 0;
    bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking) == cudaSuccess &&
              cudaGraphCreate(&b->g, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&h, b->g, 1, cudaGraphCondAssignDefault) ==
                  cudaSuccess;
    const long long k0 = thread_launch_count();
    long long k_loop0 = 0, k_loop1 = 0;
    if (ok)
        ok = cudaStreamBeginCaptureToGraph(b->cap, b->g, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
        cudaStream_t s = b->cap;
        bool rok = cudaMemsetAsync(b->bs.counts, 0,
                                   (size_t)n * (kMaxLevels + 1) * sizeof(unsigned long long),
                                   s) == cudaSuccess;
        for (size_t k = 0; rok && k < n_pyr; ++k) rok = B.run(B.launches[k], s) == cudaSuccess;
        if (rok) rok = launch_batch_plan(n, b->dL, b->dn0, b->bs, s) == cudaSuccess;
        for (size_t k = n_pyr; rok && k < n_casc; ++k) rok = B.run(B.launches[k], s) == cudaSuccess;
        if (rok) {
            // the V-cycle loop: a WHILE node after what was captured so far
            cudaStreamCaptureStatus cs;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            rok = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd) ==
                  cudaSuccess;
            cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
            p.conditional.handle = h;
            p.conditional.type = cudaGraphCondTypeWhile;
            p.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            if (rok) rok = cudaGraphAddNode(&node, cg, deps, nullptr, nd, &p) == cudaSuccess;
            if (rok)
                rok = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                                          cudaStreamSetCaptureDependencies) ==
                      cudaSuccess;
            if (rok)
                rok = cudaStreamBeginCaptureToGraph(b->cap2, p.conditional.phGraph_out[0],
                                                    nullptr, nullptr, 0,
                                                    cudaStreamCaptureModeRelaxed) == cudaSuccess;
            if (rok) {
                k_loop0 = thread_launch_count();
                for (size_t k = n_casc; rok && k < B.launches.size(); ++k)
                    rok = B.run(B.launches[k], b->cap2) == cudaSuccess;
                if (rok) rok = launch_batch_stop(n, sp_, b->bs, h, b->cap2) == cudaSuccess;
                k_loop1 = thread_launch_count();
                cudaGraph_t body = nullptr;
                rok = cudaStreamEndCapture(b->cap2, &body) == cudaSuccess && rok;
            }
        }
        cudaGraph_t outg = nullptr;
        ok = cudaStreamEndCapture(s, &outg) == cudaSuccess && rok;
    }
    b->k_cycle = k_loop1 - k_loop0;
    b->k_fixed = thread_launch_count() - k0 - b->k_cycle;
    add_launches(-(thread_launch_count() - k0));  // captured, not launched
    if (ok) ok = cudaGraphInstantiate(&b->exec, b->g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(b);
        return DI_ERR_CUDA;
    }
    *out = b;
    return DI_OK;
}

extern "C" di_status di_batch_run(di_batch* b, di_image* imgs, int n, void* stream) {
    if (!b || !imgs || n != b->n) return DI_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const BImage& I = b->im[i];
        const di_image& m = imgs[i];
        if (m.f != I.f || m.c != I.c || m.u != I.u || m.width != I.w || m.height != I.h ||
            m.channels != I.C || m.tol != I.tol)
            return DI_ERR_INVALID_ARG;  // not the batch the graph was built for
    }
    if (cudaSetDevice(b->device) != cudaSuccess) return DI_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned err = 0;
    if (cudaMemsetAsync(b->bs.err, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaGraphLaunch(b->exec, s) != cudaSuccess ||
        cudaMemcpyAsync(b->hstate, b->bs.st, (size_t)n * sizeof(StopState),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(&err, b->bs.err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
        return DI_ERR_CUDA;
    if (err) {  // a bounded wait of the block kernel ran out: nothing of the run is valid
        for (int i = 0; i < n; ++i) imgs[i].status = DI_ERR_TIMEOUT;
        return DI_ERR_TIMEOUT;
    }
    di_status worst = DI_OK;
    int iters = 1;  // the loop body runs at least once
    for (int i = 0; i < n; ++i) {
        const StopState& h = b->hstate[i];
        imgs[i].status = h.status;
        imgs[i].cycles = h.cycles;
        iters = std::max(iters, h.cycles);
        if (h.status != DI_OK && worst == DI_OK) worst = (di_status)h.status;
    }
    add_launches(b->k_fixed + b->k_cycle * iters);
    return worst;
}

extern "C" void di_batch_destroy(di_batch* b) { free_batch(b); }

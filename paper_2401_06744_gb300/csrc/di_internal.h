// Launch wrappers shared between the kernel translation unit and the host
// scheduler.  All pointers are device pointers; images are planar
// [C][h][w] float32, masks [h][w] uint8.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace di {

constexpr int kMaxChannels = 4;

inline int axis_blocks_decl(int n, int B, int o) {
    const int s = B - o;
    const int nb = (n - o + s - 1) / s;
    return nb < 1 ? 1 : nb;
}

// Kernels enqueued by the launch wrappers below (process-wide counter), and
// those the calling thread enqueued (for counting the kernels of a capture).
long long launch_count();
long long thread_launch_count();
// Adjust the launch counter (graph replays add their kernels, captures that
// launched nothing take theirs back).
void add_launches(long long k);
constexpr int kMaxLevels = 24;
constexpr int kMaxUpdSlots = 16;

// Storage of the iterate and right-hand-side arrays a kernel reads or writes:
// FP32, or FP16 / BF16 (the coarse levels in the 16-bit precision modes; the
// values match DI_PREC_*).  Arithmetic is FP32 (or FP64 where stated).
enum Storage { kF32 = 0, kF16 = 1, kBF16 = 2 };
inline size_t storage_bytes(int stor) { return stor == kF32 ? 4 : 2; }

// cH = 2x2 max pool of c.
cudaError_t launch_mask_down(const uint8_t* c, int w, int h, uint8_t* cH, cudaStream_t s);

// bH from (c, b, cH): modified (1) or naive (0) mask-value downsampling.
cudaError_t launch_values_down(const uint8_t* c, const float* b, int w, int h, int C,
                               const uint8_t* cH, float* bH, int modified, cudaStream_t s);

// r = b - A u (r may be null) and per-CTA partial sums of r^2 into
// partials[ch * nparts + cta]; returns nparts through *nparts.  f64: the
// residual formed in FP64 (the finest-grid refinement residual).
cudaError_t launch_residual(const float* u, int zero_u, const float* b, int rhs_zero,
                            const uint8_t* c, int w, int h, int C, float* r, double* partials,
                            int* nparts, cudaStream_t s, bool f64 = false);
size_t residual_partials_per_channel(int w, int h);

// The same residual + norm with the partial sums in the library's static
// device array (capacity kNoAllocPartials doubles, checked by the caller).
constexpr long long kNoAllocPartials = 131072;
cudaError_t launch_residual_noalloc(const float* u, const float* b, int rhs_zero,
                                    const uint8_t* c, int w, int h, int C, float* r,
                                    double* norm2, cudaStream_t s);

// out[ch] = sum of partials[ch * nparts + i] in a fixed order.
cudaError_t launch_reduce_partials(const double* partials, int nparts, int C, double* out,
                                   cudaStream_t s);

// rH = 4 * mean over children of (b - A u) where cH == 0, else 0.  u, b and
// rH are stored as su, sb, sr (Storage); f64: the children's residuals in FP64.
cudaError_t launch_restrict(const float* u, const float* b, int rhs_zero, const uint8_t* c,
                            int w, int h, int C, const uint8_t* cH, float* rH, cudaStream_t s,
                            int su = kF32, int sb = kF32, int sr = kF32, bool f64 = false);

// mode 0: u = c ? b : P uH.  mode 1: u += c ? 0 : P uH, max |P uH| (unknown
// pixels) folded into *maxupd (as float bits, nullable).  uH and u are stored
// as suH and su; b is FP32.
cudaError_t launch_prolong(const float* uH, const float* b, const uint8_t* c, int w, int h,
                           int C, float* u, int mode, unsigned* maxupd, cudaStream_t s,
                           int suH = kF32, int su = kF32);

// u = c ? b : 0 (keep = 0) or u = c ? b : u (keep = 1); u stored as su.
cudaError_t launch_select(const float* b, const uint8_t* c, int w, int h, int C, float* u,
                          cudaStream_t s, int keep = 0, int su = kF32);

// One CTA waits, with the block kernel's bounded mbarrier wait (`limit`
// polls), on a barrier nothing completes; *flag = 1 when the wait ran out.
cudaError_t launch_wait_selftest(unsigned* flag, int limit, cudaStream_t s);

// One pyramid level in one launch: cH = 2x2 max pool of c, bH the mask-value
// downsampling of (c, b) (modified = 1, or naive; values = 0: skipped), bits
// the bit-packed cH, *unknown (nullable, zeroed by the caller) gains the
// coarse level's unknown pixels.  Bit-identical to mask_down + values_down +
// pack_mask.
cudaError_t launch_pyramid_level(const uint8_t* c, const float* b, int w, int h, int C,
                                 uint8_t* cH, float* bH, int modified, int values, uint32_t* bits,
                                 unsigned long long* unknown, cudaStream_t s);

// Bit-packed mask (see mask_words_per_row) of c; *unknown (nullable, zeroed
// by the caller) gains the number of unknown pixels.
cudaError_t launch_pack_mask(const uint8_t* c, int w, int h, uint32_t* bits,
                             unsigned long long* unknown, cudaStream_t s);

// Floats of ORAS scratch for an image of w x h x C: four parity planes of
// pixels shared along y, then the compact strips of pixels shared along x only.
inline size_t oras_scratch_floats(int w, int h, int C, int B, int o) {
    const int nsh = o == 1 ? 1 : (o > 2 ? o - 2 : 0);
    const int nbx = axis_blocks_decl(w, B, o);
    return 4 * (size_t)w * h * C + 2 * (size_t)C * (nbx > 1 ? nbx - 1 : 0) * h * (nsh > 0 ? nsh : 1);
}

// One ORAS iteration u_in -> u_out (planes: oras_scratch_floats of workspace;
// mbits: the packed mask of this level).  Each local CG runs `iters` steps or
// until r.r <= max(rtol2, 1e-14) * (r.r)_0 (rtol2 >= 0), or until
// r.r <= max(1e-14 (r.r)_0, -rtol2) (rtol2 < 0: an absolute level, per block
// and channel, summed over the block's pixels).  max |v_i| over pixels with
// nonzero weight is folded into *maxupd (nullable).
// ev (nullable): two events recorded on `s` right before and right after the
// block kernel (the combine kernels follow the second one).  precision: 0
// FP32, 1 FP16, 2 BF16 local CG iterates (32x32 blocks; other sizes use FP32).
// errflag (nullable): set to 1 when a bounded device-side wait of the FP32
// 32x32 kernel ran out (its tile copies did not arrive).  step_count
// (nullable): gains the local CG steps completed, summed over the tasks.
// stor: storage of u_in, rhs and u_out (kF32, or on the coarse levels of the
// 16-bit modes the precision's type; 32x32 blocks only); f64: the block
// residual in FP64.  pro_e (nullable): the next coarser level's FP32 field,
// prolonged into the iteration's start, bit-identical to launch_prolong
// followed by the plain iteration: pro_mode 1 adds P e to u_in at the unknown
// pixels (the V-cycle's correction step; the largest |P e| into *pro_max,
// nullable), pro_mode 0 takes u_in at the known pixels and P e at the others
// (the cascade's interpolation, u_in = b); only where prolong_fusable() holds.
cudaError_t launch_oras(const float* u_in, int zero_in, const float* rhs, int rhs_zero,
                        const uint32_t* mbits, int w, int h, int C, int B, int o, float alpha,
                        int iters, float rtol2, float* u_out, float* planes, unsigned* maxupd,
                        cudaStream_t s, cudaEvent_t* ev = nullptr, int precision = 0,
                        unsigned* errflag = nullptr, unsigned long long* step_count = nullptr,
                        int stor = kF32, bool f64 = false, const float* pro_e = nullptr,
                        unsigned* pro_max = nullptr, int pro_mode = 1);

// Whether the 32x32 block kernel can take the correction's prolongation:
// FP32 iterates, an even block stride 32 - o (the pixel parities of every
// block are those of its tile) and a given iterate.
inline bool prolong_fusable(int precision, int o, int zero_in) {
    return precision == 0 && ((32 - o) & 1) == 0 && !zero_in;
}

// Global CG smoother: `steps` CG steps on the level's reduced system from the
// iterate `in`, out = in + correction; restart = 0 continues the previous
// call's CG state (r, p, sc, *step_par) on the same level.  r, p, q, x: C*w*h
// floats each; sc: 4*C doubles; partials as for launch_residual.
cudaError_t launch_cg_smooth(const float* in, int zero_in, const float* b, int rhs_zero,
                             const uint8_t* c, int w, int h, int C, int steps, int restart,
                             float* r, float* p, float* q, float* x, double* partials, double* sc,
                             int* step_par, float* out, unsigned* maxupd, cudaStream_t s);

// ---------------------------------------------------------------------------
// Device-driven decode: the state of the stop test lives on the device, so a
// whole decode runs as one CUDA graph without host round trips.
// ---------------------------------------------------------------------------

// Stop-test state of one decode (device memory, read back once at the end).
struct StopState {
    int cycles;          // V-cycles run
    int status;          // di_status of the decode
    int converged;       // 1 once the stop rule held
    int levels_used;     // levels down to the first one without unknown pixels
    float est;           // last error estimate (gray levels)
    float prevU, prevQ;  // last cycle's update size and decay ratio (< 0: none yet)
    float rel[kMaxChannels];       // relative residual per channel (relative-residual rule)
    unsigned long long unknowns;   // unknown pixels on the finest level
    double bnorm2[kMaxChannels];   // ||b||^2 per channel (relative-residual rule)
    double norm2[kMaxChannels];    // ||b - A u||^2 per channel of the last cycle
};

// Stop rule parameters (rule: the DI_STOP_* value of the configuration).
struct StopParams {
    int rule, nslots, min_cycles, max_cycles, C;
    float tol;
};

// Conditional handles of the decode graph.  h_sel picks the body for the
// number of levels in use (0: every pixel known, u = f; v >= 1: the cascade
// and the V-cycle loop recursing through v levels; kSelSkip: the empty mask,
// no body); h_loop[v] is the WHILE handle of body v's V-cycle loop.
constexpr unsigned kSelSkip = 0xffffu;

struct PlanParams {
    int L;                     // levels of the pyramid
    int max_cycles;
    unsigned long long n0;     // pixels of the finest level
    unsigned long long h_sel;                  // SWITCH over the levels in use
    unsigned long long h_loop[kMaxLevels + 1]; // WHILE handles, per body
};

// Levels in use and branch values of the decode from the unknown counts
// (counts[1 + l]: unknown pixels of level l); initialises *st.
cudaError_t launch_plan(const unsigned long long* counts, StopState* st, const PlanParams& p,
                        cudaStream_t s);
// The stop test after one V-cycle: reads and clears the update slots
// (upd[0 .. nslots-1]; upd[kMaxUpdSlots] is the timeout flag), updates *st
// and sets the loop handle to 0 once the decode is done.
cudaError_t launch_stop(unsigned* upd, StopState* st, const StopParams& p,
                        unsigned long long h_loop, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched form: one launch per step over the images of a batch.  Each image's
// part of a launch is a segment: its level's size and buffers, its first CTA
// (grid kernels) or first block unit (the block kernel) in the launch, and
// when it takes part, which depends on the image's levels in use, the start
// level of its cascade and whether its decode has converged -- values the
// batch's plan and stop kernels keep on the device.
// ---------------------------------------------------------------------------

enum BatchWhen {
    kWhenAlways = 0,         // pyramid steps
    kWhenTopEq = 1,          // cascade start: level == the image's start level
    kWhenCoarsestStart = 2,  // cascade start on the coarsest level (all levels in use)
    kWhenBelowTop = 3,       // cascade: level below the image's start level
    kWhenCycle = 4           // V-cycle step: not converged and level < levels in use
};

enum BatchKind {  // grid kernels of the batched form
    kBMaskDown = 0, kBValuesDown = 1, kBPack = 2, kBSelect = 3, kBRestrict = 4, kBProlong = 5,
    kBPyramid = 6  // one pyramid level in one pass (mask, values, packed words, unknown count)
};

struct BatchSeg {
    int first;             // first CTA (grid kernels) or block unit (block kernel)
    int gx, gy;            // grid kernels: CTAs along x and y per channel plane
    int w, h, C;           // level size (the fine level for restriction and prolongation)
    int img, level, when;  // image, level and participation (BatchWhen)
    int L;                 // the image's pyramid depth
    const void* in0;       // mask_down, values_down, pack: c; restrict: u; prolong: uH; block: u_in
    const void* in1;       // values_down: b; select: b; restrict: b; prolong: b; block: rhs
    const void* in2;       // values_down: cH; select: c; restrict: cH; prolong: c
    void* out0;            // mask_down: cH; values_down: bH; select: u; restrict: rH; prolong, block: u
    void* out1;            // select: a second u written alike (nullable)
    const uint32_t* mbits; // pack: bits out; block: the level's packed mask
    unsigned* maxupd;      // prolong, block: the image's update slot (nullable)
    unsigned long long* counter;  // pack: the image's unknown count of this level
    int zero_in, rhs_zero, iters, nbx, nby, wpr, mode, keep;
    float rtol2;
    // block kernel: the start prolonged from the next coarser level inside the
    // kernel (prolong_into_tile) -- pro_mode 0 none, 1 u_in + P pro_e at
    // unknown pixels (the correction; largest |P pro_e| into *pro_max), 2
    // u_in at known and P pro_e at unknown pixels (the cascade, u_in = b);
    // pro_check 1: only while level + 1 is in use for the image
    const float* pro_e;
    unsigned* pro_max;
    int pro_mode, pro_check;
    // block kernel: tma = 1 when the u_in and rhs tiles come by TMA through
    // the two tensor maps at tmaps (device memory, kTileMapsBytes, made by
    // make_tile_maps); 0: 4-byte cp.async
    const void* tmaps;
    int tma;
};

// Bytes of the two tensor maps (u_in tile, right-hand-side tile) of a block-
// kernel segment.
constexpr size_t kTileMapsBytes = 256;
// Writes the tensor maps of the 32x32 block kernel's u_in and rhs tiles over
// FP32 [C][h][w] images into out (kTileMapsBytes, 64-byte aligned host
// memory); a null image (zero_in / rhs_zero) gets no map.  False if an image
// does not meet TMA's rules (w a multiple of 4, 16-byte aligned base).
bool make_tile_maps(void* out, const float* u_in, int zero_in, const float* rhs, int rhs_zero,
                    int w, int h, int C);

// Per-image decode state of a batch (device arrays of n images).
struct BatchState {
    int* leff;   // levels in use
    int* top;    // start level of the cascade (-1: none)
    int* done;   // 1 once converged, failed or not to be solved
    StopState* st;
    unsigned* upd;  // [n][kMaxUpdSlots + 1]
    unsigned long long* counts;  // [n][kMaxLevels + 1]
    unsigned* err;               // set to 1 when a bounded wait of the block kernel ran out
    const float* tol;  // stop-rule target per image
};

// A batched grid kernel over nseg segments (segs in device memory, ordered by
// first) covering nctas CTAs.
cudaError_t launch_batch_grid(int kind, const BatchSeg* segs, int nseg, int nctas,
                              const BatchState& bs, cudaStream_t s);
// The batched block kernel (32x32 blocks, 0/1 weights) over nunits block units.
cudaError_t launch_batch_oras(const BatchSeg* segs, int nseg, int nunits, int o, float alpha,
                              const BatchState& bs, cudaStream_t s);
// Plan of every image (levels in use, cascade start, initial state); L[i]
// and n0[i] are the images' pyramid depths and pixel counts (device arrays).
cudaError_t launch_batch_plan(int n, const int* L, const unsigned long long* n0,
                              const BatchState& bs, cudaStream_t s);
// The stop test of every image still running; the loop handle is set to 0
// once none is.
cudaError_t launch_batch_stop(int n, const StopParams& p, const BatchState& bs,
                              unsigned long long h_loop, cudaStream_t s);
// CTAs per channel plane of the grid kernels for a level of w x h (2D kinds:
// 32 x 8 threads; pack and select: 256 threads).
void batch_grid_dims(int kind, int w, int h, int* gx, int* gy);

// Host-side geometry shared with the kernels.
inline int axis_blocks(int n, int B, int o) {
    const int s = B - o;
    int nb = (n - o + s - 1) / s;
    return nb < 1 ? 1 : nb;
}
// 32-bit words per row of a bit-packed mask, with one padding word.
inline int mask_words_per_row(int w) { return (w + 31) / 32 + 1; }
inline void coarse_dims(int w, int h, int* wH, int* hH) {
    *wH = (w + 1) / 2;
    *hH = (h + 1) / 2;
}
inline int num_levels(int w, int h, int B) {
    int n = 1;
    while ((w > h ? w : h) > B) {
        w = (w + 1) / 2;
        h = (h + 1) / 2;
        ++n;
    }
    return n;
}

}  // namespace di

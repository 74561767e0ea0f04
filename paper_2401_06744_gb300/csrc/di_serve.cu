// Batched decoding, the block-size / overlap autotuner and the serving loop,
// on top of di_inpaint.  Host code only: every decode still runs the library's
// kernels; this file schedules them.
//
// Concurrency model: a pool of worker slots, each with its own decoder
// context (so its pyramids and ORAS workspace stay resident between frames),
// its own non-blocking CUDA stream and its own host thread.  A decode blocks
// its thread once per V-cycle for the stop test, so several slots keep the GPU
// busy with overlapping frames: the kernels of different frames interleave on
// the device.  Every frame's arithmetic is independent of the others, so a
// frame decoded in a batch or under load is bit-identical to the same frame
// decoded alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/di.h"
#include "di_internal.h"

namespace {

struct Slot {
    di_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

di_status make_slot(const di_config* cfg, int device, Slot* s) {
    if (cudaSetDevice(device) != cudaSuccess) return DI_ERR_CUDA;
    di_status st = di_create(cfg, device, &s->ctx);
    if (st != DI_OK) return st;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) != cudaSuccess)
        return DI_ERR_CUDA;
    return DI_OK;
}

void free_slot(Slot* s) {
    if (s->done) cudaEventDestroy(s->done);
    if (s->stream) cudaStreamDestroy(s->stream);
    di_destroy(s->ctx);
    *s = Slot();
}

}  // namespace

// ---------------------------------------------------------------------------
// Batched decoding
// ---------------------------------------------------------------------------

struct di_pool {
    int device = 0;
    std::vector<Slot> slots;
    cudaEvent_t start = nullptr;
    std::mutex busy;  // one batch at a time per pool
};

extern "C" di_status di_pool_create(const di_config* cfg, int device, int concurrency,
                                    di_pool** out) {
    if (!out || concurrency < 0) return DI_ERR_INVALID_ARG;
    *out = nullptr;
    const int P = concurrency > 0 ? concurrency : 4;
    if (cudaSetDevice(device) != cudaSuccess) return DI_ERR_CUDA;
    di_pool* pool = new (std::nothrow) di_pool();
    if (!pool) return DI_ERR_OOM;
    pool->device = device;
    pool->slots.resize(P);
    di_status st = DI_OK;
    for (int k = 0; k < P && st == DI_OK; ++k) st = make_slot(cfg, device, &pool->slots[k]);
    if (st == DI_OK &&
        cudaEventCreateWithFlags(&pool->start, cudaEventDisableTiming) != cudaSuccess)
        st = DI_ERR_CUDA;
    if (st != DI_OK) {
        di_pool_destroy(pool);
        return st;
    }
    *out = pool;
    return DI_OK;
}

void di_pool_destroy(di_pool* pool) {
    if (!pool) return;
    cudaSetDevice(pool->device);
    for (auto& s : pool->slots) free_slot(&s);
    if (pool->start) cudaEventDestroy(pool->start);
    delete pool;
}

extern "C" di_status di_pool_inpaint(di_pool* pool, di_image* imgs, int n, void* stream) {
    if (!pool || !imgs || n < 0) return DI_ERR_INVALID_ARG;
    if (n == 0) return DI_OK;
    for (int i = 0; i < n; ++i) {
        const di_image& im = imgs[i];
        if (!im.f || !im.c || !im.u || im.width < 1 || im.height < 1 || im.channels < 1 ||
            im.channels > di::kMaxChannels || !(im.tol > 0.f))
            return DI_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(pool->busy);
    const int device = pool->device;
    if (cudaSetDevice(device) != cudaSuccess) return DI_ERR_CUDA;
    const int P = std::min<int>((int)pool->slots.size(), n);
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    // work starts after everything already queued on the caller's stream
    if (cudaEventRecord(pool->start, caller) != cudaSuccess) return DI_ERR_CUDA;
    // largest images first: better packing of the slots
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)imgs[a].width * imgs[a].height * imgs[a].channels >
               (long long)imgs[b].width * imgs[b].height * imgs[b].channels;
    });
    // images dealt round robin (largest first), so a repeated batch gives
    // every slot the same images and their graphs stay cached
    auto worker = [&](int k) {
        Slot& s = pool->slots[k];
        cudaSetDevice(device);
        cudaStreamWaitEvent(s.stream, pool->start, 0);
        for (int j = k; j < n; j += P) {
            di_image& im = imgs[order[j]];
            im.status = di_inpaint(s.ctx, im.f, im.c, im.width, im.height, im.channels, im.tol,
                                   im.u, s.stream);
            di_stats ss;
            di_get_stats(s.ctx, &ss);
            im.cycles = ss.cycles;
        }
        cudaEventRecord(s.done, s.stream);
    };
    std::vector<std::thread> th;
    for (int k = 1; k < P; ++k) th.emplace_back(worker, k);
    worker(0);
    for (auto& t : th) t.join();
    for (int k = 0; k < P; ++k) cudaStreamWaitEvent(caller, pool->slots[k].done, 0);
    cudaStreamSynchronize(caller);
    di_status worst = DI_OK;
    for (int i = 0; i < n; ++i)
        if (imgs[i].status != DI_OK && worst == DI_OK) worst = (di_status)imgs[i].status;
    return worst;
}

extern "C" di_status di_inpaint_batch(const di_config* cfg, int device, di_image* imgs, int n,
                                      int concurrency, void* stream) {
    if (!imgs || n < 0 || concurrency < 0) return DI_ERR_INVALID_ARG;
    if (n == 0) return DI_OK;
    // the batched form: one graph, one launch per step over every image
    di_batch* bt = nullptr;
    if (di_batch_create(cfg, device, imgs, n, &bt) == DI_OK) {
        cudaStream_t caller = static_cast<cudaStream_t>(stream);
        di_status st = di_batch_run(bt, imgs, n, caller);
        di_batch_destroy(bt);
        return st;
    }
    int P = concurrency > 0 ? concurrency : 4;
    if (P > n) P = n;
    di_pool* pool = nullptr;
    di_status st = di_pool_create(cfg, device, P, &pool);
    if (st != DI_OK) return st;
    st = di_pool_inpaint(pool, imgs, n, stream);
    di_pool_destroy(pool);
    return st;
}

// ---------------------------------------------------------------------------
// Autotuner over block size and overlap
// ---------------------------------------------------------------------------

namespace {

// Mean time of `reps` passes over the sample with configuration c (after one
// warm-up pass, which allocates the workspace and captures the graphs); a
// negative result if a decode fails or does not converge.
double time_config(const di_config& c, int device, const di_image* sample, int n, int reps,
                   cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    di_plan_info plan;
    if (di_plan(&c, 1, 1, 1, &plan) != DI_OK) return -1.0;  // not a valid configuration
    di_ctx* ctx = nullptr;
    if (di_create(&c, device, &ctx) != DI_OK) return -1.0;
    bool ok = true;
    for (int i = 0; i < n && ok; ++i)
        ok = di_inpaint(ctx, sample[i].f, sample[i].c, sample[i].width, sample[i].height,
                        sample[i].channels, sample[i].tol, sample[i].u, s) == DI_OK;
    double t = 0.0;
    for (int r = 0; r < reps && ok; ++r) {
        cudaEventRecord(e0, s);
        for (int i = 0; i < n && ok; ++i)
            ok = di_inpaint(ctx, sample[i].f, sample[i].c, sample[i].width, sample[i].height,
                            sample[i].channels, sample[i].tol, sample[i].u, s) == DI_OK;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t += ms;
    }
    di_destroy(ctx);
    return ok ? t / reps : -1.0;
}

}  // namespace

extern "C" di_status di_autotune_space(const di_config* base, int device, const di_image* sample,
                                       int n, const di_tune_space* space, int reps,
                                       di_config* best, double* best_ms) {
    if (!sample || n < 1 || !best || !space || reps < 1) return DI_ERR_INVALID_ARG;
    if ((space->nblocks > 0 && !space->blocks) || (space->noverlaps > 0 && !space->overlaps) ||
        (space->nlocal_iters > 0 && !space->local_iters) ||
        (space->nsmoothing > 0 && !space->smoothing) ||
        (space->nschedules > 0 && !space->schedules) || space->nblocks < 0 ||
        space->noverlaps < 0 || space->nlocal_iters < 0 || space->nsmoothing < 0 ||
        space->nschedules < 0)
        return DI_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DI_ERR_CUDA;
    di_config b;
    std::memset(&b, 0, sizeof b);
    if (base) b = *base;
    // an empty list keeps the base configuration's value
    auto count = [](int k) { return k > 0 ? k : 1; };
    double best_t = 1e300;
    bool found = false;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return DI_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int bi = 0; bi < count(space->nblocks); ++bi)
        for (int oi = 0; oi < count(space->noverlaps); ++oi)
            for (int ki = 0; ki < count(space->nlocal_iters); ++ki)
                for (int vi = 0; vi < count(space->nsmoothing); ++vi)
                    for (int si = 0; si < count(space->nschedules); ++si) {
                        di_config c = b;
                        if (space->nblocks) c.block = space->blocks[bi];
                        if (space->noverlaps) c.overlap = space->overlaps[oi];
                        if (space->nlocal_iters) c.local_iters = space->local_iters[ki];
                        if (space->nsmoothing) c.pre = c.post = space->smoothing[vi];
                        if (space->nschedules) c.schedule = space->schedules[si];
                        const double t = time_config(c, device, sample, n, reps, s, e0, e1);
                        if (t < 0.0) continue;  // invalid, failed or not converged
                        if (t < best_t) {
                            best_t = t;
                            *best = c;
                            found = true;
                        }
                    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (best_ms) *best_ms = found ? best_t : -1.0;
    return found ? DI_OK : DI_ERR_NOT_CONVERGED;
}

extern "C" di_status di_autotune(const di_config* base, int device, const di_image* sample, int n,
                                 const int* blocks, int nblocks, const int* overlaps,
                                 int noverlaps, int reps, di_config* best, double* best_ms) {
    if (!blocks || nblocks < 1 || !overlaps || noverlaps < 1) return DI_ERR_INVALID_ARG;
    di_tune_space sp;
    std::memset(&sp, 0, sizeof sp);
    sp.blocks = blocks;
    sp.nblocks = nblocks;
    sp.overlaps = overlaps;
    sp.noverlaps = noverlaps;
    return di_autotune_space(base, device, sample, n, &sp, reps, best, best_ms);
}

// ---------------------------------------------------------------------------
// Serving loop
//
// Every slot is a three-stage pipeline with its own host thread per stage:
// input (copy a request's f and c to the device on the slot's input stream),
// decode (di_inpaint on the slot's context and stream) and output (copy u
// back on the slot's output stream and complete the request).  Three device
// buffer sets rotate through the stages, so a slot copies the next request in
// and the previous result out while it decodes, and a copy from pageable host
// memory (which the runtime performs synchronously) blocks only its own stage.
// A slot's input stage takes a request from the queue only when the slot's
// decoder has nothing waiting, so a request does not queue behind a busy slot
// while another is idle.
// ---------------------------------------------------------------------------

namespace {

struct Request {
    long long ticket;
    const float* f;  // host
    const uint8_t* c;
    float* u;
    int w, h, ch;
    float tol;
    size_t bytes;  // device footprint while in flight
    // submitted, taken by a slot, copied in, taken by the decoder, decoded,
    // taken by the output stage, done
    std::chrono::steady_clock::time_point t_submit, t_start, t_in, t_dec0, t_dec1, t_out0, t_done;
    di_status status = DI_OK;
    int cycles = 0;
    int set = -1;  // buffer set of its slot
    bool done = false;
};

struct BufSet {
    float* f = nullptr;
    uint8_t* c = nullptr;
    float* u = nullptr;
    size_t cap = 0, cap_px = 0;  // pixel-channels and pixels of the buffers
};

// Hand-off between two stages of a slot.
template <class T>
struct Chan {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<T> q;
    bool closed = false;
    void push(T v) {
        {
            std::lock_guard<std::mutex> lock(mu);
            q.push_back(v);
        }
        cv.notify_all();
    }
    bool pop(T& v) {  // false once closed and drained
        std::unique_lock<std::mutex> lock(mu);
        cv.wait(lock, [&] { return closed || !q.empty(); });
        if (q.empty()) return false;
        v = q.front();
        q.pop_front();
        cv.notify_all();
        return true;
    }
    void wait_empty() {
        std::unique_lock<std::mutex> lock(mu);
        cv.wait(lock, [&] { return q.empty(); });
    }
    void close() {
        {
            std::lock_guard<std::mutex> lock(mu);
            closed = true;
        }
        cv.notify_all();
    }
};

constexpr int kSets = 3;

struct ServerSlot {
    Slot s;  // context and decode stream
    cudaStream_t in_stream = nullptr, out_stream = nullptr;
    // the copy stages wait on these (blocking, not spinning: a slot's three
    // threads and the decoders' own waits would otherwise spin on the cores)
    cudaEvent_t in_done = nullptr, out_done = nullptr;
    BufSet sets[kSets];
    Chan<int> free_sets;
    Chan<Request*> to_decode, to_output;
    std::thread t_in, t_dec, t_out;
};

}  // namespace

struct di_server {
    di_config cfg;
    int device = 0;
    size_t budget = 0;
    std::vector<ServerSlot*> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<long long, Request*> reqs;
    size_t in_flight_bytes = 0;
    long long next_ticket = 1;
    bool stop = false;
    long long completed = 0;
};

namespace {

size_t footprint(const di_config& cfg, int w, int h, int C) {
    di_plan_info p;
    if (di_plan(&cfg, w, h, C, &p) != DI_OK) return 0;
    // workspace + the request's own device copies of f, c and u
    return (size_t)p.workspace_bytes + (size_t)w * h * (2 * C * sizeof(float) + 1);
}

bool ensure_buffers(BufSet& b, size_t pxch, size_t px) {
    if (pxch <= b.cap && px <= b.cap_px) return true;
    if (b.f) cudaFree(b.f);
    if (b.u) cudaFree(b.u);
    if (b.c) cudaFree(b.c);
    b = BufSet();
    if (cudaMalloc(&b.f, pxch * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&b.u, pxch * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&b.c, px) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    b.cap = pxch;
    b.cap_px = px;
    return true;
}

void complete(di_server* srv, Request* r) {
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        r->t_done = std::chrono::steady_clock::now();
        r->done = true;
        srv->in_flight_bytes -= r->bytes;
        ++srv->completed;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
}

void input_stage(di_server* srv, ServerSlot* sl) {
    cudaSetDevice(srv->device);
    for (;;) {
        int set = -1;
        if (!sl->free_sets.pop(set)) break;
        sl->to_decode.wait_empty();  // the decoder is about to be free
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            // admission: the queue head runs once its footprint fits the budget
            // next to what is already in flight (a lone request always runs)
            srv->cv_work.wait(lock, [&] {
                if (srv->stop && srv->queue.empty()) return true;
                if (srv->queue.empty()) return false;
                Request* head = srv->queue.front();
                return srv->in_flight_bytes == 0 ||
                       srv->in_flight_bytes + head->bytes <= srv->budget;
            });
            if (srv->queue.empty()) break;  // stopping
            r = srv->queue.front();
            srv->queue.pop_front();
            srv->in_flight_bytes += r->bytes;
        }
        r->t_start = std::chrono::steady_clock::now();
        r->set = set;
        BufSet& b = sl->sets[set];
        const size_t px = (size_t)r->w * r->h, pxch = px * r->ch;
        if (!ensure_buffers(b, pxch, px)) {
            r->status = DI_ERR_OOM;
        } else if (cudaMemcpyAsync(b.f, r->f, pxch * sizeof(float), cudaMemcpyHostToDevice,
                                   sl->in_stream) != cudaSuccess ||
                   cudaMemcpyAsync(b.c, r->c, px, cudaMemcpyHostToDevice, sl->in_stream) !=
                       cudaSuccess ||
                   cudaEventRecord(sl->in_done, sl->in_stream) != cudaSuccess ||
                   cudaEventSynchronize(sl->in_done) != cudaSuccess) {
            cudaGetLastError();
            r->status = DI_ERR_CUDA;
        }
        r->t_in = std::chrono::steady_clock::now();
        sl->to_decode.push(r);
    }
    sl->to_decode.close();
}

void decode_stage(di_server* srv, ServerSlot* sl) {
    cudaSetDevice(srv->device);
    Request* r = nullptr;
    while (sl->to_decode.pop(r)) {
        r->t_dec0 = std::chrono::steady_clock::now();
        if (r->status == DI_OK) {
            BufSet& b = sl->sets[r->set];
            di_status st = di_inpaint(sl->s.ctx, b.f, b.c, r->w, r->h, r->ch, r->tol, b.u,
                                      sl->s.stream);
            // whatever the status, nothing of this request stays queued
            if (cudaStreamSynchronize(sl->s.stream) != cudaSuccess && st == DI_OK)
                st = DI_ERR_CUDA;
            di_stats ss;
            di_get_stats(sl->s.ctx, &ss);
            r->status = st;
            r->cycles = ss.cycles;
        }
        r->t_dec1 = std::chrono::steady_clock::now();
        sl->to_output.push(r);
    }
    sl->to_output.close();
}

void output_stage(di_server* srv, ServerSlot* sl) {
    cudaSetDevice(srv->device);
    Request* r = nullptr;
    while (sl->to_output.pop(r)) {
        r->t_out0 = std::chrono::steady_clock::now();
        if (r->status == DI_OK || r->status == DI_ERR_NOT_CONVERGED) {
            BufSet& b = sl->sets[r->set];
            const size_t pxch = (size_t)r->w * r->h * r->ch;
            if (cudaMemcpyAsync(r->u, b.u, pxch * sizeof(float), cudaMemcpyDeviceToHost,
                                sl->out_stream) != cudaSuccess ||
                cudaEventRecord(sl->out_done, sl->out_stream) != cudaSuccess ||
                cudaEventSynchronize(sl->out_done) != cudaSuccess) {
                cudaGetLastError();
                r->status = DI_ERR_CUDA;
            }
        }
        if (r->set >= 0) sl->free_sets.push(r->set);
        complete(srv, r);
    }
}

void free_server_slot(ServerSlot* sl) {
    for (auto& b : sl->sets) {
        if (b.f) cudaFree(b.f);
        if (b.u) cudaFree(b.u);
        if (b.c) cudaFree(b.c);
    }
    if (sl->in_done) cudaEventDestroy(sl->in_done);
    if (sl->out_done) cudaEventDestroy(sl->out_done);
    if (sl->in_stream) cudaStreamDestroy(sl->in_stream);
    if (sl->out_stream) cudaStreamDestroy(sl->out_stream);
    free_slot(&sl->s);
    delete sl;
}

}  // namespace

extern "C" di_status di_server_create(const di_config* cfg, int device, int slots,
                                      long long mem_budget, di_server** out) {
    if (!out || slots < 1 || slots > 64 || mem_budget < 0) return DI_ERR_INVALID_ARG;
    *out = nullptr;
    di_server* srv = new (std::nothrow) di_server();
    if (!srv) return DI_ERR_OOM;
    std::memset(&srv->cfg, 0, sizeof srv->cfg);
    if (cfg) srv->cfg = *cfg;
    srv->device = device;
    srv->budget = mem_budget > 0 ? (size_t)mem_budget : (size_t)-1;
    di_status st = DI_OK;
    for (int k = 0; k < slots && st == DI_OK; ++k) {
        ServerSlot* sl = new (std::nothrow) ServerSlot();
        if (!sl) { st = DI_ERR_OOM; break; }
        srv->slots.push_back(sl);
        st = make_slot(&srv->cfg, device, &sl->s);
        const unsigned evf = cudaEventDisableTiming | cudaEventBlockingSync;
        if (st == DI_OK &&
            (cudaStreamCreateWithFlags(&sl->in_stream, cudaStreamNonBlocking) != cudaSuccess ||
             cudaStreamCreateWithFlags(&sl->out_stream, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&sl->in_done, evf) != cudaSuccess ||
             cudaEventCreateWithFlags(&sl->out_done, evf) != cudaSuccess))
            st = DI_ERR_CUDA;
        for (int b = 0; b < kSets; ++b) sl->free_sets.push(b);
    }
    if (st != DI_OK) {
        for (auto* sl : srv->slots) free_server_slot(sl);
        delete srv;
        return st;
    }
    for (auto* sl : srv->slots) {
        sl->t_in = std::thread(input_stage, srv, sl);
        sl->t_dec = std::thread(decode_stage, srv, sl);
        sl->t_out = std::thread(output_stage, srv, sl);
    }
    *out = srv;
    return DI_OK;
}

extern "C" di_status di_server_submit(di_server* srv, const float* f, const uint8_t* c, int width,
                                      int height, int channels, float tol, float* u,
                                      long long* ticket) {
    if (!srv || !f || !c || !u || !ticket || width < 1 || height < 1 || channels < 1 ||
        channels > di::kMaxChannels || !(tol > 0.f))
        return DI_ERR_INVALID_ARG;
    Request* r = new (std::nothrow) Request();
    if (!r) return DI_ERR_OOM;
    r->f = f;
    r->c = c;
    r->u = u;
    r->w = width;
    r->h = height;
    r->ch = channels;
    r->tol = tol;
    r->bytes = footprint(srv->cfg, width, height, channels);
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        r->ticket = srv->next_ticket++;
        srv->reqs[r->ticket] = r;
        srv->queue.push_back(r);
    }
    *ticket = r->ticket;
    srv->cv_work.notify_all();
    return DI_OK;
}

extern "C" di_status di_server_wait(di_server* srv, long long ticket, di_request_info* info) {
    if (!srv) return DI_ERR_INVALID_ARG;
    Request* r = nullptr;
    {
        std::unique_lock<std::mutex> lock(srv->mu);
        auto it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) return DI_ERR_INVALID_ARG;
        r = it->second;
        srv->cv_done.wait(lock, [&] { return r->done; });
        srv->reqs.erase(it);
    }
    if (info) {
        using ms = std::chrono::duration<double, std::milli>;
        info->status = r->status;
        info->cycles = r->cycles;
        info->latency_ms = ms(r->t_done - r->t_submit).count();
        info->queue_ms = ms(r->t_start - r->t_submit).count();
        info->footprint_bytes = (long long)r->bytes;
        info->copy_in_ms = ms(r->t_in - r->t_start).count();
        info->wait_decode_ms = ms(r->t_dec0 - r->t_in).count();
        info->decode_ms = ms(r->t_dec1 - r->t_dec0).count();
        info->wait_out_ms = ms(r->t_out0 - r->t_dec1).count();
        info->copy_out_ms = ms(r->t_done - r->t_out0).count();
    }
    di_status st = r->status;
    delete r;
    return st;
}

extern "C" void di_server_destroy(di_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    // the input stages finish the queue and close their pipelines
    for (auto* sl : srv->slots) sl->free_sets.close();
    for (auto* sl : srv->slots) {
        if (sl->t_in.joinable()) sl->t_in.join();
        if (sl->t_dec.joinable()) sl->t_dec.join();
        if (sl->t_out.joinable()) sl->t_out.join();
    }
    cudaSetDevice(srv->device);
    for (auto* sl : srv->slots) free_server_slot(sl);
    for (auto& kv : srv->reqs) delete kv.second;
    delete srv;
}

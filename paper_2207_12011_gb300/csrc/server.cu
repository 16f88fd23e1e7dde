// Serving runtime: continuous batching of brushed render and histogram
// requests over resident volumes.
//
// Clients submit requests from any thread. One server thread loops:
//   1. completions: query the completion event of every in-flight launch and
//      publish finished passes (coarse image, full image, histogram);
//   2. admission: move queued requests (FIFO) into service while fewer than
//      max_inflight are in service and their outputs fit in the output pool
//      (the HBM budget for results);
//   3. launch: for every stream with fewer than two launches in flight, take
//      the oldest unlaunched requests (up to the view and pixel caps): their
//      histogram kernels first, then one batched render launch (one CUDA graph
//      replay) holding all their coarse passes and then all their full passes,
//      each group smallest image first. The persistent kernel writes a
//      completion record per view into mapped host memory, so each pass is
//      published as soon as its own tiles are done.
// Requests that arrive while launches are running are admitted as slots and
// pool memory free up and join the next launch, so their work overlaps with
// the work already on the GPU. Every pass uses the same kernels as a single
// render / histogram call, so each result is identical alone and in the mix.
// The server never waits on the GPU without a bound: it only queries events
// and sleeps at most 100 us between turns while launches are in flight.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace raypc;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over one preallocated device region (host bookkeeping
// only, so admission never calls the CUDA allocator).
struct Pool {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    size_t used = 0;
    void init(char* b, size_t s) {
        base = b;
        size = s;
        free_.clear();
        free_[0] = s;
        used = 0;
    }
    char* alloc(size_t n) {
        n = align_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                used += n;
                return base + off;
            }
        }
        return nullptr;
    }
    void release(char* p, size_t n) {
        n = align_up(n);
        size_t off = (size_t)(p - base);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum Pass { kCoarse = 0, kFull = 1, kHist = 2 };

struct Req {
    uint64_t id = 0;
    raypc_request r{};
    std::vector<float> edges;
    int status = RAYPC_OK;
    bool admitted = false, coarse_launched = false, full_launched = false;
    bool coarse_ready = false, done = false;
    double t_submit = 0, t_admit = 0, t_coarse = 0, t_done = 0;
    char* mem = nullptr;
    size_t mem_bytes = 0;
    float* coarse = nullptr;
    float* image = nullptr;
    unsigned long long* stats = nullptr;
    uint32_t* hist = nullptr;
    float* d_edges = nullptr;
    unsigned long long samples = 0;
};

struct Item {
    Req* q;
    int pass;                     // kCoarse, kFull or kHist
    int view;                     // index in the launch's batch (render passes)
    bool seen = false;
};

struct Launch {
    cudaEvent_t ev_hist = nullptr;   // after the launch's histogram kernels
    cudaEvent_t ev = nullptr;        // after the batched render
    int stream = 0;
    const ViewDone* recs = nullptr;  // completion records of the batched render
    unsigned seq = 0;
    std::vector<Item> items;
};

size_t output_bytes(const raypc_request& r) {
    if (r.kind == RAYPC_REQ_HISTOGRAM)
        return align_up(sizeof(uint32_t) * ((size_t)(r.naxes - 1) * r.bins * r.bins + 1)) +
               align_up(sizeof(float) * (size_t)r.naxes * (r.bins + 1));
    size_t img = align_up(sizeof(float) * 4 * (size_t)r.w * r.h);
    return img * (r.coarse_lod >= 0 ? 2 : 1) + align_up(sizeof(unsigned long long) * kNStats);
}

}  // namespace

struct raypc_server {
    raypc_ctx* ctx = nullptr;
    raypc_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queued;
    std::vector<Req*> active;           // admitted, not done
    std::map<uint64_t, Req*> all;
    std::vector<Launch> inflight;
    std::vector<int> busy;              // launches in flight per stream
    std::vector<cudaStream_t> streams;
    std::vector<raypc_batch*> batches;
    std::vector<void*> hscratch;        // per stream: histogram scratch (partial copies, sub-brick bits)
    std::vector<size_t> hscratch_bytes;
    Pool pool;
    char* pool_mem = nullptr;
    uint64_t next_id = 1;
    int rr = 0;
    bool stop = false;
    std::thread th;
};

namespace {

void finish(raypc_server* S, Req* q, int status) {
    if (q->done) return;
    if (status != RAYPC_OK && q->status == RAYPC_OK) q->status = status;
    q->done = true;
    q->t_done = now_s();
    for (size_t i = 0; i < S->active.size(); ++i)
        if (S->active[i] == q) {
            S->active.erase(S->active.begin() + i);
            break;
        }
}

// Histogram of one request on stream si (the request's brush, its own edges). Like
// raypc_pc_histogram, a brushed request first classifies the level's sub-bricks
// under its own brush, so the kernel skips the cells of inactive ones, and large
// grids spread the counts over zeroed partial histograms that a reduction sums
// into the output; both live in the stream's scratch, which the requests of one
// stream use one after the other in stream order.
raypc_status launch_hist(raypc_server* S, Req* q, int si) {
    cudaStream_t s = S->streams[si];
    std::lock_guard<std::mutex> lk(S->ctx->mu);
    DeviceGuard g(S->ctx->device);
    Volume* V = nullptr;
    Level* L = nullptr;
    raypc_status st;
    if ((st = get_volume(S->ctx, q->r.vol, &V)) || (st = get_level(V, q->r.lod, &L))) return st;
    if (V->stale && q->r.lod > 0) return fail(RAYPC_ERR_INVALID_ARG, "level is stale");
    BrushArgs b{};
    if ((st = brush_from_host(V, q->r.lo, q->r.hi, q->r.active_mask, &b))) return st;
    if ((st = pos_from_host(q->r.pos_lo, q->r.pos_hi, q->r.pos_mask, &b))) return st;
    const int naxes = q->r.naxes, bins = q->r.bins;
    HistArgs h{};
    h.cells = L->cells;
    h.n = L->n;
    h.nvars = V->nvars;
    h.brush = b;
    h.use_brush = q->r.use_brush ? 1 : 0;
    h.naxes = naxes;
    h.bins = bins;
    for (int a = 0; a < kMaxVars; ++a) h.axis[a] = a < naxes ? q->r.axis_order[a] : 0;
    h.need_mask = h.use_brush ? b.mask : 0u;
    for (int a = 0; a < naxes; ++a) {
        if (q->r.axis_order[a] < kPosAxisBase) h.need_mask |= 1u << q->r.axis_order[a];
        const float e0 = q->edges[(size_t)a * (bins + 1)], eN = q->edges[(size_t)a * (bins + 1) + bins];
        h.guess_e0[a] = e0;
        h.guess_scale[a] = (eN > e0 && isfinite(eN - e0)) ? (float)bins / (eN - e0) : 0.0f;
    }
    double ri = (double)V->r_in * (double)L->n, ro = (double)V->r_out * (double)L->n;
    h.s_in = (int64_t)ceil(ri * ri);
    h.s_out = (int64_t)floor(ro * ro);
    h.edges = q->d_edges;
    h.edges_host = q->edges.data();       // small tables travel in the launch parameters
    h.out = q->hist;
    cudaError_t e = cudaSuccess;
    if (q->edges.size() > (size_t)kHistInlineEdges)
        e = cudaMemcpyAsync(q->d_edges, q->edges.data(), sizeof(float) * q->edges.size(), cudaMemcpyHostToDevice, s);
    // scratch: the partial copies and their row counter (large grids), then the sub-brick bits
    const size_t count = (size_t)(naxes - 1) * bins * bins;
    const int ncopies = ((uintptr_t)q->hist & 15u) ? 1 : hist_copies(L->n, naxes, bins);
    const size_t copy_bytes = ncopies > 1 ? (sizeof(uint32_t) * (count * ncopies + 4) + 255) / 256 * 256 : 0;
    const bool activity = h.use_brush && L->sbmin;
    const size_t need = copy_bytes + (activity ? sizeof(uint32_t) * L->nswords() : 0);
    if (need > S->hscratch_bytes[si]) {
        // the stream's earlier histograms may still read the old scratch
        if (S->hscratch[si]) {
            cudaStreamSynchronize(s);
            cudaFree(S->hscratch[si]);
            S->ctx->used -= S->hscratch_bytes[si] < S->ctx->used ? S->hscratch_bytes[si] : S->ctx->used;
            S->hscratch[si] = nullptr;
            S->hscratch_bytes[si] = 0;
        }
        size_t charged = 0;
        if ((st = S->ctx->alloc(&S->hscratch[si], need, &charged))) return st;
        S->hscratch_bytes[si] = need;
    }
    char* scratch = static_cast<char*>(S->hscratch[si]);
    if (activity && e == cudaSuccess) {
        ClassifyArgs c{};
        c.nvars = V->nvars;
        c.rin2 = V->r_in * V->r_in;
        c.rout2 = V->r_out * V->r_out;
        c.brush = b;
        c.nlev = 1;
        c.nbrick = 0;
        c.lv[0].bmin = L->sbmin;
        c.lv[0].bmax = L->sbmax;
        c.lv[0].n = L->n;
        c.lv[0].bs = kSub;
        c.lv[0].active = reinterpret_cast<uint32_t*>(scratch + copy_bytes);
        e = launch_classify(c, s);
        h.sactive = c.lv[0].active;
        h.nsb = L->nsb;
    }
    if (ncopies > 1) {
        // the counts spread over zeroed partial copies, summed into the output afterwards
        uint32_t* copies = reinterpret_cast<uint32_t*>(scratch);
        h.copies = copies;
        h.ncopies = ncopies;
        h.rowctr = copies + count * ncopies;
        if (e == cudaSuccess) e = cudaMemsetAsync(copies, 0, sizeof(uint32_t) * (count * ncopies + 4), s);
        if (e == cudaSuccess) e = launch_histogram(h, V->dtype, s);
        if (e == cudaSuccess) e = launch_histogram_reduce(copies, ncopies, count, q->hist, s);
    } else {
        // the counts and, after them, the row counter that balances the warps
        h.rowctr = q->hist + count;
        if (e == cudaSuccess) e = cudaMemsetAsync(q->hist, 0, sizeof(uint32_t) * (count + 1), s);
        if (e == cudaSuccess) e = launch_histogram(h, V->dtype, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "server histogram");
    return RAYPC_OK;
}

void publish(raypc_server* S, Item& it, double t, unsigned long long marched) {
    Req* q = it.q;
    it.seen = true;
    if (it.pass == kCoarse) {
        q->coarse_ready = true;
        q->t_coarse = t;
        return;
    }
    if (it.pass == kFull) q->samples = marched;
    finish(S, q, RAYPC_OK);
    q->t_done = t;
}

void turn(raypc_server* S) {
    // 1. completions: per-view records of the batched renders, histogram events
    bool any = false;
    for (size_t i = 0; i < S->inflight.size();) {
        Launch& L = S->inflight[i];
        const double t = now_s();
        const cudaError_t eh = L.ev_hist ? cudaEventQuery(L.ev_hist) : cudaSuccess;
        const cudaError_t e = cudaEventQuery(L.ev);
        const bool failed = (eh != cudaSuccess && eh != cudaErrorNotReady) || (e != cudaSuccess && e != cudaErrorNotReady);
        for (Item& it : L.items) {
            if (it.seen || it.q->done) continue;
            if (failed) {
                it.seen = true;
                finish(S, it.q, RAYPC_ERR_CUDA);
                any = true;
                continue;
            }
            if (it.pass == kHist) {
                if (eh == cudaSuccess) { publish(S, it, t, 0); any = true; }
                continue;
            }
            const ViewDone& r = L.recs[it.view];
            if (r.seq == L.seq) {
                std::atomic_thread_fence(std::memory_order_acquire);
                publish(S, it, t, r.stats[RAYPC_STAT_MARCHED]);
                any = true;
            }
        }
        if (e == cudaErrorNotReady || (L.ev_hist && eh == cudaErrorNotReady)) {
            ++i;
            continue;
        }
        if (failed) cudaGetLastError();
        for (Item& it : L.items)                 // launch over: every record is final
            if (!it.seen && !it.q->done) {
                const unsigned long long m = it.pass == kHist ? 0ull : L.recs[it.view].stats[RAYPC_STAT_MARCHED];
                publish(S, it, t, m);
                any = true;
            }
        if (L.ev_hist) cudaEventDestroy(L.ev_hist);
        cudaEventDestroy(L.ev);
        S->busy[L.stream]--;
        S->inflight.erase(S->inflight.begin() + i);
    }
    if (any) S->cv_done.notify_all();
    // 2. admission (FIFO)
    while (!S->queued.empty() && (int)S->active.size() < S->cfg.max_inflight) {
        Req* q = S->queued.front();
        char* m = S->pool.alloc(q->mem_bytes);
        if (!m) break;                                  // wait for outputs to be released
        S->queued.pop_front();
        q->mem = m;
        q->admitted = true;
        q->t_admit = now_s();
        char* p = m;
        if (q->r.kind == RAYPC_REQ_HISTOGRAM) {
            q->hist = reinterpret_cast<uint32_t*>(p);
            p += align_up(sizeof(uint32_t) * ((size_t)(q->r.naxes - 1) * q->r.bins * q->r.bins + 1));
            q->d_edges = reinterpret_cast<float*>(p);
        } else {
            const size_t img = align_up(sizeof(float) * 4 * (size_t)q->r.w * q->r.h);
            q->image = reinterpret_cast<float*>(p);
            p += img;
            if (q->r.coarse_lod >= 0) {
                q->coarse = reinterpret_cast<float*>(p);
                p += img;
            }
            q->stats = reinterpret_cast<unsigned long long*>(p);
        }
        S->active.push_back(q);
    }
    // 3. launches: every stream with room takes the oldest unlaunched requests
    for (int k = 0; k < (int)S->streams.size(); ++k) {
        const int s = (S->rr + k) % (int)S->streams.size();
        if (S->busy[s] >= 2) continue;
        std::vector<Req*> renders, hists;
        long long pixels = 0;
        int nviews = 0;
        for (Req* q : S->active) {
            if (q->done || q->full_launched) continue;
            if (q->r.kind == RAYPC_REQ_HISTOGRAM) {
                hists.push_back(q);
                continue;
            }
            const int nv = q->r.coarse_lod >= 0 ? 2 : 1;
            const long long px = (long long)q->r.w * q->r.h * nv;
            if (nviews + nv > S->cfg.max_batch_views) continue;
            if (!renders.empty() && S->cfg.max_batch_pixels > 0 && pixels + px > S->cfg.max_batch_pixels) continue;
            renders.push_back(q);
            pixels += px;
            nviews += nv;
        }
        if (renders.empty() && hists.empty()) break;    // nothing pending for any stream
        S->rr = (s + 1) % (int)S->streams.size();
        Launch L;
        L.stream = s;
        cudaStream_t st = S->streams[s];
        // histograms first (short), with their own completion event
        for (Req* q : hists) {
            q->full_launched = true;
            raypc_status hs = launch_hist(S, q, s);
            if (hs != RAYPC_OK) { finish(S, q, hs); continue; }
            L.items.push_back({q, kHist, -1});
        }
        if (!L.items.empty() &&
            (cudaEventCreateWithFlags(&L.ev_hist, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventRecord(L.ev_hist, st) != cudaSuccess)) {
            cudaStreamSynchronize(st);
            for (Item& it : L.items) finish(S, it.q, RAYPC_ERR_CUDA);
            L.items.clear();
            if (L.ev_hist) cudaEventDestroy(L.ev_hist);
            L.ev_hist = nullptr;
        }
        // render passes: all coarse passes, then all full passes, each smallest first
        std::vector<std::pair<Req*, int>> passes;
        for (int pass = kCoarse; pass <= kFull; ++pass) {
            std::vector<Req*> v;
            for (Req* q : renders)
                if (pass == kFull || q->r.coarse_lod >= 0) v.push_back(q);
            std::stable_sort(v.begin(), v.end(), [](Req* a, Req* b) {
                return (long long)a->r.w * a->r.h < (long long)b->r.w * b->r.h;
            });
            for (Req* q : v) passes.push_back({q, pass});
        }
        if (!passes.empty()) {
            std::vector<raypc_view> views;
            for (auto& pr : passes) {
                Req* q = pr.first;
                raypc_view v{};
                v.vol = q->r.vol;
                v.lod = pr.second == kCoarse ? q->r.coarse_lod : q->r.lod;
                v.cam = q->r.cam;
                v.w = q->r.w;
                v.h = q->r.h;
                memcpy(v.lo, q->r.lo, sizeof(v.lo));
                memcpy(v.hi, q->r.hi, sizeof(v.hi));
                v.active_mask = q->r.active_mask;
                memcpy(v.pos_lo, q->r.pos_lo, sizeof(v.pos_lo));
                memcpy(v.pos_hi, q->r.pos_hi, sizeof(v.pos_hi));
                v.pos_mask = q->r.pos_mask;
                v.opts = q->r.opts;
                v.opts.counts_dev = nullptr;
                v.out_rgba_dev = pr.second == kCoarse ? q->coarse : q->image;
                v.stats_dev = pr.second == kCoarse ? nullptr : q->stats;
                views.push_back(v);
            }
            for (Req* q : renders) cudaMemsetAsync(q->stats, 0, sizeof(unsigned long long) * kNStats, st);
            raypc_status rs = raypc_render_batch(S->batches[s], views.data(), (int)views.size(), st);
            if (rs != RAYPC_OK) {
                for (Req* q : renders) finish(S, q, rs);
            } else {
                batch_last_records(S->batches[s], &L.recs, &L.seq);
                for (size_t i = 0; i < passes.size(); ++i) {
                    Req* q = passes[i].first;
                    if (passes[i].second == kCoarse) q->coarse_launched = true;
                    else q->full_launched = true;
                    L.items.push_back({q, passes[i].second, (int)i});
                }
            }
        }
        if (L.items.empty()) {
            if (L.ev_hist) cudaEventDestroy(L.ev_hist);
            continue;
        }
        if (cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(L.ev, st) != cudaSuccess) {
            cudaStreamSynchronize(st);
            for (Item& it : L.items) finish(S, it.q, RAYPC_ERR_CUDA);
            if (L.ev) cudaEventDestroy(L.ev);
            if (L.ev_hist) cudaEventDestroy(L.ev_hist);
            continue;
        }
        S->busy[s]++;
        S->inflight.push_back(L);
    }
}

void loop(raypc_server* S) {
    DeviceGuard g(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        turn(S);
        if (S->inflight.empty() && (S->queued.empty() || (int)S->active.size() >= S->cfg.max_inflight))
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        else
            S->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
    // drain: wait for launches, end everything else
    for (auto& L : S->inflight) {
        cudaEventSynchronize(L.ev);
        cudaEventDestroy(L.ev);
        if (L.ev_hist) cudaEventDestroy(L.ev_hist);
    }
    S->inflight.clear();
    for (auto& kv : S->all)
        if (!kv.second->done) finish(S, kv.second, RAYPC_ERR_BUSY);
    S->cv_done.notify_all();
}

}  // namespace

extern "C" {

raypc_status raypc_server_create(raypc_ctx* ctx, const raypc_server_config* cfg, raypc_server** out) {
    if (!ctx || !cfg || !out) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 4096) return fail(RAYPC_ERR_INVALID_ARG, "max_inflight not in 1..4096");
    if (cfg->max_batch_views < 1 || cfg->max_batch_views > 4096) return fail(RAYPC_ERR_INVALID_ARG, "max_batch_views not in 1..4096");
    if (cfg->num_streams < 1 || cfg->num_streams > 8) return fail(RAYPC_ERR_INVALID_ARG, "num_streams not in 1..8");
    *out = nullptr;
    raypc_server* S = new raypc_server();
    S->ctx = ctx;
    S->cfg = *cfg;
    if (S->cfg.output_budget_bytes == 0) S->cfg.output_budget_bytes = (size_t)1 << 30;
    raypc_status st = RAYPC_OK;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard g(ctx->device);
        size_t charged = 0;
        st = ctx->alloc((void**)&S->pool_mem, S->cfg.output_budget_bytes, &charged);
        if (st == RAYPC_OK) S->pool.init(S->pool_mem, S->cfg.output_budget_bytes);

        for (int i = 0; i < cfg->num_streams && st == RAYPC_OK; ++i) {
            cudaStream_t s = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) { st = cuda_fail(e, "server stream"); break; }
            S->streams.push_back(s);
            S->busy.push_back(0);
            S->hscratch.push_back(nullptr);
            S->hscratch_bytes.push_back(0);
        }
    }
    for (int i = 0; i < cfg->num_streams && st == RAYPC_OK; ++i) {
        raypc_batch* b = nullptr;
        st = raypc_batch_create(ctx, cfg->max_batch_views, &b);
        if (st == RAYPC_OK) S->batches.push_back(b);
    }
    if (st != RAYPC_OK) {
        raypc_server_destroy(S);
        return st;
    }
    S->th = std::thread(loop, S);
    *out = S;
    return RAYPC_OK;
}

raypc_status raypc_server_destroy(raypc_server* S) {
    if (!S) return RAYPC_OK;
    if (S->th.joinable()) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv_work.notify_all();
        S->th.join();
    }
    for (raypc_batch* b : S->batches) raypc_batch_destroy(b);
    {
        std::lock_guard<std::mutex> lk(S->ctx->mu);
        DeviceGuard g(S->ctx->device);
        for (cudaStream_t s : S->streams) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        for (size_t i = 0; i < S->hscratch.size(); ++i)
            if (S->hscratch[i]) {
                cudaFree(S->hscratch[i]);
                S->ctx->used -= S->hscratch_bytes[i] < S->ctx->used ? S->hscratch_bytes[i] : S->ctx->used;
            }
        if (S->pool_mem) {
            cudaFree(S->pool_mem);
            S->ctx->used -= S->cfg.output_budget_bytes < S->ctx->used ? S->cfg.output_budget_bytes : S->ctx->used;
        }
    }
    for (auto& kv : S->all) delete kv.second;
    delete S;
    return RAYPC_OK;
}

raypc_status raypc_serve_submit(raypc_server* S, const raypc_request* r, uint64_t* out_id) {
    if (!S || !r || !out_id) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    Req* q = new Req();
    q->r = *r;
    q->t_submit = now_s();
    {
        // validate against the volume now (context lock only)
        std::lock_guard<std::mutex> lk(S->ctx->mu);
        DeviceGuard g(S->ctx->device);
        Volume* V = nullptr;
        Level* L = nullptr;
        raypc_status st;
        if ((st = get_volume(S->ctx, r->vol, &V)) || (st = get_level(V, r->lod, &L))) { delete q; return st; }
        BrushArgs b{};
        if ((st = brush_from_host(V, r->lo, r->hi, r->active_mask, &b))) { delete q; return st; }
        if ((st = pos_from_host(r->pos_lo, r->pos_hi, r->pos_mask, &b))) { delete q; return st; }
        if (r->kind == RAYPC_REQ_RENDER) {
            RenderArgs a{};
            if (r->opts.depth_dev) {          // outputs of a request are server-owned
                delete q;
                return fail(RAYPC_ERR_UNSUPPORTED, "depth_dev is not available for served requests");
            }
            if (r->w < 1 || r->h < 1 || r->w > 32768 || r->h > 32768) { delete q; return fail(RAYPC_ERR_INVALID_ARG, "image size out of range"); }
            // validate camera / options with a stand-in aligned output pointer
            if ((st = make_render_args(V, L, &r->cam, r->w, r->h, &r->opts, reinterpret_cast<float*>(256), nullptr, &a))) { delete q; return st; }
            if (r->coarse_lod >= 0) {
                Level* C = nullptr;
                if ((st = get_level(V, r->coarse_lod, &C))) { delete q; return st; }
                if (!C->bricks) { delete q; return fail(RAYPC_ERR_INVALID_ARG, "coarse level has no bricks"); }
            }
        } else if (r->kind == RAYPC_REQ_HISTOGRAM) {
            if (r->naxes < 2 || r->naxes > RAYPC_MAX_VARS || r->bins < 2 || r->bins > 1024 || !r->edges) {
                delete q;
                return fail(RAYPC_ERR_INVALID_ARG, "bad histogram request (naxes 2..8, bins 2..1024, edges)");
            }
            for (int a = 0; a < r->naxes; ++a) {
                if (!((r->axis_order[a] >= 0 && r->axis_order[a] < V->nvars) ||
                      (r->axis_order[a] >= kPosAxisBase && r->axis_order[a] < kPosAxisBase + kNumPos))) {
                    delete q;
                    return fail(RAYPC_ERR_INVALID_ARG, "bad axis");
                }
                for (int k = 0; k <= r->bins; ++k) {
                    float e = r->edges[(size_t)a * (r->bins + 1) + k];
                    if (isnan(e) || (k && e < r->edges[(size_t)a * (r->bins + 1) + k - 1])) {
                        delete q;
                        return fail(RAYPC_ERR_INVALID_ARG, "edges must be non-decreasing and not NaN");
                    }
                }
            }
            q->edges.assign(r->edges, r->edges + (size_t)r->naxes * (r->bins + 1));
        } else {
            delete q;
            return fail(RAYPC_ERR_INVALID_ARG, "unknown request kind %d", r->kind);
        }
    }
    q->r.edges = nullptr;
    q->mem_bytes = output_bytes(q->r);
    if (q->mem_bytes > S->cfg.output_budget_bytes) {
        const size_t bytes = q->mem_bytes;
        delete q;
        return fail(RAYPC_ERR_OOM, "request outputs (%zu bytes) exceed the server's output budget", bytes);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) { delete q; return fail(RAYPC_ERR_BUSY, "server is stopping"); }
        q->id = S->next_id++;
        S->all[q->id] = q;
        S->queued.push_back(q);
        *out_id = q->id;
    }
    S->cv_work.notify_all();
    return RAYPC_OK;
}

raypc_status raypc_serve_poll(raypc_server* S, uint64_t id, int timeout_us, raypc_result* out) {
    if (!S || !out) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(RAYPC_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)id);
    Req* q = it->second;
    if (!q->done && timeout_us > 0) {
        const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
        S->cv_done.wait_until(lk, until, [&] { return q->done; });
    }
    memset(out, 0, sizeof(*out));
    out->status = q->status;
    out->coarse_ready = q->coarse_ready ? 1 : 0;
    out->done = q->done ? 1 : 0;
    out->t_submit = q->t_submit;
    out->t_admit = q->t_admit;
    out->t_coarse = q->t_coarse;
    out->t_done = q->t_done;
    out->coarse_dev = q->coarse;
    out->image_dev = q->image;
    out->hist_dev = q->hist;
    out->samples = q->samples;
    if (!q->done) return fail(RAYPC_ERR_TIMEOUT, "request %llu not done", (unsigned long long)id);
    return RAYPC_OK;
}

raypc_status raypc_serve_release(raypc_server* S, uint64_t id) {
    if (!S) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(RAYPC_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)id);
    Req* q = it->second;
    if (!q->done) return fail(RAYPC_ERR_BUSY, "request %llu still in service", (unsigned long long)id);
    if (q->mem) S->pool.release(q->mem, q->mem_bytes);
    S->all.erase(it);
    delete q;
    S->cv_work.notify_all();
    return RAYPC_OK;
}

}  // extern "C"

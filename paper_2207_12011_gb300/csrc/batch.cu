// Batched rendering: many views (each with its own camera, image size and
// brush box) rendered by one persistent launch, captured once in a CUDA graph
// and replayed with new view tables.
//
// Per batch the host fills a view table (double-buffered in pinned memory);
// the graph uploads it, zeroes the tile counter and the per-view selectivity
// counts, classifies every view's bricks under that view's brush into the
// view's own bitmasks, and runs the persistent render kernel, whose blocks
// pull 16x8-pixel tiles of all views from one atomic counter. Kernel
// parameters never change between batches (everything variable lives in the
// table), so the graph is captured once per table buffer and storage dtype.
#include <vector>

#include "runtime.h"

using namespace raypc;

struct raypc_batch {
    raypc_ctx* ctx = nullptr;
    int max_views = 0;
    size_t table_bytes = 0;
    char* d_table = nullptr;          // BatchHeader, then max_views BatchView (device)
    unsigned* d_counter = nullptr;    // tile counter
    unsigned* d_pass = nullptr;       // max_views x kMaxVars selectivity counts
    unsigned* d_tiles = nullptr;      // max_views finished-tile counters, then max_views sub-brick list lengths
    ViewDone* h_done[2] = {nullptr, nullptr};   // mapped pinned completion records per table slot
    ViewDone* d_done[2] = {nullptr, nullptr};   // their device aliases
    unsigned seq = 0;                 // launch sequence number
    int last_slot = 0;
    char* h_table[2] = {nullptr, nullptr};   // pinned host copies of the table
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    int cur = 0;
    std::vector<uint32_t*> bits;      // per view slot: active words, sub-brick active words, sub-brick list
    std::vector<size_t> bits_words;   // capacity (words) per slot
    std::vector<uint16_t*> cls;       // per view slot: cell classes under the view's brush (n^3 words)
    std::vector<size_t> cls_cells;    // capacity (cells) per slot
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int exec_key[2] = {-1, -1};       // dtype * 16 + variant of the captured graph
    size_t charged = 0;
};

namespace {

constexpr size_t kHeaderBytes = 256;   // BatchHeader padded so the views start aligned

BatchHeader* hdr_of(char* table) { return reinterpret_cast<BatchHeader*>(table); }
BatchView* views_of(char* table) { return reinterpret_cast<BatchView*>(table + kHeaderBytes); }

void wait_idle(raypc_batch* b) {
    for (int i = 0; i < 2; ++i)
        if (b->used[i]) cudaEventSynchronize(b->done[i]);
}

void release(raypc_batch* b) {
    wait_idle(b);
    for (int i = 0; i < 2; ++i) {
        if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
        if (b->h_table[i]) cudaFreeHost(b->h_table[i]);
        if (b->h_done[i]) cudaFreeHost(b->h_done[i]);
        if (b->done[i]) cudaEventDestroy(b->done[i]);
    }
    for (uint32_t* p : b->bits)
        if (p) cudaFree(p);
    for (uint16_t* p : b->cls)
        if (p) cudaFree(p);
    if (b->d_table) cudaFree(b->d_table);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_pass) cudaFree(b->d_pass);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ctx) b->ctx->used -= b->charged < b->ctx->used ? b->charged : b->ctx->used;
}

raypc_status capture(raypc_batch* b, int slot, int dtype, int variant, bool depth) {
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int blocks = sms * render_batch_blocks_per_sm(dtype, variant, depth);
    const unsigned cls_blocks = (unsigned)sms * 8u;
    if (b->exec[slot]) {
        cudaGraphExecDestroy(b->exec[slot]);
        b->exec[slot] = nullptr;
    }
    cudaStream_t s = b->cap_stream;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin graph capture");
    cudaError_t e = cudaMemcpyAsync(b->d_table, b->h_table[slot], b->table_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_pass, 0, sizeof(unsigned) * kMaxVars * b->max_views, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_tiles, 0, sizeof(unsigned) * 2 * b->max_views, s);
    if (e == cudaSuccess)
        e = launch_render_batch(hdr_of(b->d_table), views_of(b->d_table), b->d_counter, depth, dtype, variant,
                                cls_blocks, blocks, s);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[slot], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
    b->exec_key[slot] = dtype * 16 + variant + (depth ? 8 : 0);
    return RAYPC_OK;
}

}  // namespace

void raypc::batch_last_records(raypc_batch* b, const ViewDone** records, unsigned* seq) {
    *records = b->h_done[b->last_slot];
    *seq = b->seq;
}

extern "C" {

raypc_status raypc_batch_create(raypc_ctx* ctx, int max_views, raypc_batch** out) {
    if (!ctx || !out) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (max_views < 1 || max_views > 4096) return fail(RAYPC_ERR_INVALID_ARG, "max_views %d not in 1..4096", max_views);
    *out = nullptr;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    raypc_batch* b = new raypc_batch();
    b->ctx = ctx;
    b->max_views = max_views;
    b->table_bytes = kHeaderBytes + sizeof(BatchView) * (size_t)max_views;
    b->bits.assign(max_views, nullptr);
    b->bits_words.assign(max_views, 0);
    b->cls.assign(max_views, nullptr);
    b->cls_cells.assign(max_views, 0);
    raypc_status st = ctx->alloc((void**)&b->d_table, b->table_bytes, &b->charged);
    if (st == RAYPC_OK) st = ctx->alloc((void**)&b->d_counter, sizeof(unsigned), &b->charged);
    if (st == RAYPC_OK) st = ctx->alloc((void**)&b->d_pass, sizeof(unsigned) * kMaxVars * max_views, &b->charged);
    if (st == RAYPC_OK) st = ctx->alloc((void**)&b->d_tiles, sizeof(unsigned) * 2 * max_views, &b->charged);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && st == RAYPC_OK && e == cudaSuccess; ++i) {
        e = cudaHostAlloc((void**)&b->h_table[i], b->table_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) memset(b->h_table[i], 0, b->table_bytes);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->h_done[i], sizeof(ViewDone) * max_views, cudaHostAllocMapped);
        if (e == cudaSuccess) {
            memset((void*)b->h_done[i], 0, sizeof(ViewDone) * max_views);
            e = cudaHostGetDevicePointer((void**)&b->d_done[i], b->h_done[i], 0);
        }
    }
    if (st == RAYPC_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (st == RAYPC_OK && e != cudaSuccess) st = cuda_fail(e, "batch resources");
    if (st != RAYPC_OK) {
        release(b);
        delete b;
        return st;
    }
    *out = b;
    return RAYPC_OK;
}

raypc_status raypc_batch_destroy(raypc_batch* b) {
    if (!b) return RAYPC_OK;
    {
        std::lock_guard<std::mutex> lk(b->ctx->mu);
        DeviceGuard g(b->ctx->device);
        release(b);
    }
    delete b;
    return RAYPC_OK;
}

raypc_status raypc_render_batch(raypc_batch* b, const raypc_view* views, int nviews, void* stream) {
    if (!b || !views) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (nviews < 1 || nviews > b->max_views) return fail(RAYPC_ERR_INVALID_ARG, "nviews %d not in 1..%d", nviews, b->max_views);
    raypc_ctx* ctx = b->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    const int slot = b->cur;
    // the table buffer of this slot was last read by the batch two calls ago
    if (b->used[slot]) CK(cudaEventSynchronize(b->done[slot]), "wait for the previous use of the view table");
    BatchHeader* H = hdr_of(b->h_table[slot]);
    BatchView* T = views_of(b->h_table[slot]);
    int dtype = -1, variant = 0;
    // a depth output in any view selects the depth instance of the kernel (8x4 tiles)
    bool depth = false;
    for (int i = 0; i < nviews; ++i) depth = depth || views[i].opts.depth_dev != nullptr;
    unsigned long long cls = 0, dist = 0;
    long long tiles = 0;
    raypc_status st;
    for (int i = 0; i < nviews; ++i) {
        const raypc_view& q = views[i];
        Volume* V = nullptr;
        if ((st = get_volume(ctx, q.vol, &V))) return st;
        Level* L = nullptr;
        if ((st = get_level(V, q.lod, &L))) return st;
        if (dtype < 0) dtype = V->dtype;
        if (V->dtype != dtype) return fail(RAYPC_ERR_INVALID_ARG, "view %d: all views of a batch need one storage dtype", i);
        BatchView bv{};
        if ((st = make_render_args(V, L, &q.cam, q.w, q.h, &q.opts, q.out_rgba_dev, q.stats_dev, &bv.a))) return st;
        if ((st = brush_from_host(V, q.lo, q.hi, q.active_mask, &bv.a.brush))) return st;
        if ((st = pos_from_host(q.pos_lo, q.pos_hi, q.pos_mask, &bv.a.brush))) return st;
        finish_position_brush(bv.a);
        if (i == 0) variant = depth ? 1 : bv.a.variant;
        bv.a.variant = variant;
        // per view: brick and sub-brick activity bits, the list of active sub-bricks, and
        // the sub-bricks' empty-space distance with its scratch (bytes)
        const size_t nsub = L->nsbricks();
        const size_t words = L->nwords(), need = words + L->nswords() + nsub + (2 * nsub + 3) / 4;
        if (b->bits_words[i] < need) {
            // growing a slot's masks: no batch may still be reading the old ones
            wait_idle(b);
            if (b->bits[i]) cudaFree(b->bits[i]);
            b->bits[i] = nullptr;
            b->bits_words[i] = 0;
            size_t ch = 0;
            if ((st = ctx->alloc((void**)&b->bits[i], need * sizeof(uint32_t), &ch))) return st;
            b->charged += ch;
            b->bits_words[i] = need;
        }
        bv.a.lv.active = b->bits[i];
        bv.a.lv.sactive = b->bits[i] + words;
        bv.slist = b->bits[i] + words + L->nswords();
        uint8_t* dist_buf = reinterpret_cast<uint8_t*>(b->bits[i] + words + L->nswords() + nsub);
        bv.a.lv.sdist = bv.a.skip ? dist_buf : nullptr;   // renders with skipping jump by the distance
        bv.stmp = dist_buf + nsub;
        bv.dist_begin = dist;
        if (bv.a.skip) dist += (nsub + 31) & ~(size_t)31;
        bv.scount = b->d_tiles + b->max_views + i;
        const size_t cells = (size_t)L->n * L->n * L->n;
        if (b->cls_cells[i] < cells) {
            // growing a slot's cell classes: no batch may still be reading the old ones
            wait_idle(b);
            if (b->cls[i]) cudaFree(b->cls[i]);
            b->cls[i] = nullptr;
            b->cls_cells[i] = 0;
            size_t ch = 0;
            if ((st = ctx->alloc((void**)&b->cls[i], cells * sizeof(uint16_t), &ch))) return st;
            b->charged += ch;
            b->cls_cells[i] = cells;
        }
        bv.a.cls = b->cls[i];
        bv.a.pass_count = b->d_pass + (size_t)i * kMaxVars;
        bv.bmin = L->bmin;
        bv.bmax = L->bmax;
        bv.sbmin = L->sbmin;
        bv.sbmax = L->sbmax;
        bv.cls_begin = cls;
        bv.cls_sub = (unsigned long long)words * 32;
        cls += (unsigned long long)(words + L->nswords()) * 32;
        bv.tiles_x = (q.w + block_tile_w(variant) - 1) / block_tile_w(variant);
        bv.tile_begin = (int)tiles;
        bv.ntiles = bv.tiles_x * ((q.h + block_tile_h(variant) - 1) / block_tile_h(variant));
        tiles += (long long)bv.ntiles;
        bv.tile_done = b->d_tiles + i;
        bv.done = b->d_done[slot] + i;
        bv.seq = b->seq + 1;
        if (tiles > 0x7fffffffLL) return fail(RAYPC_ERR_INVALID_ARG, "batch has more than 2^31 tiles");
        T[i] = bv;
    }
    H->nviews = nviews;
    H->total_tiles = (int)tiles;
    H->cls_total = cls;
    H->dist_total = dist;
    if (!b->exec[slot] || b->exec_key[slot] != dtype * 16 + variant + (depth ? 8 : 0))
        if ((st = capture(b, slot, dtype, variant, depth))) return st;
    CK(cudaGraphLaunch(b->exec[slot], (cudaStream_t)stream), "batch graph launch");
    CK(cudaEventRecord(b->done[slot], (cudaStream_t)stream), "batch completion event");
    b->used[slot] = true;
    b->last_slot = slot;
    b->seq += 1;
    b->cur ^= 1;
    count_launches(6);
    return RAYPC_OK;
}

}  // extern "C"

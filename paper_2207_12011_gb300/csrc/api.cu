// Host runtime behind the C ABI declared in include/raypc.h: contexts,
// resident volumes with their levels of detail, brick min/max and brush
// classification, transfer functions, and the render / histogram entry
// points. Every entry point validates its arguments, enqueues its work on
// the caller's stream and reports failures as status codes with a
// thread-local message; nothing aborts the process.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>

#include "host_math.h"
#include "runtime.h"

using namespace raypc;

namespace {
thread_local std::string g_err;
std::atomic<unsigned long long> g_launches{0};
}  // namespace

namespace raypc {

raypc_status fail(raypc_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

raypc_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(RAYPC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(RAYPC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace raypc

namespace {

void free_level(Level& L) {
    void* ptrs[] = {L.cells, L.pairs, L.bmin, L.bmax, L.active, L.skippable, L.list, L.n_active, L.pass_count,
                    L.sbmin, L.sbmax, L.sactive, L.slist, L.scount, L.cls, L.tf_active, L.tf_sactive,
                    L.sdist, L.sdist_tmp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    L = Level{};
}

void free_bricks(Level& L) {
    void* ptrs[] = {L.bmin, L.bmax, L.active, L.skippable, L.list, L.n_active, L.pass_count,
                    L.sbmin, L.sbmax, L.sactive, L.slist, L.scount, L.tf_active, L.tf_sactive,
                    L.sdist, L.sdist_tmp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    L.bmin = L.bmax = L.sbmin = L.sbmax = nullptr;
    L.active = L.skippable = L.list = L.n_active = L.sactive = L.slist = L.scount = nullptr;
    L.tf_active = L.tf_sactive = nullptr;
    L.sdist = L.sdist_tmp = nullptr;
    L.sdist_of = nullptr;
    L.pass_count = nullptr;
    L.bricks = L.classified = L.cls_valid = false;
}

void free_staging(Volume* V) {
    for (int i = 0; i < 2; ++i) {
        if (V->staging[i]) cudaFree(V->staging[i]);
        if (V->ev_consumed[i]) cudaEventDestroy(V->ev_consumed[i]);
        V->staging[i] = nullptr;
        V->ev_consumed[i] = nullptr;
        V->consumed_pending[i] = false;
    }
    if (V->ev_copied) cudaEventDestroy(V->ev_copied);
    if (V->copy_stream) cudaStreamDestroy(V->copy_stream);
    V->staging_bytes = 0;
    V->stage_next = 0;
    V->ev_copied = nullptr;
    V->copy_stream = nullptr;
}

void free_volume(raypc_ctx* ctx, Volume* V) {
    free_staging(V);
    for (auto& L : V->lv) free_level(L);
    if (V->tf) cudaFree(V->tf);
    if (V->tf_prefix) cudaFree(V->tf_prefix);
    ctx->used -= V->bytes < ctx->used ? V->bytes : ctx->used;
    delete V;
}


// Classify the bricks and sub-bricks of every built level under the current
// brush (three launches total).
raypc_status classify_all(Volume* V, cudaStream_t s) {
    ClassifyArgs c{};
    c.nvars = V->nvars;
    c.rin2 = V->r_in * V->r_in;
    c.rout2 = V->r_out * V->r_out;
    c.brush = V->brush;
    for (int l = 0; l < V->nlev; ++l) {
        Level& L = V->lv[l];
        if (!L.bricks) return fail(RAYPC_ERR_INVALID_ARG, "bricks of level %d are not built", l);
        ClassifyLevel& C = c.lv[c.nlev++];
        C.bmin = L.bmin;
        C.bmax = L.bmax;
        C.n = L.n;
        C.bs = kBrick;
        C.active = L.active;
        C.skippable = L.skippable;
        C.list = L.list;
        C.n_active = L.n_active;
        C.pass_count = L.pass_count;
    }
    c.nbrick = c.nlev;
    for (int l = 0; l < V->nlev; ++l) {
        Level& L = V->lv[l];
        ClassifyLevel& C = c.lv[c.nlev++];
        C.bmin = L.sbmin;
        C.bmax = L.sbmax;
        C.n = L.n;
        C.bs = kSub;
        C.active = L.sactive;
        C.alist = L.slist;
        C.acount = L.scount;
    }
    CK(launch_classify(c, s), "classify kernels");
    for (int l = 0; l < V->nlev; ++l) {
        V->lv[l].classified = true;
        V->lv[l].cls_valid = false;          // cell classes follow the brush; computed on demand
        V->lv[l].sdist_of = nullptr;         // so does the empty-space distance
    }
    return RAYPC_OK;
}

// Lazily classify when a brush is set but the bricks changed since.
raypc_status ensure_classified(Volume* V, Level& L, cudaStream_t s) {
    if (L.classified) return RAYPC_OK;
    if (!V->brush_set) return fail(RAYPC_ERR_INVALID_ARG, "raypc_set_brush must run first");
    return classify_all(V, s);
}

raypc_status alloc_bricks(raypc_ctx* ctx, Volume* V, Level& L) {
    if (L.bmin) return RAYPC_OK;
    size_t nbk = L.nbricks();
    size_t mm = nbk * V->nvars * sizeof(float);
    size_t words = L.nwords() * sizeof(uint32_t);
    size_t smm = L.nsbricks() * V->nvars * sizeof(float);
    raypc_status st;
    if ((st = ctx->alloc((void**)&L.sbmin, smm, &V->bytes)) ||
        (st = ctx->alloc((void**)&L.sbmax, smm, &V->bytes)) ||
        (st = ctx->alloc((void**)&L.sactive, L.nswords() * sizeof(uint32_t), &V->bytes)) ||
        (st = ctx->alloc((void**)&L.tf_sactive, L.nswords() * sizeof(uint32_t), &V->bytes)) ||
        (st = ctx->alloc((void**)&L.tf_active, words, &V->bytes)) ||
        (st = ctx->alloc((void**)&L.slist, L.nsbricks() * sizeof(uint32_t), &V->bytes)) ||
        (st = ctx->alloc((void**)&L.scount, sizeof(uint32_t), &V->bytes)) ||
        (st = ctx->alloc((void**)&L.bmin, mm, &V->bytes)) ||
        (st = ctx->alloc((void**)&L.bmax, mm, &V->bytes)) ||
        (st = ctx->alloc((void**)&L.active, words, &V->bytes)) ||
        (st = ctx->alloc((void**)&L.skippable, words, &V->bytes)) ||
        (st = ctx->alloc((void**)&L.list, nbk * sizeof(uint32_t), &V->bytes)) ||
        (st = ctx->alloc((void**)&L.n_active, sizeof(uint32_t), &V->bytes)) ||
        (st = ctx->alloc((void**)&L.pass_count, sizeof(unsigned) * kMaxVars, &V->bytes))) {
        free_bricks(L);
        return st;
    }
    return RAYPC_OK;
}

// Staging of a host source for raypc_update_volume: two buffers of the volume's own, used in
// turn, and its copy stream (created on first use, charged to the budget). The copy into a
// buffer waits only until the ingest two updates back has read it, so consecutive time steps'
// copies run back to back and overlap whatever runs on the caller's stream; the caller's stream
// waits for the copy. Returns false when the buffers cannot be had (budget), and the caller
// falls back to a stream-ordered temporary.
bool stage_host_source(raypc_ctx* ctx, Volume* V, const void* src, size_t bytes, cudaStream_t s,
                       const void** dsrc, int* slot, raypc_status* st) {
    *st = RAYPC_OK;
    if (V->staging_bytes != bytes) {
        if (V->copy_stream) cudaStreamSynchronize(V->copy_stream);
        for (int i = 0; i < 2; ++i) {
            if (V->consumed_pending[i]) cudaEventSynchronize(V->ev_consumed[i]);
            if (V->staging[i]) cudaFree(V->staging[i]);
            V->staging[i] = nullptr;
            V->consumed_pending[i] = false;
        }
        V->bytes -= 2 * V->staging_bytes < V->bytes ? 2 * V->staging_bytes : V->bytes;
        ctx->used -= 2 * V->staging_bytes < ctx->used ? 2 * V->staging_bytes : ctx->used;
        V->staging_bytes = 0;
        if (ctx->alloc(&V->staging[0], bytes, &V->bytes) != RAYPC_OK) {
            cudaGetLastError();
            return false;
        }
        if (ctx->alloc(&V->staging[1], bytes, &V->bytes) != RAYPC_OK) {
            cudaGetLastError();
            cudaFree(V->staging[0]);
            V->staging[0] = nullptr;
            V->bytes -= bytes < V->bytes ? bytes : V->bytes;
            ctx->used -= bytes < ctx->used ? bytes : ctx->used;
            return false;
        }
        V->staging_bytes = bytes;
        V->stage_next = 0;
    }
    const int i = V->stage_next;
    cudaError_t e = cudaSuccess;
    if (!V->copy_stream) e = cudaStreamCreateWithFlags(&V->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !V->ev_copied) e = cudaEventCreateWithFlags(&V->ev_copied, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        if (!V->ev_consumed[k]) e = cudaEventCreateWithFlags(&V->ev_consumed[k], cudaEventDisableTiming);
    if (e == cudaSuccess && V->consumed_pending[i]) e = cudaStreamWaitEvent(V->copy_stream, V->ev_consumed[i], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(V->staging[i], src, bytes, cudaMemcpyHostToDevice, V->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(V->ev_copied, V->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, V->ev_copied, 0);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "host to device copy");
        return true;
    }
    *dsrc = V->staging[i];
    *slot = i;
    V->stage_next = i ^ 1;
    return true;
}

raypc_status ingest(raypc_ctx* ctx, Volume* V, const void* src, int src_is_device, int src_dtype,
                    cudaStream_t s, bool own_staging = false) {
    Level& L = V->lv[0];
    const size_t nvox = (size_t)L.n * L.n * L.n;
    const void* dsrc = src;
    void* staging = nullptr;
    cudaError_t e;
    bool staged = false;
    int slot = 0;
    if (!src_is_device && own_staging) {
        raypc_status st;
        staged = stage_host_source(ctx, V, src, nvox * V->nvars * elem_size(src_dtype), s, &dsrc, &slot, &st);
        if (st != RAYPC_OK) return st;
    }
    if (!src_is_device && !staged) {
        size_t src_bytes = nvox * V->nvars * elem_size(src_dtype);
        e = cudaMallocAsync(&staging, src_bytes, s);
        if (e != cudaSuccess) return cuda_fail(e, "staging allocation");
        e = cudaMemcpyAsync(staging, src, src_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { cudaFreeAsync(staging, s); return cuda_fail(e, "host to device copy"); }
        dsrc = staging;
    }
    // when the next level is allocated (raypc_build_bricks built it before), its cells and
    // x-pairs come out of the same pass over the source
    Level& C = V->lv[1];
    const bool next = C.cells && C.pairs && C.n * 2 == L.n && ingest_next_level_fits(dsrc, L.n);
    if (next)
        e = launch_ingest_next_level(dsrc, src_dtype, L.cells, L.pairs, V->dtype, L.n, V->nvars, L.bmin, L.bmax,
                                     L.sbmin, L.sbmax, C.cells, C.pairs, s);
    else
        e = launch_ingest(dsrc, src_dtype, L.cells, L.pairs, V->dtype, L.n, V->nvars, L.bmin, L.bmax, L.sbmin,
                          L.sbmax, s);
    C.fresh = next && e == cudaSuccess;
    if (staging) cudaFreeAsync(staging, s);
    if (staged && e == cudaSuccess) {
        e = cudaEventRecord(V->ev_consumed[slot], s);  // the staging buffer is free once this ingest ran
        V->consumed_pending[slot] = e == cudaSuccess;
    }
    if (e != cudaSuccess) return cuda_fail(e, "ingest kernel");
    L.bricks = true;               // level-0 brick min/max come out of the ingest pass
    for (auto& l : V->lv) l.classified = l.cls_valid = false;
    return RAYPC_OK;
}

}  // namespace

void raypc::count_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

namespace raypc {

void set_last_error(const char* msg) { g_err = msg; }

raypc_status get_volume(raypc_ctx* ctx, int vol, Volume** out) {
    auto it = ctx->vols.find(vol);
    if (it == ctx->vols.end()) return fail(RAYPC_ERR_NOT_FOUND, "unknown volume id %d", vol);
    *out = it->second;
    return RAYPC_OK;
}

raypc_status get_level(Volume* V, int lod, Level** out) {
    if (lod < 0 || lod >= V->nlev) return fail(RAYPC_ERR_NOT_FOUND, "level %d not built (have %d)", lod, V->nlev);
    *out = &V->lv[lod];
    return RAYPC_OK;
}

void finish_position_brush(RenderArgs& a) {
    a.keep_lo2 = a.rin2;
    a.keep_hi2 = a.rout2;
    if ((a.brush.pmask >> 3) & 1u) {
        // lo_r <= sqrt_rn(|p|^2) <= hi_r  <=>  L <= |p|^2 <= H for the exact thresholds L, H
        const float L = radius_threshold2(a.brush.plo[3], false), H = radius_threshold2(a.brush.phi[3], true);
        a.keep_lo2 = fmaxf(a.keep_lo2, L);
        a.keep_hi2 = fminf(a.keep_hi2, H);
    }
    a.keep_lo2 = fminf(a.keep_lo2, 0x1p100f);          // finite (the core-jump bound scales it)
}

raypc_status make_render_args(Volume* V, Level* L, const raypc_camera* cam, int w, int h,
                              const raypc_render_opts* opts, float* out_rgba_dev,
                              unsigned long long* stats_dev, RenderArgs* out) {
    if (!cam || !out_rgba_dev) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (w < 1 || h < 1 || w > 32768 || h > 32768) return fail(RAYPC_ERR_INVALID_ARG, "image size %d x %d out of range", w, h);
    if (((uintptr_t)out_rgba_dev) & 15u) return fail(RAYPC_ERR_INVALID_ARG, "out_rgba_dev must be 16-byte aligned");
    for (int i = 0; i < 3; ++i)
        if (!isfinite(cam->eye[i]) || !isfinite(cam->target[i]) || !isfinite(cam->up[i]))
            return fail(RAYPC_ERR_INVALID_ARG, "non-finite camera");
    if (!(cam->tan_half_vfov > 0.f) || !isfinite(cam->tan_half_vfov)) return fail(RAYPC_ERR_INVALID_ARG, "tan_half_vfov must be > 0");
    {
        float fx = cam->target[0] - cam->eye[0], fy = cam->target[1] - cam->eye[1], fz = cam->target[2] - cam->eye[2];
        if (fx == 0.f && fy == 0.f && fz == 0.f) return fail(RAYPC_ERR_INVALID_ARG, "eye == target");
        float cx = fy * cam->up[2] - fz * cam->up[1], cy = fz * cam->up[0] - fx * cam->up[2], cz = fx * cam->up[1] - fy * cam->up[0];
        if (cx == 0.f && cy == 0.f && cz == 0.f) return fail(RAYPC_ERR_INVALID_ARG, "up is parallel to the view direction");
    }
    raypc_render_opts o{};
    o.ert = 1;
    if (opts) o = *opts;
    for (int i = 0; i < 4; ++i)
        if (!isfinite(o.bg[i])) return fail(RAYPC_ERR_INVALID_ARG, "non-finite background");
    if (V->stale) return fail(RAYPC_ERR_INVALID_ARG, "volume updated: raypc_build_bricks must run before render");
    if (!L->bricks) return fail(RAYPC_ERR_INVALID_ARG, "bricks of the level are not built");
    if (!V->tf_set) return fail(RAYPC_ERR_INVALID_ARG, "set_tf must run before render");
    float dt = o.step > 0.f ? o.step : 1.0f / (float)L->n;
    if (!isfinite(dt) || dt < 2.0f * V->r_out / 4194304.0f)
        return fail(RAYPC_ERR_INVALID_ARG, "step %g too small (at most 2^21 samples per chord)", dt);
    RenderArgs a{};
    a.lv.cells = L->cells;
    a.lv.pairs = L->pairs;
    a.lv.n = L->n;
    a.lv.nb = L->nb;
    a.lv.nsb = L->nsb;
    a.lv.sactive = L->sactive;
    a.lv.bmin = L->bmin;
    a.lv.bmax = L->bmax;
    a.lv.active = L->active;
    a.nvars = V->nvars;
    a.brush = V->brush;
    a.pass_count = L->pass_count;
    for (int i = 0; i < 3; ++i) { a.eye[i] = cam->eye[i]; a.target[i] = cam->target[i]; a.up[i] = cam->up[i]; }
    a.tan_half = cam->tan_half_vfov;
    a.w = w;
    a.h = h;
    a.dt = dt;
    a.rin2 = V->r_in * V->r_in;
    a.rout2 = V->r_out * V->r_out;
    finish_position_brush(a);
    a.tf = V->tf;
    a.color_var = V->color_var;
    a.tf_lo = V->tf_lo;
    a.tf_scale = 255.0f / (V->tf_hi - V->tf_lo);
    for (int i = 0; i < 4; ++i) a.bg[i] = o.bg[i];
    a.ert = o.ert ? 1 : 0;
    if (o.skip < RAYPC_AUTO || o.skip > RAYPC_SKIP_OFF) return fail(RAYPC_ERR_INVALID_ARG, "bad skip option %d", o.skip);
    if (o.variant < RAYPC_AUTO || o.variant > kNumVariants) return fail(RAYPC_ERR_INVALID_ARG, "bad variant %d", o.variant);
    int variant = o.variant, skip = o.skip;
    int dev = 0;
    cudaGetDevice(&dev);
    resolve_launch(dev, V->dtype, L->n, &variant, &skip);
    a.skip = skip == RAYPC_SKIP_OFF ? 0 : 1;
    a.variant = variant;
    a.out = reinterpret_cast<float4*>(out_rgba_dev);
    a.counts = o.counts_dev;
    a.depth = o.depth_dev;
    a.tf_prefix = V->tf_prefix;
    a.tf_skip = o.tf_skip ? 1 : 0;
    a.stats = stats_dev;
    *out = a;
    return RAYPC_OK;
}

raypc_status ensure_cell_classes(raypc_ctx* ctx, Volume* V, Level& L, cudaStream_t s) {
    if (L.cls_valid) return RAYPC_OK;
    raypc_status cst = ensure_classified(V, L, s);           // the classes cover the active sub-bricks
    if (cst) return cst;
    if (!L.cls) {
        const size_t bytes = (size_t)L.n * L.n * L.n * sizeof(uint16_t);
        raypc_status st = ctx->alloc((void**)&L.cls, bytes, &V->bytes);
        if (st) return st;
        CK(cudaMemsetAsync(L.cls, 0, bytes, s), "clear cell classes");
    }
    CellClassArgs c{};
    c.pairs = L.pairs;
    c.n = L.n;
    c.nvars = V->nvars;
    c.brush = V->brush;
    c.slist = L.slist;
    c.scount = L.scount;
    c.out = L.cls;
    CK(launch_cell_classes(c, V->dtype, s), "cell class kernel");
    L.cls_valid = true;
    return RAYPC_OK;
}

raypc_status brush_from_host(const Volume* V, const float* lo, const float* hi, uint32_t active_mask, BrushArgs* out) {
    if (!lo || !hi) return fail(RAYPC_ERR_INVALID_ARG, "NULL brush bounds");
    if (active_mask >> V->nvars) return fail(RAYPC_ERR_INVALID_ARG, "active_mask 0x%x names variables >= nvars %d", active_mask, V->nvars);
    BrushArgs b{};
    for (int v = 0; v < kMaxVars; ++v) { b.lo[v] = -INFINITY; b.hi[v] = INFINITY; }
    for (int v = 0; v < V->nvars; ++v) {
        if (isnan(lo[v]) || isnan(hi[v])) return fail(RAYPC_ERR_INVALID_ARG, "NaN brush bound for variable %d", v);
        b.lo[v] = lo[v];
        b.hi[v] = hi[v];
    }
    b.mask = active_mask;
    for (int a = 0; a < kNumPos; ++a) { b.plo[a] = -INFINITY; b.phi[a] = INFINITY; }
    b.pmask = 0u;
    *out = b;
    return RAYPC_OK;
}

raypc_status pos_from_host(const float* lo, const float* hi, uint32_t pos_mask, BrushArgs* b) {
    if (pos_mask >> kNumPos) return fail(RAYPC_ERR_INVALID_ARG, "pos_mask 0x%x names axes >= %d", pos_mask, kNumPos);
    for (int a = 0; a < kNumPos; ++a) { b->plo[a] = -INFINITY; b->phi[a] = INFINITY; }
    b->pmask = pos_mask;
    if (!pos_mask) return RAYPC_OK;
    if (!lo || !hi) return fail(RAYPC_ERR_INVALID_ARG, "NULL position bounds");
    for (int a = 0; a < kNumPos; ++a) {
        if (!((pos_mask >> a) & 1u)) continue;
        if (isnan(lo[a]) || isnan(hi[a])) return fail(RAYPC_ERR_INVALID_ARG, "NaN bound for position axis %d", a);
        b->plo[a] = lo[a];
        b->phi[a] = hi[a];
    }
    return RAYPC_OK;
}

}  // namespace raypc

extern "C" {

const char* raypc_last_error(void) { return g_err.c_str(); }

raypc_status raypc_kernel_launches(unsigned long long* out) {
    if (!out) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    *out = g_launches.load();
    return RAYPC_OK;
}

raypc_status raypc_create(raypc_ctx** out, int device, size_t hbm_budget_bytes) {
    if (!out) return fail(RAYPC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(RAYPC_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, ndev);
    raypc_ctx* c = new raypc_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    *out = c;
    g_err.clear();
    return RAYPC_OK;
}

raypc_status raypc_destroy(raypc_ctx* ctx) {
    if (!ctx) return RAYPC_OK;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard g(ctx->device);
        for (auto& kv : ctx->vols) free_volume(ctx, kv.second);
        ctx->vols.clear();
    }
    delete ctx;
    return RAYPC_OK;
}

raypc_status raypc_memory_used(raypc_ctx* ctx, size_t* out_bytes) {
    if (!ctx || !out_bytes) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    *out_bytes = ctx->used;
    return RAYPC_OK;
}

raypc_status raypc_load_volume(raypc_ctx* ctx, const void* src, int src_is_device, int src_dtype,
                               int store_dtype, int nx, int ny, int nz, int nvars, float r_in,
                               float r_out, void* stream, int* out_vol) {
    if (!ctx || !src || !out_vol) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if ((src_dtype != RAYPC_F32 && src_dtype != RAYPC_F16) || (store_dtype != RAYPC_F32 && store_dtype != RAYPC_F16))
        return fail(RAYPC_ERR_INVALID_ARG, "dtype must be RAYPC_F32 or RAYPC_F16");
    if (nvars < 1 || nvars > RAYPC_MAX_VARS) return fail(RAYPC_ERR_INVALID_ARG, "nvars %d not in 1..%d", nvars, RAYPC_MAX_VARS);
    if (nx < 2 || ny < 2 || nz < 2) return fail(RAYPC_ERR_INVALID_ARG, "grid must be at least 2 cells per axis");
    if (nx != ny || ny != nz) return fail(RAYPC_ERR_UNSUPPORTED, "only cubic grids are supported (%d x %d x %d)", nx, ny, nz);
    if (nx > kMaxRowsEdge) return fail(RAYPC_ERR_UNSUPPORTED, "grid edge %d > %d", nx, kMaxRowsEdge);
    if (!(r_in >= 0.f) || !(r_out > r_in) || !isfinite(r_out))
        return fail(RAYPC_ERR_INVALID_ARG, "need 0 <= r_in < r_out (got %g, %g)", r_in, r_out);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(RAYPC_ERR_CUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = nx;
    const size_t nvox = (size_t)n * n * n;
    Volume* V = new Volume();
    V->nvars = nvars;
    V->dtype = store_dtype;
    V->r_in = r_in;
    V->r_out = r_out;
    Level& L = V->lv[0];
    L.set_edge(n);
    L.cells_bytes = nvox * nvars * elem_size(store_dtype);
    L.pairs_bytes = 2 * L.cells_bytes;
    raypc_status st = ctx->alloc(&L.cells, L.cells_bytes, &V->bytes);
    if (st == RAYPC_OK) st = ctx->alloc(&L.pairs, L.pairs_bytes, &V->bytes);
    if (st == RAYPC_OK) st = alloc_bricks(ctx, V, L);
    if (st != RAYPC_OK) { free_volume(ctx, V); return st; }
    st = ingest(ctx, V, src, src_is_device, src_dtype, s);
    if (st != RAYPC_OK) { free_volume(ctx, V); return st; }
    if (!src_is_device) {
        // keep the simple contract of this entry point: the host source is consumed on return
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { free_volume(ctx, V); return cuda_fail(e, "ingest"); }
    }
    V->nlev = 1;
    int id = ctx->next_id++;
    ctx->vols[id] = V;
    *out_vol = id;
    return RAYPC_OK;
}

raypc_status raypc_update_volume(raypc_ctx* ctx, int vol, const void* src, int src_is_device,
                                 int src_dtype, void* stream) {
    if (!ctx || !src) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (src_dtype != RAYPC_F32 && src_dtype != RAYPC_F16) return fail(RAYPC_ERR_INVALID_ARG, "bad src_dtype");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    if ((st = ingest(ctx, V, src, src_is_device, src_dtype, (cudaStream_t)stream, true))) return st;
    V->stale = true;
    for (int l = 1; l <= RAYPC_MAX_LOD; ++l) V->lv[l].bricks = false;
    return RAYPC_OK;
}

raypc_status raypc_free_volume(raypc_ctx* ctx, int vol) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    ctx->vols.erase(vol);
    cudaDeviceSynchronize();
    free_volume(ctx, V);
    return RAYPC_OK;
}

raypc_status raypc_build_bricks(raypc_ctx* ctx, int vol, int brick_dim, int n_lod, void* stream) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    if (brick_dim != RAYPC_BRICK) return fail(RAYPC_ERR_UNSUPPORTED, "brick_dim must be %d", RAYPC_BRICK);
    if (n_lod < 0 || n_lod > RAYPC_MAX_LOD) return fail(RAYPC_ERR_INVALID_ARG, "n_lod %d not in 0..%d", n_lod, RAYPC_MAX_LOD);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // Level 0 brick min/max come out of every ingest; build the coarser levels,
    // each fused with its own brick min/max.
    for (int l = 1; l <= n_lod; ++l) {
        Level& P = V->lv[l - 1];
        Level& L = V->lv[l];
        int m = (P.n + 1) / 2;
        if (m < 2) return fail(RAYPC_ERR_INVALID_ARG, "level %d would have fewer than 2 cells per axis", l);
        if (!L.cells) {
            L.set_edge(m);
            L.cells_bytes = (size_t)m * m * m * V->nvars * elem_size(V->dtype);
            L.pairs_bytes = 2 * L.cells_bytes;
            st = ctx->alloc(&L.cells, L.cells_bytes, &V->bytes);
            if (st == RAYPC_OK) st = ctx->alloc(&L.pairs, L.pairs_bytes, &V->bytes);
            if (st) return st;
        }
        if ((st = alloc_bricks(ctx, V, L))) return st;
        if (L.fresh)             // the ingest already wrote this level's cells: its bricks only
            CK(launch_level_bricks(L.cells, V->dtype, L.n, V->nvars, L.bmin, L.bmax, L.sbmin, L.sbmax, s),
               "level bricks kernel");
        else
            CK(launch_lod(P.cells, P.n, L.cells, L.pairs, V->dtype, V->nvars, L.bmin, L.bmax, L.sbmin, L.sbmax, s),
               "LOD kernel");
        L.fresh = false;
        L.bricks = true;
    }
    if (V->stale || 1 + n_lod > V->nlev) V->nlev = 1 + n_lod;   // stale coarser levels drop out
    V->stale = false;
    for (auto& L : V->lv) L.classified = L.cls_valid = false;
    return RAYPC_OK;
}

// Re-classify every built level under the volume's (new) brush and compute the
// cell classes of level 0.
static raypc_status reclassify(raypc_ctx* ctx, Volume* V, cudaStream_t s) {
    if (V->stale) {            // coarser levels are rebuilt by raypc_build_bricks, which classifies lazily
        for (auto& L : V->lv) L.classified = L.cls_valid = false;
        return RAYPC_OK;
    }
    raypc_status st = classify_all(V, s);
    if (st) return st;
    // the full-resolution level's cell classes now, so that a render runs its kernel
    // alone (coarser levels get theirs when first rendered)
    return ensure_cell_classes(ctx, V, V->lv[0], s);
}

raypc_status raypc_set_brush(raypc_ctx* ctx, int vol, const float* lo, const float* hi,
                             uint32_t active_mask, void* stream) {
    if (!ctx || !lo || !hi) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    BrushArgs b{};
    if ((st = brush_from_host(V, lo, hi, active_mask, &b))) return st;
    // the position brush stays as raypc_set_position_brush left it
    for (int a = 0; a < kNumPos; ++a) { b.plo[a] = V->brush.plo[a]; b.phi[a] = V->brush.phi[a]; }
    b.pmask = V->brush.pmask;
    V->brush = b;
    V->brush_set = true;
    return reclassify(ctx, V, (cudaStream_t)stream);
}

raypc_status raypc_set_position_brush(raypc_ctx* ctx, int vol, const float* lo, const float* hi,
                                      uint32_t pos_mask, void* stream) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    BrushArgs b = V->brush;
    if (!V->brush_set) {           // no variable brush yet: nothing restricted
        for (int v = 0; v < kMaxVars; ++v) { b.lo[v] = -INFINITY; b.hi[v] = INFINITY; }
        b.mask = 0u;
    }
    if ((st = pos_from_host(lo, hi, pos_mask, &b))) return st;
    V->brush = b;
    V->brush_set = true;
    return reclassify(ctx, V, (cudaStream_t)stream);
}

raypc_status raypc_set_tf(raypc_ctx* ctx, int vol, const float* rgbs, int color_var, float v_lo,
                          float v_hi, void* stream) {
    if (!ctx || !rgbs) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (!(v_lo < v_hi) || !isfinite(v_lo) || !isfinite(v_hi)) return fail(RAYPC_ERR_INVALID_ARG, "need finite v_lo < v_hi");
    for (int i = 0; i < 4 * RAYPC_TF_ENTRIES; ++i)
        if (!isfinite(rgbs[i])) return fail(RAYPC_ERR_INVALID_ARG, "non-finite transfer function entry %d", i);
    for (int i = 0; i < RAYPC_TF_ENTRIES; ++i)
        if (rgbs[4 * i + 3] < 0.f) return fail(RAYPC_ERR_INVALID_ARG, "negative extinction at entry %d", i);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    if (color_var < 0 || color_var >= V->nvars) return fail(RAYPC_ERR_INVALID_ARG, "color_var %d out of range", color_var);
    if (!V->tf) {
        size_t dummy = 0;
        if ((st = ctx->alloc((void**)&V->tf, sizeof(float4) * RAYPC_TF_ENTRIES, &dummy))) return st;
        V->bytes += dummy;
    }
    if (!V->tf_prefix) {
        size_t dummy = 0;
        if ((st = ctx->alloc((void**)&V->tf_prefix, sizeof(int) * (RAYPC_TF_ENTRIES + 1), &dummy))) return st;
        V->bytes += dummy;
    }
    int prefix[RAYPC_TF_ENTRIES + 1];
    prefix[0] = 0;
    for (int i = 0; i < RAYPC_TF_ENTRIES; ++i) prefix[i + 1] = prefix[i] + (rgbs[4 * i + 3] > 0.f ? 1 : 0);
    CK(cudaMemcpyAsync(V->tf_prefix, prefix, sizeof(prefix), cudaMemcpyHostToDevice, (cudaStream_t)stream),
       "transfer function prefix upload");
    // pageable host source: cudaMemcpyAsync stages it before returning
    CK(cudaMemcpyAsync(V->tf, rgbs, sizeof(float4) * RAYPC_TF_ENTRIES, cudaMemcpyHostToDevice, (cudaStream_t)stream),
       "transfer function upload");
    V->color_var = color_var;
    V->tf_lo = v_lo;
    V->tf_hi = v_hi;
    V->tf_set = true;
    return RAYPC_OK;
}

// With tf_skip, the render reads the activity bits ANDed with the TF visibility of
// the level's bricks and sub-bricks (computed for this render on its stream).
// Empty-space distance of the sub-bricks under the activity bits the render reads (the
// brush's, or the TF-visible ones with tf_skip), for renders with skipping.
static raypc_status ensure_distance(raypc_ctx* ctx, Volume* V, Level& L, RenderArgs& a, bool recompute,
                                    cudaStream_t s) {
    if (!a.skip) return RAYPC_OK;
    if (!L.sdist) {
        const size_t bytes = L.nsbricks();
        raypc_status st = ctx->alloc((void**)&L.sdist, bytes, &V->bytes);
        if (st == RAYPC_OK) st = ctx->alloc((void**)&L.sdist_tmp, bytes, &V->bytes);
        if (st) return st;
        L.sdist_of = nullptr;
    }
    if (recompute || L.sdist_of != a.lv.sactive) {
        CK(launch_subbrick_distance(a.lv.sactive, L.nsb, L.sdist, L.sdist_tmp, s), "empty-space distance");
        L.sdist_of = a.lv.sactive;
    }
    a.lv.sdist = L.sdist;
    return RAYPC_OK;
}

static raypc_status apply_tf_skip(Volume* V, Level& L, const raypc_render_opts* opts, RenderArgs& a, cudaStream_t s) {
    if (!opts || !opts->tf_skip) return RAYPC_OK;
    TfVisArgs t{};
    t.n = L.n;
    t.nb = L.nb;
    t.nsb = L.nsb;
    t.nvars = V->nvars;
    t.color_var = V->color_var;
    t.bmin = L.bmin;
    t.bmax = L.bmax;
    t.sbmin = L.sbmin;
    t.sbmax = L.sbmax;
    t.active = L.active;
    t.sactive = L.sactive;
    t.tf = V->tf;
    t.tf_lo = a.tf_lo;
    t.tf_scale = a.tf_scale;
    t.out_active = L.tf_active;
    t.out_sactive = L.tf_sactive;
    CK(launch_tf_visibility(t, s), "TF visibility kernel");
    a.lv.active = L.tf_active;
    a.lv.sactive = L.tf_sactive;
    return RAYPC_OK;
}

raypc_status raypc_render(raypc_ctx* ctx, int vol, int lod, const raypc_camera* cam, int w, int h,
                          const raypc_render_opts* opts, float* out_rgba_dev,
                          unsigned long long* stats_dev, void* stream) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    RenderArgs a{};
    if ((st = make_render_args(V, L, cam, w, h, opts, out_rgba_dev, stats_dev, &a))) return st;
    if ((st = ensure_classified(V, *L, (cudaStream_t)stream))) return st;
    if ((st = ensure_cell_classes(ctx, V, *L, (cudaStream_t)stream))) return st;
    a.cls = L->cls;
    if ((st = apply_tf_skip(V, *L, opts, a, (cudaStream_t)stream))) return st;
    if ((st = ensure_distance(ctx, V, *L, a, opts && opts->tf_skip, (cudaStream_t)stream))) return st;
    CK(launch_render(a, V->dtype, (cudaStream_t)stream), "render kernel");
    return RAYPC_OK;
}

raypc_status raypc_render_progressive(raypc_ctx* ctx, int vol, int lod, const raypc_camera* cam, int w, int h,
                                      const raypc_render_opts* opts, uint32_t seed, uint32_t pass,
                                      float* accum_rgba_dev, float* out_rgba_dev,
                                      unsigned long long* stats_dev, void* stream) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    if (pass == 0xFFFFFFFFu) return fail(RAYPC_ERR_INVALID_ARG, "pass index 2^32 - 1 out of range");
    if (((uintptr_t)accum_rgba_dev) & 15u) return fail(RAYPC_ERR_INVALID_ARG, "accum_rgba_dev must be 16-byte aligned");
    if (accum_rgba_dev && accum_rgba_dev == out_rgba_dev) return fail(RAYPC_ERR_INVALID_ARG, "accum_rgba_dev and out_rgba_dev alias");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    RenderArgs a{};
    if ((st = make_render_args(V, L, cam, w, h, opts, out_rgba_dev, stats_dev, &a))) return st;
    if ((st = ensure_classified(V, *L, (cudaStream_t)stream))) return st;
    if ((st = ensure_cell_classes(ctx, V, *L, (cudaStream_t)stream))) return st;
    a.cls = L->cls;
    a.jit_seed = seed;
    a.jit_pass = pass;
    a.accum = reinterpret_cast<float4*>(accum_rgba_dev);
    a.accum_w = 1.0f / (float)((double)pass + 1.0);
    if ((st = apply_tf_skip(V, *L, opts, a, (cudaStream_t)stream))) return st;
    if ((st = ensure_distance(ctx, V, *L, a, opts && opts->tf_skip, (cudaStream_t)stream))) return st;
    CK(launch_render(a, V->dtype, (cudaStream_t)stream), "render kernel");
    return RAYPC_OK;
}

// PC axis ids: stored variables 0..nvars-1 and position axes RAYPC_AXIS_POS(0..3).
static raypc_status check_axes(const Volume* V, const int* axis_order, int naxes) {
    for (int a = 0; a < naxes; ++a) {
        const int id = axis_order[a];
        const bool ok = (id >= 0 && id < V->nvars) || (id >= kPosAxisBase && id < kPosAxisBase + kNumPos);
        if (!ok) return fail(RAYPC_ERR_INVALID_ARG, "axis %d names variable %d", a, id);
    }
    return RAYPC_OK;
}

raypc_status raypc_pc_histogram(raypc_ctx* ctx, int vol, int lod, const int* axis_order, int naxes,
                                int bins, const float* edges, int use_brush, uint32_t* out_counts_dev,
                                void* stream) {
    if (!ctx || !axis_order || !edges || !out_counts_dev) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (naxes < 2 || naxes > RAYPC_MAX_VARS) return fail(RAYPC_ERR_INVALID_ARG, "naxes %d not in 2..%d", naxes, RAYPC_MAX_VARS);
    if (bins < 2 || bins > 1024) return fail(RAYPC_ERR_INVALID_ARG, "bins %d not in 2..1024", bins);
    for (int a = 0; a < naxes; ++a)
        for (int k = 0; k <= bins; ++k) {
            float e = edges[(size_t)a * (bins + 1) + k];
            if (isnan(e)) return fail(RAYPC_ERR_INVALID_ARG, "NaN edge (axis %d, edge %d)", a, k);
            if (k && e < edges[(size_t)a * (bins + 1) + k - 1]) return fail(RAYPC_ERR_INVALID_ARG, "edges of axis %d decrease at %d", a, k);
        }
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    if ((st = check_axes(V, axis_order, naxes))) return st;
    if (use_brush && !V->brush_set) return fail(RAYPC_ERR_INVALID_ARG, "use_brush needs raypc_set_brush");
    if (V->stale && lod > 0) return fail(RAYPC_ERR_INVALID_ARG, "level %d is stale after raypc_update_volume", lod);
    cudaStream_t s = (cudaStream_t)stream;
    // with the volume's brush, its sub-brick classification lets the kernel skip inactive sub-bricks
    const bool use_activity = use_brush && !V->stale;
    if (use_activity && (st = ensure_classified(V, *L, s))) return st;
    HistArgs h{};
    h.cells = L->cells;
    h.n = L->n;
    h.nvars = V->nvars;
    h.brush = V->brush;
    h.use_brush = use_brush ? 1 : 0;
    h.naxes = naxes;
    h.bins = bins;
    for (int a = 0; a < kMaxVars; ++a) h.axis[a] = a < naxes ? axis_order[a] : 0;
    for (int a = 0; a < naxes; ++a) {
        const float e0 = edges[(size_t)a * (bins + 1)], eN = edges[(size_t)a * (bins + 1) + bins];
        h.guess_e0[a] = e0;
        h.guess_scale[a] = (eN > e0 && isfinite(eN - e0)) ? (float)bins / (eN - e0) : 0.0f;
    }
    h.need_mask = use_brush ? V->brush.mask : 0u;
    for (int a = 0; a < naxes; ++a)
        if (axis_order[a] < kPosAxisBase) h.need_mask |= 1u << axis_order[a];
    double ri = (double)V->r_in * (double)L->n, ro = (double)V->r_out * (double)L->n;
    h.s_in = (int64_t)ceil(ri * ri);
    h.s_out = (int64_t)floor(ro * ro);
    // edges: in the launch parameters when the table is small, else a device copy owned by
    // this call (freed in stream order)
    const size_t ne = (size_t)naxes * (bins + 1);
    float* dedges = nullptr;
    cudaError_t e = cudaSuccess;
    h.edges_host = edges;
    if (ne > (size_t)kHistInlineEdges) {
        CK(cudaMallocAsync((void**)&dedges, sizeof(float) * ne, s), "edge buffer");
        e = cudaMemcpyAsync(dedges, edges, sizeof(float) * ne, cudaMemcpyHostToDevice, s);
    }
    // hot bins of large grids: the blocks spread their atomics over zeroed copies in stream-ordered
    // scratch, summed into the output afterwards (which then needs no clearing); the same
    // scratch holds the row counter that balances the warps
    const size_t count = (size_t)(naxes - 1) * bins * bins;
    const int ncopies = ((uintptr_t)out_counts_dev & 15u) ? 1 : hist_copies(L->n, naxes, bins);
    const size_t copy_bytes = sizeof(uint32_t) * (count * ncopies + 4);
    uint32_t* copies = nullptr;
    if (e == cudaSuccess && ncopies > 1) {
        e = cudaMallocAsync((void**)&copies, copy_bytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(copies, 0, copy_bytes, s);
    } else if (e == cudaSuccess) {
        e = cudaMemsetAsync(out_counts_dev, 0, sizeof(uint32_t) * count, s);
    }
    if (e == cudaSuccess) {
        h.edges = dedges;
        h.out = out_counts_dev;
        h.copies = copies;
        h.ncopies = copies ? ncopies : 1;
        h.rowctr = copies ? copies + count * ncopies : nullptr;
        h.sactive = use_activity ? L->sactive : nullptr;
        h.nsb = L->nsb;
        e = launch_histogram(h, V->dtype, s);
        if (e == cudaSuccess && copies) e = launch_histogram_reduce(copies, ncopies, count, out_counts_dev, s);
    }
    if (copies) cudaFreeAsync(copies, s);
    if (dedges) cudaFreeAsync(dedges, s);
    if (e != cudaSuccess) return cuda_fail(e, "histogram");
    return RAYPC_OK;
}

raypc_status raypc_pc_subsample(raypc_ctx* ctx, int vol, int lod, uint32_t seed, long long k,
                                const int* axis_order, int naxes, long long* out_cells_dev,
                                float* out_values_dev, uint8_t* out_in_brush_dev, long long* out_count,
                                void* stream) {
    if (!ctx || !out_count) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (k < 0 || k > 0x7fffffffLL) return fail(RAYPC_ERR_INVALID_ARG, "k %lld not in 0..2^31-1", k);
    if (naxes < 0 || naxes > RAYPC_MAX_VARS) return fail(RAYPC_ERR_INVALID_ARG, "naxes %d not in 0..%d", naxes, RAYPC_MAX_VARS);
    if (naxes > 0 && !axis_order) return fail(RAYPC_ERR_INVALID_ARG, "NULL axis_order");
    if (k > 0 && (!out_cells_dev || !out_in_brush_dev || (naxes > 0 && !out_values_dev)))
        return fail(RAYPC_ERR_INVALID_ARG, "NULL output");
    if (((uintptr_t)out_cells_dev) & 7u) return fail(RAYPC_ERR_INVALID_ARG, "out_cells_dev must be 8-byte aligned");
    if (((uintptr_t)out_values_dev) & 3u) return fail(RAYPC_ERR_INVALID_ARG, "out_values_dev must be 4-byte aligned");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    if ((st = check_axes(V, axis_order, naxes))) return st;
    if (V->stale && lod > 0) return fail(RAYPC_ERR_INVALID_ARG, "level %d is stale after raypc_update_volume", lod);
    const double ri = (double)V->r_in * (double)L->n, ro = (double)V->r_out * (double)L->n;
    const int64_t s_in = (int64_t)ceil(ri * ri), s_out = (int64_t)floor(ro * ro);
    const unsigned long long N = s_out < 0 ? 0ull : count_in_shell(L->n, s_in, s_out);
    const unsigned long long m = std::min<unsigned long long>((unsigned long long)k, N);
    *out_count = (long long)m;
    if (m == 0) return RAYPC_OK;
    SubsampleArgs a{};
    a.cells = L->cells;
    a.n = L->n;
    a.nvars = V->nvars;
    const int64_t imax = 0x7fffffff;
    a.s_in = (int)std::min<int64_t>(std::max<int64_t>(s_in, 0), imax);
    a.s_out = (int)std::min<int64_t>(s_out, imax);
    a.key = ((unsigned long long)seed << 32) | 0xFFFFFFFFull;
    if (V->brush_set) {
        a.brush = V->brush;
    } else {
        for (int v = 0; v < kMaxVars; ++v) { a.brush.lo[v] = -INFINITY; a.brush.hi[v] = INFINITY; }
        for (int p = 0; p < kNumPos; ++p) { a.brush.plo[p] = -INFINITY; a.brush.phi[p] = INFINITY; }
    }
    a.naxes = naxes;
    for (int i = 0; i < naxes; ++i) {
        a.axis[i] = axis_order[i];
        if (axis_order[i] >= kPosAxisBase) a.use_pos = 1;
    }
    if (a.brush.pmask) a.use_pos = 1;
    a.m = m;
    a.out_cells = out_cells_dev;
    a.out_values = out_values_dev;
    a.out_flags = out_in_brush_dev;
    cudaStream_t s = (cudaStream_t)stream;
    // select state and per-block counts: a small device buffer owned by this call (freed in stream order)
    void* scratch = nullptr;
    CK(cudaMallocAsync(&scratch, pc_subsample_scratch_bytes(), s), "subsample scratch");
    cudaError_t e = launch_pc_subsample(a, V->dtype, m, N, scratch, s);
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "pc subsample");
    return RAYPC_OK;
}

raypc_status raypc_filter_points(raypc_ctx* ctx, int vol, int lod, const float* points_dev, long long npts,
                                 uint8_t* out_pass_dev, void* stream) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    if (npts < 0) return fail(RAYPC_ERR_INVALID_ARG, "npts %lld < 0", npts);
    if (npts > 0 && (!points_dev || !out_pass_dev)) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (((uintptr_t)points_dev) & 3u) return fail(RAYPC_ERR_INVALID_ARG, "points_dev must be 4-byte aligned");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    if (V->stale && lod > 0) return fail(RAYPC_ERR_INVALID_ARG, "level %d is stale after raypc_update_volume", lod);
    RenderArgs r{};                       // the brush and the per-sample |p|^2 range of a render
    if (V->brush_set) {
        r.brush = V->brush;
    } else {
        for (int v = 0; v < kMaxVars; ++v) { r.brush.lo[v] = -INFINITY; r.brush.hi[v] = INFINITY; }
        for (int p = 0; p < kNumPos; ++p) { r.brush.plo[p] = -INFINITY; r.brush.phi[p] = INFINITY; }
    }
    r.rin2 = V->r_in * V->r_in;
    r.rout2 = V->r_out * V->r_out;
    finish_position_brush(r);
    PointFilterArgs a{};
    a.pairs = L->pairs;
    a.n = L->n;
    a.nvars = V->nvars;
    a.brush = r.brush;
    a.keep_lo2 = r.keep_lo2;
    a.keep_hi2 = r.keep_hi2;
    a.pts = points_dev;
    a.npts = npts;
    a.out = out_pass_dev;
    CK(launch_filter_points(a, V->dtype, (cudaStream_t)stream), "point filter kernel");
    return RAYPC_OK;
}

static raypc_status check_camera(const raypc_camera* cam) {
    if (!cam) return fail(RAYPC_ERR_INVALID_ARG, "NULL camera");
    for (int i = 0; i < 3; ++i)
        if (!isfinite(cam->eye[i]) || !isfinite(cam->target[i]) || !isfinite(cam->up[i]))
            return fail(RAYPC_ERR_INVALID_ARG, "non-finite camera");
    if (!(cam->tan_half_vfov > 0.f) || !isfinite(cam->tan_half_vfov)) return fail(RAYPC_ERR_INVALID_ARG, "tan_half_vfov must be > 0");
    float fx = cam->target[0] - cam->eye[0], fy = cam->target[1] - cam->eye[1], fz = cam->target[2] - cam->eye[2];
    if (fx == 0.f && fy == 0.f && fz == 0.f) return fail(RAYPC_ERR_INVALID_ARG, "eye == target");
    float cx = fy * cam->up[2] - fz * cam->up[1], cy = fz * cam->up[0] - fx * cam->up[2], cz = fx * cam->up[1] - fy * cam->up[0];
    if (cx == 0.f && cy == 0.f && cz == 0.f) return fail(RAYPC_ERR_INVALID_ARG, "up is parallel to the view direction");
    return RAYPC_OK;
}

raypc_status raypc_warp_image(raypc_ctx* ctx, const raypc_camera* from, const raypc_camera* to, int w, int h,
                              const float* src_rgba_dev, const float* src_depth_dev, const float* bg,
                              int fill_holes, float* out_rgba_dev, int32_t* out_src_dev, void* stream) {
    if (!ctx || !src_rgba_dev || !src_depth_dev || !out_rgba_dev) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    raypc_status st;
    if ((st = check_camera(from)) || (st = check_camera(to))) return st;
    if (w < 1 || h < 1 || w > 32768 || h > 32768) return fail(RAYPC_ERR_INVALID_ARG, "image size %d x %d out of range", w, h);
    if ((((uintptr_t)src_rgba_dev) | ((uintptr_t)out_rgba_dev)) & 15u)
        return fail(RAYPC_ERR_INVALID_ARG, "src_rgba_dev and out_rgba_dev must be 16-byte aligned");
    if (((uintptr_t)src_depth_dev) & 3u || ((uintptr_t)out_src_dev) & 3u) return fail(RAYPC_ERR_INVALID_ARG, "misaligned depth or source index buffer");
    if (src_rgba_dev == out_rgba_dev) return fail(RAYPC_ERR_INVALID_ARG, "out_rgba_dev must not alias src_rgba_dev");
    WarpArgs a{};
    for (int i = 0; i < 3; ++i) {
        a.from_eye[i] = from->eye[i]; a.from_target[i] = from->target[i]; a.from_up[i] = from->up[i];
        a.to_eye[i] = to->eye[i]; a.to_target[i] = to->target[i]; a.to_up[i] = to->up[i];
    }
    a.from_tan_half = from->tan_half_vfov;
    a.to_tan_half = to->tan_half_vfov;
    a.w = w;
    a.h = h;
    a.src_rgba = reinterpret_cast<const float4*>(src_rgba_dev);
    a.src_depth = src_depth_dev;
    for (int c = 0; c < 4; ++c) {
        a.bg[c] = bg ? bg[c] : 0.0f;
        if (!isfinite(a.bg[c])) return fail(RAYPC_ERR_INVALID_ARG, "non-finite background");
    }
    a.out = reinterpret_cast<float4*>(out_rgba_dev);
    a.out_src = out_src_dev;
    a.fill_holes = fill_holes ? 1 : 0;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // per-pixel selection keys: a device buffer owned by this call (freed in stream order)
    CK(cudaMallocAsync((void**)&a.keys, sizeof(unsigned long long) * (size_t)w * h, s), "warp keys");
    cudaError_t e = launch_warp(a, s);
    cudaFreeAsync(a.keys, s);
    if (e != cudaSuccess) return cuda_fail(e, "warp kernels");
    return RAYPC_OK;
}

raypc_status raypc_volume_info(raypc_ctx* ctx, int vol, int lod, int* out_n, int* out_nvars,
                               int* out_dtype, int* out_bricks_per_axis) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    if (out_n) *out_n = L->n;
    if (out_nvars) *out_nvars = V->nvars;
    if (out_dtype) *out_dtype = V->dtype;
    if (out_bricks_per_axis) *out_bricks_per_axis = L->nb;
    return RAYPC_OK;
}

raypc_status raypc_export_volume(raypc_ctx* ctx, int vol, int lod, void* out_dev, void* stream) {
    if (!ctx || !out_dev) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    CK(cudaMemcpyAsync(out_dev, L->cells, L->cells_bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
       "export copy");
    return RAYPC_OK;
}

raypc_status raypc_get_bricks(raypc_ctx* ctx, int vol, int lod, float* out_min_dev, float* out_max_dev,
                              void* stream) {
    if (!ctx || !out_min_dev || !out_max_dev) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    if (!L->bricks) return fail(RAYPC_ERR_INVALID_ARG, "bricks of level %d not built", lod);
    size_t bytes = L->nbricks() * V->nvars * sizeof(float);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(out_min_dev, L->bmin, bytes, cudaMemcpyDeviceToDevice, s), "copy brick min");
    CK(cudaMemcpyAsync(out_max_dev, L->bmax, bytes, cudaMemcpyDeviceToDevice, s), "copy brick max");
    return RAYPC_OK;
}

raypc_status raypc_get_skip_list(raypc_ctx* ctx, int vol, int lod, uint32_t* active_bits_dev,
                                 uint32_t* skippable_bits_dev, uint32_t* active_list_dev,
                                 uint32_t* n_active_dev, void* stream) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (V->stale) return fail(RAYPC_ERR_INVALID_ARG, "volume updated: raypc_build_bricks must run first");
    if ((st = ensure_classified(V, *L, s))) return st;
    size_t wb = L->nwords() * sizeof(uint32_t);
    if (active_bits_dev) CK(cudaMemcpyAsync(active_bits_dev, L->active, wb, cudaMemcpyDeviceToDevice, s), "copy active bits");
    if (skippable_bits_dev) CK(cudaMemcpyAsync(skippable_bits_dev, L->skippable, wb, cudaMemcpyDeviceToDevice, s), "copy skippable bits");
    if (active_list_dev) CK(cudaMemcpyAsync(active_list_dev, L->list, L->nbricks() * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s), "copy active list");
    if (n_active_dev) CK(cudaMemcpyAsync(n_active_dev, L->n_active, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s), "copy active count");
    return RAYPC_OK;
}

raypc_status raypc_get_cell_classes(raypc_ctx* ctx, int vol, int lod, uint16_t* out_dev, void* stream) {
    if (!ctx || !out_dev) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    if (V->stale) return fail(RAYPC_ERR_INVALID_ARG, "volume updated: raypc_build_bricks must run first");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_cell_classes(ctx, V, *L, s))) return st;
    CK(cudaMemcpyAsync(out_dev, L->cls, (size_t)L->n * L->n * L->n * sizeof(uint16_t), cudaMemcpyDeviceToDevice, s),
       "copy cell classes");
    return RAYPC_OK;
}

raypc_status raypc_get_skip_distance(raypc_ctx* ctx, int vol, int lod, uint8_t* out_dev, void* stream) {
    if (!ctx || !out_dev) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    if (V->stale) return fail(RAYPC_ERR_INVALID_ARG, "volume updated: raypc_build_bricks must run first");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_classified(V, *L, s))) return st;
    RenderArgs a{};
    a.skip = 1;
    a.lv.sactive = L->sactive;
    if ((st = ensure_distance(ctx, V, *L, a, false, s))) return st;
    CK(cudaMemcpyAsync(out_dev, L->sdist, L->nsbricks(), cudaMemcpyDeviceToDevice, s), "copy skip distance");
    return RAYPC_OK;
}

raypc_status raypc_get_sub_bricks(raypc_ctx* ctx, int vol, int lod, float* out_min_dev, float* out_max_dev,
                                  uint32_t* active_bits_dev, void* stream) {
    if (!ctx) return fail(RAYPC_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Volume* V = nullptr;
    raypc_status st = get_volume(ctx, vol, &V);
    if (st) return st;
    Level* L = nullptr;
    if ((st = get_level(V, lod, &L))) return st;
    if (!L->bricks) return fail(RAYPC_ERR_INVALID_ARG, "bricks of level %d not built", lod);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = L->nsbricks() * V->nvars * sizeof(float);
    if (out_min_dev) CK(cudaMemcpyAsync(out_min_dev, L->sbmin, bytes, cudaMemcpyDeviceToDevice, s), "copy sub-brick min");
    if (out_max_dev) CK(cudaMemcpyAsync(out_max_dev, L->sbmax, bytes, cudaMemcpyDeviceToDevice, s), "copy sub-brick max");
    if (active_bits_dev) {
        if (V->stale) return fail(RAYPC_ERR_INVALID_ARG, "volume updated: raypc_build_bricks must run first");
        if ((st = ensure_classified(V, *L, s))) return st;
        CK(cudaMemcpyAsync(active_bits_dev, L->sactive, L->nswords() * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s),
           "copy sub-brick active bits");
    }
    return RAYPC_OK;
}

}  // extern "C"

// Render-launch autotuner: times the tile variants with brick skipping on and
// off on caller-given views (each with its own brush classification and cell
// classes, as a single-view render runs) and keeps the fastest per (device, storage dtype,
// grid edge). Renders and batches asked for RAYPC_AUTO use the table. None of
// the choices changes a pixel; they only change speed. The table can persist
// in a small JSON-lines file named by RAYPC_TUNE_CACHE.
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.h"

using namespace raypc;

namespace {

struct Choice {
    int variant = RAYPC_VARIANT_8x4;
    int skip = RAYPC_SKIP_ON;
    float ms = 0.f;
};

std::mutex g_tune_mu;
std::map<std::string, Choice> g_table;
bool g_loaded = false;

std::string device_tag(int dev) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    char buf[320];
    snprintf(buf, sizeof(buf), "%s/sm%d%d/%dSM", p.name, p.major, p.minor, p.multiProcessorCount);
    for (char* c = buf; *c; ++c)
        if (*c == '"' || *c == '\\' || *c == '\n') *c = '_';
    return buf;
}

std::string key_of(int dev, int dtype, int n) {
    char buf[64];
    snprintf(buf, sizeof(buf), "|%s|%d", dtype == RAYPC_F16 ? "f16" : "f32", n);
    return device_tag(dev) + buf;
}

// One line per entry: {"key": "...", "variant": v, "skip": s, "ms": x}
void load_cache_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = getenv("RAYPC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (fgets(line, sizeof(line), f)) {
        char key[512];
        Choice c;
        if (sscanf(line, " {\"key\": \"%511[^\"]\", \"variant\": %d, \"skip\": %d, \"ms\": %f", key, &c.variant,
                   &c.skip, &c.ms) == 4 &&
            c.variant >= 1 && c.variant <= kNumVariants && (c.skip == RAYPC_SKIP_ON || c.skip == RAYPC_SKIP_OFF))
            g_table[key] = c;
    }
    fclose(f);
}

void save_cache_locked() {
    const char* path = getenv("RAYPC_TUNE_CACHE");
    if (!path || !*path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (auto& kv : g_table)
        fprintf(f, "{\"key\": \"%s\", \"variant\": %d, \"skip\": %d, \"ms\": %.6f}\n", kv.first.c_str(),
                kv.second.variant, kv.second.skip, kv.second.ms);
    fclose(f);
    rename(tmp.c_str(), path);
}

}  // namespace

namespace raypc {

void resolve_launch(int device, int dtype, int n, int* variant, int* skip) {
    if (*variant != RAYPC_AUTO && *skip != RAYPC_AUTO) return;
    Choice c;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_cache_locked();
        auto it = g_table.find(key_of(device, dtype, n));
        if (it != g_table.end()) c = it->second;
    }
    if (*variant == RAYPC_AUTO) *variant = c.variant;
    if (*skip == RAYPC_AUTO) *skip = c.skip;
}

}  // namespace raypc

extern "C" {

raypc_status raypc_get_tuning(raypc_ctx* ctx, int dtype, int n, raypc_tuning* out) {
    if (!ctx || !out) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_locked();
    auto it = g_table.find(key_of(ctx->device, dtype, n));
    if (it == g_table.end()) return fail(RAYPC_ERR_NOT_FOUND, "no tuning for this device, dtype and grid");
    out->variant = it->second.variant;
    out->skip = it->second.skip;
    out->ms = it->second.ms;
    return RAYPC_OK;
}

raypc_status raypc_autotune(raypc_ctx* ctx, const raypc_view* views, int nviews, int reps,
                            raypc_tuning* best_out, raypc_tuning* all_out, void* stream) {
    if (!ctx || !views || !best_out) return fail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (nviews < 1 || nviews > 4096) return fail(RAYPC_ERR_INVALID_ARG, "nviews %d not in 1..4096", nviews);
    if (reps < 1 || reps > 1000) return fail(RAYPC_ERR_INVALID_ARG, "reps %d not in 1..1000", reps);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // classify every view under its own brush into temporary bitmasks
    std::vector<RenderArgs> args(nviews);
    std::vector<void*> temps;
    auto free_temps = [&]() {
        cudaStreamSynchronize(s);
        for (void* p : temps) cudaFree(p);
    };
    int dtype = -1, n0 = 0;
    raypc_status st = RAYPC_OK;
    for (int i = 0; i < nviews && st == RAYPC_OK; ++i) {
        const raypc_view& q = views[i];
        Volume* V = nullptr;
        Level* L = nullptr;
        if ((st = get_volume(ctx, q.vol, &V)) || (st = get_level(V, q.lod, &L))) break;
        if (dtype < 0) { dtype = V->dtype; n0 = L->n; }
        if (V->dtype != dtype) { st = fail(RAYPC_ERR_INVALID_ARG, "view %d: all views need one storage dtype", i); break; }
        raypc_render_opts o = q.opts;
        o.variant = RAYPC_VARIANT_8x4;
        o.skip = RAYPC_SKIP_ON;
        if ((st = make_render_args(V, L, &q.cam, q.w, q.h, &o, q.out_rgba_dev, nullptr, &args[i]))) break;
        args[i].counts = nullptr;
        if ((st = brush_from_host(V, q.lo, q.hi, q.active_mask, &args[i].brush))) break;
        if ((st = pos_from_host(q.pos_lo, q.pos_hi, q.pos_mask, &args[i].brush))) break;
        finish_position_brush(args[i]);
        const size_t words = L->nwords();
        void* bits = nullptr;
        void* list = nullptr;
        void* misc = nullptr;
        void* cls = nullptr;
        cudaError_t e = cudaMalloc(&bits, (2 * words + L->nswords()) * sizeof(uint32_t));
        if (e == cudaSuccess) temps.push_back(bits);
        if (e == cudaSuccess) e = cudaMalloc(&list, L->nbricks() * sizeof(uint32_t) + 16);
        if (e == cudaSuccess) temps.push_back(list);
        if (e == cudaSuccess) e = cudaMalloc(&misc, sizeof(unsigned) * (kMaxVars + 4));
        if (e == cudaSuccess) temps.push_back(misc);
        // cell classes under the view's brush, as a single-view render uses them
        if (e == cudaSuccess) e = cudaMalloc(&cls, (size_t)L->n * L->n * L->n * sizeof(uint16_t));
        if (e == cudaSuccess) temps.push_back(cls);
        void* slist = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&slist, L->nsbricks() * sizeof(uint32_t) + 16);
        if (e == cudaSuccess) temps.push_back(slist);
        void* dist = nullptr;                 // empty-space distance (renders with skipping), + scratch
        if (e == cudaSuccess) e = cudaMalloc(&dist, 2 * L->nsbricks() + 16);
        if (e == cudaSuccess) temps.push_back(dist);
        if (e != cudaSuccess) { st = cuda_fail(e, "tuning buffers"); break; }
        ClassifyArgs c{};
        c.nlev = 2;
        c.nbrick = 1;
        c.nvars = V->nvars;
        c.rin2 = V->r_in * V->r_in;
        c.rout2 = V->r_out * V->r_out;
        c.brush = args[i].brush;
        c.lv[0].bmin = L->bmin;
        c.lv[0].bmax = L->bmax;
        c.lv[0].n = L->n;
        c.lv[0].bs = kBrick;
        c.lv[0].active = (uint32_t*)bits;
        c.lv[0].skippable = (uint32_t*)bits + words;
        c.lv[0].list = (uint32_t*)list;
        c.lv[0].pass_count = (unsigned*)misc;
        c.lv[0].n_active = (uint32_t*)misc + kMaxVars;
        c.lv[1].bmin = L->sbmin;
        c.lv[1].bmax = L->sbmax;
        c.lv[1].n = L->n;
        c.lv[1].bs = kSub;
        c.lv[1].active = (uint32_t*)bits + 2 * words;
        c.lv[1].alist = (uint32_t*)slist;
        c.lv[1].acount = (uint32_t*)misc + kMaxVars + 1;
        cudaError_t ce = launch_classify(c, s);
        if (ce != cudaSuccess) { st = cuda_fail(ce, "tuning classification"); break; }
        args[i].lv.active = c.lv[0].active;
        args[i].lv.sactive = c.lv[1].active;
        CellClassArgs cc{};
        cc.pairs = L->pairs;
        cc.n = L->n;
        cc.nvars = V->nvars;
        cc.brush = args[i].brush;
        cc.slist = c.lv[1].alist;
        cc.scount = c.lv[1].acount;
        cc.out = (uint16_t*)cls;
        ce = launch_cell_classes(cc, V->dtype, s);
        if (ce != cudaSuccess) { st = cuda_fail(ce, "tuning cell classes"); break; }
        args[i].cls = cc.out;
        args[i].pass_count = c.lv[0].pass_count;
        ce = launch_subbrick_distance(args[i].lv.sactive, L->nsb, (uint8_t*)dist, (uint8_t*)dist + L->nsbricks(), s);
        if (ce != cudaSuccess) { st = cuda_fail(ce, "tuning empty-space distance"); break; }
        args[i].lv.sdist = (const uint8_t*)dist;
    }
    if (st != RAYPC_OK) {
        free_temps();
        return st;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Choice best;
    best.ms = -1.f;
    int idx = 0;
    for (int variant = 1; variant <= kNumVariants && st == RAYPC_OK; ++variant) {
        for (int sk = 0; sk < 2 && st == RAYPC_OK; ++sk, ++idx) {
            const int skip = sk == 0 ? RAYPC_SKIP_ON : RAYPC_SKIP_OFF;
            cudaError_t e = cudaSuccess;
            for (int r = -1; r < reps && e == cudaSuccess; ++r) {
                if (r == 0) e = cudaEventRecord(e0, s);
                for (int i = 0; i < nviews && e == cudaSuccess; ++i) {
                    RenderArgs a = args[i];
                    a.variant = variant;
                    a.skip = skip == RAYPC_SKIP_ON ? 1 : 0;
                    e = launch_render(a, dtype, s);
                }
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) { st = cuda_fail(e, "tuning run"); break; }
            ms /= (float)reps;
            if (all_out) {
                all_out[idx].variant = variant;
                all_out[idx].skip = skip;
                all_out[idx].ms = ms;
            }
            if (best.ms < 0.f || ms < best.ms) {
                best.variant = variant;
                best.skip = skip;
                best.ms = ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    free_temps();
    if (st != RAYPC_OK) return st;
    {
        std::lock_guard<std::mutex> tl(g_tune_mu);
        load_cache_locked();
        g_table[key_of(ctx->device, dtype, n0)] = best;
        save_cache_locked();
    }
    best_out->variant = best.variant;
    best_out->skip = best.skip;
    best_out->ms = best.ms;
    return RAYPC_OK;
}

}  // extern "C"

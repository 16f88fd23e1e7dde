// Internal host-runtime types shared by the C-ABI translation units
// (contexts, resident volumes and their levels, error reporting). Not part of
// the public interface; include/raypc.h is.
#pragma once

#include <stdarg.h>
#include <stdio.h>

#include <map>
#include <mutex>
#include <string>

#include "common.cuh"
#include "raypc.h"

namespace raypc {

// Error reporting: the message of the last failing call on this thread.
raypc_status fail(raypc_status code, const char* fmt, ...);
raypc_status cuda_fail(cudaError_t e, const char* what);
void set_last_error(const char* msg);

#define CK(call, what)                                       \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return raypc::cuda_fail(e_, what); \
    } while (0)

// Selects a device for the lifetime of the guard and restores the previous one.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return;
        ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct Level {
    int n = 0, nb = 0, nsb = 0;   // edge, 8^3 bricks per axis, 4^3 sub-bricks per axis
    void* cells = nullptr;     // planar values, storage dtype
    void* pairs = nullptr;     // per-variable x-pairs (render layout)
    size_t cells_bytes = 0, pairs_bytes = 0;
    float* bmin = nullptr;
    float* bmax = nullptr;
    uint32_t* active = nullptr;
    uint32_t* skippable = nullptr;
    uint32_t* list = nullptr;
    uint32_t* n_active = nullptr;
    unsigned* pass_count = nullptr;
    float* sbmin = nullptr;       // [nsb^3][nvars]
    float* sbmax = nullptr;
    uint32_t* sactive = nullptr;  // sub-brick activity bits under the current brush
    uint32_t* slist = nullptr;    // active sub-brick ids (any order) and their number
    uint32_t* scount = nullptr;
    uint16_t* cls = nullptr;      // cell classes under the current brush (n^3), computed on demand
    uint32_t* tf_active = nullptr;   // activity AND TF visibility (renders with tf_skip)
    uint32_t* tf_sactive = nullptr;
    uint8_t* sdist = nullptr;        // empty-space distance of the sub-bricks (renders with skipping)
    uint8_t* sdist_tmp = nullptr;
    const uint32_t* sdist_of = nullptr;   // activity bits the distance was computed from (null: stale)
    bool cls_valid = false;
    bool bricks = false;
    bool classified = false;
    bool fresh = false;           // cells and pairs written by the last ingest of the finer level,
                                  // brick min/max not yet (raypc_build_bricks computes them)
    size_t nbricks() const { return (size_t)nb * nb * nb; }
    size_t nwords() const { return (nbricks() + 31) / 32; }
    size_t nsbricks() const { return (size_t)nsb * nsb * nsb; }
    size_t nswords() const { return (nsbricks() + 31) / 32; }
    void set_edge(int edge) {
        n = edge;
        nb = (edge + kBrick - 1) / kBrick;
        nsb = (edge + kSub - 1) / kSub;
    }
};

struct Volume {
    int nvars = 0, dtype = 0;
    bool stale = false;       // level 0 updated since the last build_bricks
    float r_in = 0.f, r_out = 1.f;
    int nlev = 0;             // built levels (1 + coarser)
    Level lv[1 + RAYPC_MAX_LOD];
    bool brush_set = false;
    BrushArgs brush{};
    float4* tf = nullptr;
    int* tf_prefix = nullptr;     // [257]: TF entries < j with sigma > 0 (TF-aware skipping)
    bool tf_set = false;
    int color_var = 0;
    float tf_lo = 0.f, tf_hi = 1.f;
    size_t bytes = 0;
    // host-source updates: two staging buffers of the source's size used in turn, filled on a
    // copy stream of the volume's own; ev_consumed[i] marks the last ingest that read buffer i
    void* staging[2] = {nullptr, nullptr};
    size_t staging_bytes = 0;
    int stage_next = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied = nullptr, ev_consumed[2] = {nullptr, nullptr};
    bool consumed_pending[2] = {false, false};
};

inline size_t elem_size(int dtype) { return dtype == RAYPC_F16 ? 2 : 4; }

raypc_status get_volume(raypc_ctx* ctx, int vol, Volume** out);
raypc_status get_level(Volume* V, int lod, Level** out);

// Fill the march arguments of one render of level L of volume V (brush and
// classification taken from V / L; callers may override them).
raypc_status make_render_args(Volume* V, Level* L, const raypc_camera* cam, int w, int h,
                              const raypc_render_opts* opts, float* out_rgba_dev,
                              unsigned long long* stats_dev, RenderArgs* a);

// Resolve RAYPC_AUTO launch choices from the tuning table (tune.cu).
void resolve_launch(int device, int dtype, int n, int* variant, int* skip);

// Completion records of a batch's most recent launch: *records points at the
// mapped host array indexed like the launch's views, *seq is the value a
// record's seq field takes when that view is finished (see ViewDone).
void batch_last_records(raypc_batch* b, const ViewDone** records, unsigned* seq);

// Compute the cell classes of level L under the volume's brush if they are
// not current (allocates them on first use).
raypc_status ensure_cell_classes(raypc_ctx* ctx, Volume* V, Level& L, cudaStream_t s);

// Validated brush box of a volume from host arrays (nvars entries each); no position brush.
raypc_status brush_from_host(const Volume* V, const float* lo, const float* hi, uint32_t active_mask, BrushArgs* out);

// Validated position brush (axes x, y, z, radius; bounds read only for axes in pos_mask) into b.
raypc_status pos_from_host(const float* lo, const float* hi, uint32_t pos_mask, BrushArgs* b);

// Per-sample |p|^2 range of a render (keep_lo2, keep_hi2) from its shell radii and the radius
// brush; call after the brush is final.
void finish_position_brush(RenderArgs& a);

}  // namespace raypc

struct raypc_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    std::mutex mu;
    std::map<int, raypc::Volume*> vols;
    int next_id = 1;

    // Device allocation charged against the budget.
    raypc_status alloc(void** p, size_t bytes, size_t* charged) {
        if (budget && used + bytes > budget)
            return raypc::fail(RAYPC_ERR_OOM, "HBM budget exceeded: %zu used + %zu requested > %zu", used, bytes, budget);
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e != cudaSuccess) return raypc::cuda_fail(e, "cudaMalloc");
        used += bytes;
        *charged += bytes;
        return RAYPC_OK;
    }
};

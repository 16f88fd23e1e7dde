// Parallel-coordinates histograms without any device allocation.
//
// raypc_pc_histogram copies the caller's bin edges into a small device buffer
// that it allocates (stream-ordered) on every call. Some callers cannot let a
// library allocate: a host whose device memory is fully reserved up front by
// its own pool (a cudaMalloc there fails or fragments the pool), a real-time
// render loop that must not take the allocator's locks or wait on it, or an
// embedding application that owns every byte of the GPU. For them this entry
// point keeps the edge scratch in a file-scope device array of fixed size and
// runs the same histogram kernel on the caller's own field data.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <stdint.h>

#include <mutex>

#include <cuda.h>

#include "runtime.h"

using namespace raypc;

namespace {

// Largest edge table the entry point accepts: RAYPC_MAX_VARS axes of up to
// 1024 bins (1025 edges each), 32.8 KB. Every GPU that loads the library holds
// this array until the process exits.
constexpr int kMaxEdges = RAYPC_MAX_VARS * (1024 + 1);
static __device__ __align__(256) float g_edge_scratch[kMaxEdges];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;

// The array's device address belongs to the context the library's module was
// loaded into, so it is cached per device together with that context's unique
// id (cuCtxGetId; ids are never reused within a process). A device reset or a
// new context therefore makes the next call look the address up again
// instead of passing a stale one to the kernel.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    float* ptr = nullptr;
};
ScratchAddr g_edge_addr[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_driver_fns_tried = false;

// Reports through raypc_last_error (the message store lives in api.cu).
raypc_status nfail(raypc_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return code;
}

// Unique id of the calling thread's current context, or 0 when none is current
// or the driver entry points are unavailable (then nothing is cached).
unsigned long long current_ctx_id() {
    if (!g_driver_fns_tried) {
        g_driver_fns_tried = true;
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q0 == cudaDriverEntryPointSuccess && q1 == cudaDriverEntryPointSuccess) {
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f1);
        }
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (g_ctx_get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current context of device dev.
// The host-side name g_edge_scratch is only a stand-in, never a device
// address, so it is looked up (cudaGetSymbolAddress, with dev current) once
// per device and context.
raypc_status edge_scratch(int dev, float** out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    ScratchAddr& a = g_edge_addr[dev];
    const unsigned long long before = current_ctx_id();
    if (before != 0 && a.ptr && a.ctx_id == before) {
        *out = a.ptr;
        return RAYPC_OK;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_edge_scratch);
    if (e != cudaSuccess)
        return nfail(RAYPC_ERR_CUDA, "cudaGetSymbolAddress of the edge scratch: %s", cudaGetErrorString(e));
    // the lookup may have created the context: key the address on the one now current
    a.ctx_id = current_ctx_id();
    a.ptr = a.ctx_id ? static_cast<float*>(p) : nullptr;
    *out = static_cast<float*>(p);
    return RAYPC_OK;
}

}  // namespace

extern "C" {

raypc_status raypc_pc_histogram_noalloc(const void* cells_dev, int dtype, int n, int nvars, float r_in,
                                        float r_out, const float* lo, const float* hi,
                                        uint32_t active_mask, int use_brush, const int* axis_order,
                                        int naxes, int bins, const float* edges,
                                        uint32_t* out_counts_dev, void* stream) {
    if (!cells_dev || !axis_order || !edges || !out_counts_dev)
        return nfail(RAYPC_ERR_INVALID_ARG, "NULL argument");
    if (dtype != RAYPC_F32 && dtype != RAYPC_F16) return nfail(RAYPC_ERR_INVALID_ARG, "dtype must be RAYPC_F32 or RAYPC_F16");
    if (n < 2 || n > kMaxRowsEdge) return nfail(RAYPC_ERR_INVALID_ARG, "grid edge %d not in 2..%d", n, kMaxRowsEdge);
    if (reinterpret_cast<uintptr_t>(cells_dev) % (dtype == RAYPC_F32 ? 4 : 2) != 0)
        return nfail(RAYPC_ERR_INVALID_ARG, "cells_dev is not aligned to its element size");
    if (reinterpret_cast<uintptr_t>(out_counts_dev) % 4 != 0)
        return nfail(RAYPC_ERR_INVALID_ARG, "out_counts_dev is not 4-byte aligned");
    if (nvars < 1 || nvars > RAYPC_MAX_VARS) return nfail(RAYPC_ERR_INVALID_ARG, "nvars %d not in 1..%d", nvars, RAYPC_MAX_VARS);
    if (!(r_in >= 0.f) || !(r_out > r_in) || !isfinite(r_out)) return nfail(RAYPC_ERR_INVALID_ARG, "need 0 <= r_in < r_out");
    if (naxes < 2 || naxes > RAYPC_MAX_VARS) return nfail(RAYPC_ERR_INVALID_ARG, "naxes %d not in 2..%d", naxes, RAYPC_MAX_VARS);
    if (bins < 2 || bins > 1024)
        return nfail(RAYPC_ERR_INVALID_ARG, "bins %d not in 2..1024 (the edge scratch holds %d floats)", bins, kMaxEdges);
    if ((size_t)naxes * (bins + 1) > (size_t)kMaxEdges)
        return nfail(RAYPC_ERR_INVALID_ARG, "edge table of %d x %d exceeds the %d-float scratch", naxes, bins + 1, kMaxEdges);
    for (int a = 0; a < naxes; ++a) {
        if (axis_order[a] < 0 || axis_order[a] >= nvars)
            return nfail(RAYPC_ERR_INVALID_ARG, "axis %d names variable %d (stored variables 0..%d only; no position axes here)",
                         a, axis_order[a], nvars - 1);
        for (int k = 0; k <= bins; ++k) {
            float e = edges[(size_t)a * (bins + 1) + k];
            if (isnan(e)) return nfail(RAYPC_ERR_INVALID_ARG, "NaN edge (axis %d, edge %d)", a, k);
            if (k && e < edges[(size_t)a * (bins + 1) + k - 1]) return nfail(RAYPC_ERR_INVALID_ARG, "edges of axis %d decrease at %d", a, k);
        }
    }
    if (use_brush) {
        if (!lo || !hi) return nfail(RAYPC_ERR_INVALID_ARG, "use_brush needs lo and hi");
        if (active_mask >> nvars) return nfail(RAYPC_ERR_INVALID_ARG, "active_mask names variables >= nvars");
        for (int v = 0; v < nvars; ++v)
            if (isnan(lo[v]) || isnan(hi[v])) return nfail(RAYPC_ERR_INVALID_ARG, "NaN brush bound for variable %d", v);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(RAYPC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nfail(RAYPC_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    float* scratch = nullptr;
    raypc_status st = edge_scratch(dev, &scratch);
    if (st != RAYPC_OK) return st;

    cudaStream_t s = (cudaStream_t)stream;
    HistArgs h{};
    h.cells = cells_dev;
    h.n = n;
    h.nvars = nvars;
    for (int v = 0; v < kMaxVars; ++v) { h.brush.lo[v] = -INFINITY; h.brush.hi[v] = INFINITY; }
    if (use_brush)
        for (int v = 0; v < nvars; ++v) { h.brush.lo[v] = lo[v]; h.brush.hi[v] = hi[v]; }
    h.brush.mask = use_brush ? active_mask : 0u;
    h.use_brush = use_brush ? 1 : 0;
    h.naxes = naxes;
    h.bins = bins;
    for (int a = 0; a < kMaxVars; ++a) h.axis[a] = a < naxes ? axis_order[a] : 0;
    for (int a = 0; a < naxes; ++a) {
        const float e0 = edges[(size_t)a * (bins + 1)], eN = edges[(size_t)a * (bins + 1) + bins];
        h.guess_e0[a] = e0;
        h.guess_scale[a] = (eN > e0 && isfinite(eN - e0)) ? (float)bins / (eN - e0) : 0.0f;
    }
    h.need_mask = h.brush.mask;
    for (int a = 0; a < naxes; ++a) h.need_mask |= 1u << axis_order[a];
    double ri = (double)r_in * (double)n, ro = (double)r_out * (double)n;
    h.s_in = (int64_t)ceil(ri * ri);
    h.s_out = (int64_t)floor(ro * ro);
    h.edges = scratch;
    h.out = out_counts_dev;
    // The scratch keeps the previous call's edges; this call overwrites every
    // float it reads. Calls that overlap on the GPU race on the scratch.
    e = cudaMemcpyAsync(scratch, edges, sizeof(float) * naxes * (bins + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out_counts_dev, 0, sizeof(uint32_t) * (size_t)(naxes - 1) * bins * bins, s);
    if (e == cudaSuccess) e = launch_histogram(h, dtype, s);
    if (e != cudaSuccess) return nfail(RAYPC_ERR_CUDA, "histogram: %s", cudaGetErrorString(e));
    return RAYPC_OK;
}

}  // extern "C"

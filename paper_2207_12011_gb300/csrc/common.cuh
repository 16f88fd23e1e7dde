// Internal definitions shared by the CUDA translation units of libraypc.
//
// Integer decisions of the method (how many lattice samples a ray has,
// whether a sample is in the shell, which cell it interpolates from, whether
// its trilinear value passes the brush, which bricks are active) are taken
// with correctly rounded FP32 intrinsics (__fmaf_rn, __fadd_rn, __fsub_rn,
// __fmul_rn, __fdiv_rn, __fsqrt_rn) in one fixed order. The compiler never
// contracts or reorders these, so the decisions do not depend on tiling,
// skipping or launch shape.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace raypc {

constexpr int kBrick = 8;
constexpr int kMaxVars = 8;
constexpr int kTF = 256;
constexpr int kNStats = 8;
constexpr float kErtThreshold = 1.0f - 0x1p-12f;   // A >= 1 - 2^-12 ends a ray

// ---------------------------------------------------------------------------
// Exactly rounded FP32 building blocks (Section 2.2: samples are interpolated
// and tested against the brush in FP32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float lerp_rn(float a, float b, float f) {
    return __fmaf_rn(f, __fsub_rn(b, a), a);
}

__device__ __forceinline__ float dot3_rn(float ax, float ay, float az, float bx, float by, float bz) {
    return __fmaf_rn(az, bz, __fmaf_rn(ay, by, __fmul_rn(ax, bx)));
}

// Clamped cell-centred grid coordinate of world coordinate p on an n-cell
// axis: u = p * n/2 + (n/2 - 1/2), clamped to [0, n-1]; lower index
// i0 = min(floor(u), n-2); weight f = u - i0 (exact).
__device__ __forceinline__ void grid_coord_rn(float p, int n, float hn, float off, int& i0, float& f) {
    float u = __fmaf_rn(p, hn, off);
    u = fminf(fmaxf(u, 0.0f), (float)(n - 1));
    int i = (int)floorf(u);
    i = min(i, n - 2);
    i0 = i;
    f = __fsub_rn(u, (float)i);
}

// Trilinear interpolation of corner values c[dz][dy][dx]: x, then y, then z.
__device__ __forceinline__ float trilerp_rn(float c000, float c100, float c010, float c110,
                                            float c001, float c101, float c011, float c111,
                                            float fx, float fy, float fz) {
    float c00 = lerp_rn(c000, c100, fx);
    float c10 = lerp_rn(c010, c110, fx);
    float c01 = lerp_rn(c001, c101, fx);
    float c11 = lerp_rn(c011, c111, fx);
    float c0 = lerp_rn(c00, c10, fy);
    float c1 = lerp_rn(c01, c11, fy);
    return lerp_rn(c0, c1, fz);
}

// ---------------------------------------------------------------------------
// Storage layouts. Every level of a volume is kept twice in HBM:
//  - cells: planar, one plane of n^3 values per variable in the storage
//    dtype, x fastest: cells[((v * n + z) * n + y) * n + x]. Exactly the
//    method's data; read by the histogram, brick min/max and LOD kernels.
//  - pairs: per variable, the value at x and at min(x+1, n-1) side by side
//    (float2 for FP32, half2 in one 32-bit word for FP16):
//    pairs[((v * n + z) * n + y) * n + x] = (c[x], c[x+1]). One load fetches
//    both x-corners of a trilinear cell, so a variable costs 4 loads per
//    sample; read by the render kernel.
// ---------------------------------------------------------------------------
enum DType : int { kF32 = 0, kF16 = 1 };

template <int DT> struct Pair;

template <> struct Pair<kF32> {
    __device__ __forceinline__ static float2 load(const void* base, size_t idx) {
        return __ldg(reinterpret_cast<const float2*>(base) + idx);
    }
};

template <> struct Pair<kF16> {
    __device__ __forceinline__ static float2 load(const void* base, size_t idx) {
        unsigned w = __ldg(reinterpret_cast<const unsigned*>(base) + idx);
        return __half22float2(*reinterpret_cast<const __half2*>(&w));
    }
};

template <int DT> __device__ __forceinline__ float load_cell(const void* base, size_t idx);
template <> __device__ __forceinline__ float load_cell<kF32>(const void* base, size_t idx) {
    return __ldg(reinterpret_cast<const float*>(base) + idx);
}
template <> __device__ __forceinline__ float load_cell<kF16>(const void* base, size_t idx) {
    return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(base) + idx)));
}

// ---------------------------------------------------------------------------
// Kernel argument blocks.
// ---------------------------------------------------------------------------
struct LevelArgs {
    const void* cells;         // planar values
    const void* pairs;         // x-pairs per variable
    int n;                     // cube edge in cells
    int nb;                    // bricks per axis
    const float* bmin;         // [nb^3][nvars]
    const float* bmax;
    const uint32_t* active;    // bitmask, ceil(nb^3/32) words
    const uint32_t* skippable; // bitmask
};

struct BrushArgs {
    float lo[kMaxVars];
    float hi[kMaxVars];
    uint32_t mask;
};

struct RenderArgs {
    LevelArgs lv;
    int nvars;
    BrushArgs brush;
    const unsigned* pass_count;   // per variable: bricks passing that variable alone (order hint)
    float eye[3], target[3], up[3], tan_half;
    int w, h;
    float dt;
    float rin2, rout2;            // r_in * r_in, r_out * r_out rounded to FP32
    const float4* tf;             // 256 entries (r, g, b, sigma)
    int color_var;
    float tf_lo, tf_scale;        // s = (v - tf_lo) * tf_scale
    float bg[4];
    int ert, skip;
    float4* out;
    uint32_t* counts;             // optional [h][w][2]
    unsigned long long* stats;    // optional kNStats counters
};

struct HistArgs {
    const void* cells;
    int n;
    int nvars;
    BrushArgs brush;
    int use_brush;
    unsigned need_mask;           // variables the kernel must load (brushed and axes)
    int naxes, bins;
    int axis[kMaxVars];
    const float* edges;           // naxes x (bins + 1), device
    float guess_e0[kMaxVars];     // per axis: first edge and bins / (last - first), for the
    float guess_scale[kMaxVars];  // starting guess of the bin walk (any value is correct)
    int64_t s_in, s_out;
    uint32_t* out;                // (naxes-1) x bins x bins
};

// Classification of all built levels of a volume in one launch per kernel.
struct ClassifyLevel {
    const float* bmin;
    const float* bmax;
    int n;                        // level edge
    float sc;                     // 2 / n, set by the launcher
    size_t first;                 // first flat index of this level (multiple of 32), set by the launcher
    uint32_t* active;
    uint32_t* skippable;
    uint32_t* list;
    uint32_t* n_active;
    unsigned* pass_count;
};

struct ClassifyArgs {
    int nlev;
    int nvars;
    float rin2, rout2;            // r_in * r_in, r_out * r_out rounded to FP32
    BrushArgs brush;
    size_t total;                 // set by the launcher
    ClassifyLevel lv[3];
};

// Process-wide count of launched kernels (defined in api.cu).
void count_launches(int k);

// Launchers (defined in the .cu files; all enqueue on `stream`).
// Ingest (level 0) and LOD (coarser level) also write the level's brick min/max.
cudaError_t launch_ingest(const void* src, int src_dtype, void* cells, void* pairs, int dtype,
                          int n, int nvars, float* bmin, float* bmax, cudaStream_t stream);
cudaError_t launch_lod(const void* fine, int n_fine, void* cells, void* pairs, int dtype, int nvars,
                       float* bmin, float* bmax, cudaStream_t stream);
cudaError_t launch_classify(ClassifyArgs& c, cudaStream_t stream);
cudaError_t launch_render(const RenderArgs& a, int dtype, cudaStream_t stream);
cudaError_t launch_histogram(const HistArgs& a, int dtype, cudaStream_t stream);

}  // namespace raypc

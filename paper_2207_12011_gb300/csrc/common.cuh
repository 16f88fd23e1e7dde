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
// Storage layout. A level of a volume is n^3 vertices, each holding VP
// element slots (VP >= nvars, padding is zero), x fastest:
//   data[((z * n + y) * n + x) * VP + v]
// FP16 levels use VP = 8 (one 16-byte vector per vertex); FP32 levels use
// VP = 4 (one 16-byte vector, nvars <= 4) or VP = 8 (two vectors).
// ---------------------------------------------------------------------------
enum DType : int { kF32 = 0, kF16 = 1 };

template <int DT, int VP> struct Vertex;

template <> struct Vertex<kF16, 8> {
    uint4 w;
    __device__ __forceinline__ static Vertex load(const void* base, size_t idx) {
        Vertex r;
        r.w = __ldg(reinterpret_cast<const uint4*>(base) + idx);
        return r;
    }
    template <int V> __device__ __forceinline__ float get() const {
        uint32_t word = (V >> 1) == 0 ? w.x : (V >> 1) == 1 ? w.y : (V >> 1) == 2 ? w.z : w.w;
        unsigned short bits = (V & 1) ? (unsigned short)(word >> 16) : (unsigned short)(word & 0xFFFFu);
        return __half2float(__ushort_as_half(bits));
    }
};

template <> struct Vertex<kF32, 4> {
    float4 a;
    __device__ __forceinline__ static Vertex load(const void* base, size_t idx) {
        Vertex r;
        r.a = __ldg(reinterpret_cast<const float4*>(base) + idx);
        return r;
    }
    template <int V> __device__ __forceinline__ float get() const {
        return V == 0 ? a.x : V == 1 ? a.y : V == 2 ? a.z : a.w;
    }
};

template <> struct Vertex<kF32, 8> {
    float4 a, b;
    __device__ __forceinline__ static Vertex load(const void* base, size_t idx) {
        Vertex r;
        const float4* p = reinterpret_cast<const float4*>(base) + 2 * idx;
        r.a = __ldg(p);
        r.b = __ldg(p + 1);
        return r;
    }
    template <int V> __device__ __forceinline__ float get() const {
        return V == 0 ? a.x : V == 1 ? a.y : V == 2 ? a.z : V == 3 ? a.w
             : V == 4 ? b.x : V == 5 ? b.y : V == 6 ? b.z : b.w;
    }
};

// ---------------------------------------------------------------------------
// Kernel argument blocks.
// ---------------------------------------------------------------------------
struct LevelArgs {
    const void* data;          // interleaved vertices
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
    const void* data;
    int n;
    int nvars;
    BrushArgs brush;
    int use_brush;
    int naxes, bins;
    int axis[kMaxVars];
    const float* edges;           // naxes x (bins + 1), device
    int64_t s_in, s_out;
    uint32_t* out;                // (naxes-1) x bins x bins
};

// Process-wide count of launched kernels (defined in api.cu).
void count_launches(int k);

// Launchers (defined in the .cu files; all enqueue on `stream`).
cudaError_t launch_ingest(const void* src, int src_dtype, void* dst, int dst_dtype, int vp,
                          int n, int nvars, cudaStream_t stream);
cudaError_t launch_export(const void* src, int dtype, int vp, void* dst, int n, int nvars,
                          cudaStream_t stream);
cudaError_t launch_lod(const void* src, int n_src, void* dst, int dtype, int vp, int nvars,
                       cudaStream_t stream);
cudaError_t launch_brick_minmax(const void* data, int dtype, int vp, int n, int nvars,
                                float* bmin, float* bmax, cudaStream_t stream);
cudaError_t launch_classify(const float* bmin, const float* bmax, int n, int nvars, float r_in,
                            float r_out, const BrushArgs& brush, uint32_t* active,
                            uint32_t* skippable, uint32_t* list, uint32_t* n_active,
                            unsigned* pass_count, cudaStream_t stream);
cudaError_t launch_render(const RenderArgs& a, int dtype, int vp, cudaStream_t stream);
cudaError_t launch_histogram(const HistArgs& a, int dtype, int vp, cudaStream_t stream);

}  // namespace raypc

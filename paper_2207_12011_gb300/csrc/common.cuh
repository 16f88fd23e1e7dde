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
constexpr int kSub = 4;          // edge of the sub-bricks whose activity the render tests per sample
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
// axis: u = p * n/2 + (n/2 - 1/2) clamped to [0, n-1], lower index
// i0 = min(floor(u), n-2), weight f = u - i0 (exact). grid_index_rn gives i0
// from the integer side -- min(max(floor(u), 0), n-2) equals
// min(floor(clamp(u, 0, n-1)), n-2) for every u -- and returns the unclamped
// u, from which grid_weight_rn (nm1 = n-1) gives f when a sample needs it.
__device__ __forceinline__ int grid_index_rn(float p, int n, float hn, float off, float& u) {
    u = __fmaf_rn(p, hn, off);
    return min(max(__float2int_rd(u), 0), n - 2);
}

__device__ __forceinline__ float grid_weight_rn(float u, int i, float nm1) {
    return __fsub_rn(fminf(fmaxf(u, 0.0f), nm1), (float)i);
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

// Exactly rounded vector helpers of the camera model.
__device__ __forceinline__ void normalize_rn(float& x, float& y, float& z) {
    float l = __fsqrt_rn(dot3_rn(x, y, z, x, y, z));
    x = __fdiv_rn(x, l);
    y = __fdiv_rn(y, l);
    z = __fdiv_rn(z, l);
}

__device__ __forceinline__ void cross_rn(float ax, float ay, float az, float bx, float by, float bz,
                                         float& cx, float& cy, float& cz) {
    cx = __fmaf_rn(ay, bz, -__fmul_rn(az, by));
    cy = __fmaf_rn(az, bx, -__fmul_rn(ax, bz));
    cz = __fmaf_rn(ax, by, -__fmul_rn(ay, bx));
}

// Pinhole camera basis (exactly rounded, fixed order): F = normalize(target - eye),
// R = normalize(cross(F, up)), U = cross(R, F).
__device__ __forceinline__ void camera_basis_rn(const float* eye, const float* target, const float* up,
                                                float& Fx, float& Fy, float& Fz, float& Rx, float& Ry, float& Rz,
                                                float& Ux, float& Uy, float& Uz) {
    Fx = __fsub_rn(target[0], eye[0]);
    Fy = __fsub_rn(target[1], eye[1]);
    Fz = __fsub_rn(target[2], eye[2]);
    normalize_rn(Fx, Fy, Fz);
    cross_rn(Fx, Fy, Fz, up[0], up[1], up[2], Rx, Ry, Rz);
    normalize_rn(Rx, Ry, Rz);
    cross_rn(Rx, Ry, Rz, Fx, Fy, Fz, Ux, Uy, Uz);
}

// Unit direction of the ray through pixel (px, py) of a w x h image.
__device__ __forceinline__ void camera_ray_rn(const float* eye, const float* target, const float* up, float tan_half,
                                              int w, int h, int px, int py, float& dx, float& dy, float& dz) {
    float Fx, Fy, Fz, Rx, Ry, Rz, Ux, Uy, Uz;
    camera_basis_rn(eye, target, up, Fx, Fy, Fz, Rx, Ry, Rz, Ux, Uy, Uz);
    const float aspect = __fdiv_rn((float)w, (float)h);
    const float sxs = __fmul_rn(tan_half, aspect);
    const float qx = __fdiv_rn((float)(2 * px + 1), (float)w);
    const float qy = __fdiv_rn((float)(2 * py + 1), (float)h);
    const float sx = __fmul_rn(__fsub_rn(qx, 1.0f), sxs);
    const float sy = __fmul_rn(__fsub_rn(1.0f, qy), tan_half);
    dx = __fmaf_rn(sy, Ux, __fmaf_rn(sx, Rx, Fx));
    dy = __fmaf_rn(sy, Uy, __fmaf_rn(sx, Ry, Fy));
    dz = __fmaf_rn(sy, Uz, __fmaf_rn(sx, Rz, Fz));
    normalize_rn(dx, dy, dz);
}

// SplitMix64 (Steele, Lea and Flood 2014) as a counter-based generator: the
// output function of the state key + (i + 1) * 0x9E3779B97F4A7C15 for stream
// `key` and counter i. The output function is a bijection of 64-bit words.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long key, unsigned long long i) {
    unsigned long long z = key + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Lattice offset of pixel index pix in progressive pass `pass` (Section 2:
// passes keep refining the image while the camera rests): pass 0 uses 1/2 (the
// fixed lattice t0 + (k + 1/2) dt); pass p >= 1 takes the top 24 bits of
// splitmix64_at(seed * 2^32 + p, pix) as a fraction in [0, 1). The stream
// seed * 2^32 + 2^32 - 1 is reserved for the PC line subsample.
__device__ __forceinline__ float lattice_offset(uint32_t seed, uint32_t pass, unsigned long long pix) {
    if (pass == 0u) return 0.5f;
    const unsigned long long z = splitmix64_at((((unsigned long long)seed) << 32) | pass, pix);
    return (float)(unsigned)(z >> 40) * 0x1p-24f;
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
    int nsb;                   // sub-bricks per axis
    const float* bmin;         // [nb^3][nvars]
    const float* bmax;
    const uint32_t* active;    // bitmask, ceil(nb^3/32) words
    const uint32_t* sactive;   // sub-brick bitmask, ceil(nsb^3/32) words
    const uint8_t* sdist;      // optional: empty-space distance of the sub-bricks under sactive (see
                               // launch_subbrick_distance); renders with skipping jump by it
};

// Cap of the sub-brick empty-space distance (sub-bricks).
constexpr int kDistCap = 8;

// Implicit position axes (x, y, z, radius) usable in brushes and as PC axes;
// PC axis id kPosAxisBase + a names position axis a.
constexpr int kNumPos = 4;
constexpr int kPosAxisBase = 8;

struct BrushArgs {
    float lo[kMaxVars];
    float hi[kMaxVars];
    uint32_t mask;
    float plo[kNumPos];           // position brush: axis a restricted iff bit a of pmask
    float phi[kNumPos];
    uint32_t pmask;
};

// Position axis a of point (x, y, z) whose squared radius r2 =
// dot3_rn(p, p) is known: the coordinate, or (a = 3) the radius sqrt_rn(r2).
__device__ __forceinline__ float pos_axis(float x, float y, float z, float r2, int a) {
    return a == 0 ? x : (a == 1 ? y : (a == 2 ? z : __fsqrt_rn(r2)));
}

// Whether a point passes the position brush (inclusive bounds, every restricted axis).
__device__ __forceinline__ bool pos_pass(float x, float y, float z, float r2, const BrushArgs& b) {
#pragma unroll
    for (int a = 0; a < kNumPos; ++a) {
        if (!((b.pmask >> a) & 1u)) continue;
        const float v = pos_axis(x, y, z, r2, a);
        if (!(v >= b.plo[a] && v <= b.phi[a])) return false;
    }
    return true;
}

// Centre coordinate of cell index i on an axis of n cells: RN((2i + 1 - n) / n).
__device__ __forceinline__ float cell_centre_rn(int i, int n) {
    return __fdiv_rn((float)(2 * i + 1 - n), (float)n);
}

struct RenderArgs {
    LevelArgs lv;
    int nvars;
    BrushArgs brush;
    const unsigned* pass_count;   // per variable: bricks passing that variable alone (order hint)
    float eye[3], target[3], up[3], tan_half;
    int w, h;
    float dt;
    float rin2, rout2;            // r_in * r_in, r_out * r_out rounded to FP32
    float keep_lo2, keep_hi2;     // per-sample |p|^2 range of the shell and the radius brush
                                  // (set by finish_position_brush)
    const float4* tf;             // 256 entries (r, g, b, sigma)
    int color_var;
    float tf_lo, tf_scale;        // s = (v - tf_lo) * tf_scale
    float bg[4];
    int ert, skip;
    int variant;                  // 1..kNumVariants (tile shape of the launch)
    uint32_t jit_seed, jit_pass;  // progressive pass (0: the fixed lattice t0 + (k + 1/2) dt)
    float4* accum;                // optional running mean of the passes ([h][w], updated in place)
    float accum_w;                // 1 / (jit_pass + 1)
    const uint16_t* cls;          // optional cell classes under this brush (kCellFail / need bits), n^3
    float4* out;
    uint32_t* counts;             // optional [h][w][2]
    float* depth;                 // optional [h][w]: t of the first kept sample, +inf if none
    const int* tf_prefix;         // [kTF + 1]: entries < j with sigma > 0 (TF visibility)
    int tf_skip;                  // batched views: classify against the TF visibility too
    unsigned long long* stats;    // optional kNStats counters
};

// Completion record of one view, in mapped pinned host memory: the block that
// finishes the view's last tile copies the view's statistics here and then
// stores the launch sequence number (after a system-scope fence), so the host
// sees a finished view without waiting for the whole launch.
struct ViewDone {
    volatile unsigned seq;
    unsigned pad;
    unsigned long long stats[kNStats];
};

// One view of a batched render: the march arguments (lv.active / lv.sactive /
// pass_count point at this view's own classification), the
// level's brick and sub-brick min/max for that classification, and the view's
// ranges in the flat brick and tile spaces of the batch. A view's flat brick
// range holds its bricks (padded to a multiple of 32) followed by its
// sub-bricks.
struct BatchView {
    RenderArgs a;
    const float* bmin;
    const float* bmax;
    const float* sbmin;
    const float* sbmax;
    unsigned long long cls_begin;  // first flat brick index (multiple of 32)
    unsigned long long cls_sub;    // offset of the first sub-brick in the view's range (multiple of 32)
    uint32_t* slist;               // active sub-bricks of the view (any order), for its cell classes
    uint32_t* scount;              // their number (zeroed per launch)
    int tiles_x;                   // tiles per image row
    int tile_begin;                // first flat tile index
    int ntiles;                    // tiles of this view
    unsigned seq;                  // launch sequence number written on completion
    unsigned* tile_done;           // device counter of finished tiles (zeroed per launch)
    ViewDone* done;                // device alias of the mapped host record (may be null)
    uint8_t* stmp;                 // nsb^3 bytes of scratch for the view's empty-space distance
    unsigned long long dist_begin; // first flat sub-brick index of the view's distance range (multiple
                                   // of 32; the range is empty for views that render without skipping)
};

struct BatchHeader {
    int nviews;
    int total_tiles;
    unsigned long long cls_total;  // flat brick range over all views (multiple of 32)
    unsigned long long dist_total; // flat sub-brick range of the distance passes over all views
};

// Render launch variants: a 128-thread block is 2 x 2 warps; each warp marches
// a WTW x (32 / WTW) pixel tile. Variant 1: 8 x 4 warps (16 x 8 block tile),
// 2: 16 x 2 (32 x 4), 3: 4 x 8 (8 x 16). All variants produce identical
// pixels (the march of a pixel does not depend on the tiling).
constexpr int kRenderThreads = 128;
constexpr int kNumVariants = 3;
__host__ __device__ constexpr int warp_tile_w(int variant) { return variant == 2 ? 16 : variant == 3 ? 4 : 8; }
__host__ __device__ constexpr int block_tile_w(int variant) { return 2 * warp_tile_w(variant); }
__host__ __device__ constexpr int block_tile_h(int variant) { return 2 * (32 / warp_tile_w(variant)); }

// Partial histograms of a spread-out histogram call: enough copies that the
// hottest bins of a smooth field no longer serialise the L2 atomics, within
// kHistCopyBytes of scratch.
constexpr int kHistMaxCopies = 16;
constexpr size_t kHistCopyBytes = (size_t)32 << 20;
int hist_copies(int n, int naxes, int bins);
// Sums the copies into out (launch after launch_histogram on the same stream).
cudaError_t launch_histogram_reduce(const uint32_t* copies, int ncopies, size_t count, uint32_t* out,
                                    cudaStream_t stream);

// Histogram edge tables of at most this many floats (8 axes x 257 edges) are
// passed to the kernel in its launch parameters; larger ones need a device copy.
constexpr int kHistInlineEdges = 8 * 257;

struct HistArgs {
    const void* cells;
    int n;
    int nvars;
    BrushArgs brush;
    int use_brush;
    unsigned need_mask;           // variables the kernel must load (brushed and axes)
    int naxes, bins;
    int axis[kMaxVars];
    const float* edges;           // naxes x (bins + 1), device (may be null when edges_host is given)
    const float* edges_host;      // naxes x (bins + 1), host: small tables travel in the launch parameters
    float guess_e0[kMaxVars];     // per axis: first edge and bins / (last - first), for the
    float guess_scale[kMaxVars];  // starting guess of the bin walk (any value is correct)
    int64_t s_in, s_out;
    uint32_t* out;                // (naxes-1) x bins x bins
    uint32_t* copies;             // optional: ncopies zeroed partial histograms that the blocks spread
    int ncopies;                  // their atomics over (hot bins), summed into out afterwards
    uint32_t* rowctr;             // optional: a zeroed counter from which the warps take their rows
                                  // (null: rows by warp stride)
    const uint32_t* sactive;      // optional: 4^3 sub-brick activity under this brush (cells of inactive
    int nsb;                      // sub-bricks are never counted), sub-bricks per axis
};

// World box that the samples assigned to brick b of edge bs (lower
// interpolation index in [bs b, bs b + bs)) can occupy along one axis, widened
// by 2^-10; the first and last bricks also own the clamped border.
__device__ __forceinline__ void brick_box_axis(int b, int nb, float sc, int bs, float& lo, float& hi) {
    lo = __fsub_rn(__fmaf_rn(__fadd_rn((float)(b * bs), 0.5f), sc, -1.0f), 0x1p-10f);
    hi = __fadd_rn(__fmaf_rn(__fadd_rn((float)(b * bs + bs), 0.5f), sc, -1.0f), 0x1p-10f);
    if (b == 0) lo = -2.0f;
    if (b == nb - 1) hi = 2.0f;
}

// TF entry index J(v) of a colour value, as the march computes it (FP32, monotone in v).
__device__ __forceinline__ int tf_entry(float v, float tf_lo, float tf_scale) {
    float sp = __fmul_rn(__fsub_rn(v, tf_lo), tf_scale);
    sp = fminf(fmaxf(sp, 0.0f), 255.0f);
    return min((int)sp, kTF - 2);
}

// TF visibility of a brick whose colour values lie in [mn, mx] (prefix[j] =
// entries < j with sigma > 0): visible iff sigma > 0 at entry 0 (a NaN colour
// value lands there), or the range cannot be bounded (max(|mn|,|mx|) > 2^126),
// or sigma > 0 at an entry of J(mn - d) .. J(mx + d) + 1, d the brush margin
// that bounds the FP32 interpolation. A sample whose two entries both have
// sigma = 0 adds exactly nothing to the image.
__device__ __forceinline__ bool tf_range_visible(float mn, float mx, const int* prefix, float tf_lo, float tf_scale) {
    if (prefix[1] > 0) return true;
    const float m = fmaxf(fabsf(mn), fabsf(mx));
    if (!(m <= 0x1p126f)) return true;
    const float d = __fmaf_rn(m, 0x1p-20f, 0x1p-120f);
    const int j0 = tf_entry(__fsub_rn(mn, d), tf_lo, tf_scale);
    const int j1 = tf_entry(__fadd_rn(mx, d), tf_lo, tf_scale) + 1;
    return j0 <= j1 && prefix[j1 + 1] - prefix[j0] > 0;
}

// Brush classification of brick b (edge bs) of a level with nb such bricks per
// axis (sc = 2/n): active iff its widened sample box meets the shell and, for every
// restricted v, max_v + d >= lo_v and min_v - d <= hi_v with
// d = max(|min_v|, |max_v|) * 2^-20 + 2^-120 (covers FP32 interpolation
// rounding), and the box meets the position brush. A variable with
// max(|min_v|, |max_v|) > 2^126 never deactivates
// a brick (a corner difference can overflow and the interpolated value be
// infinite). pass_bits gets bit v set for each restricted variable the brick
// passes on its own (only meaningful when the box meets the shell).
__device__ __forceinline__ bool classify_brick(size_t b, int nb, int bs, float sc, float rin2, float rout2,
                                               const BrushArgs& brush, int nvars, const float* bmin,
                                               const float* bmax, unsigned& pass_bits) {
    int c[3] = {(int)(b % nb), (int)((b / nb) % nb), (int)(b / ((size_t)nb * nb))};
    float nearc[3], farc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float lo, hi;
        brick_box_axis(c[a], nb, sc, bs, lo, hi);
        nearc[a] = (lo > 0.0f) ? lo : ((hi < 0.0f) ? -hi : 0.0f);
        farc[a] = fmaxf(fabsf(lo), fabsf(hi));
    }
    const float near2 = dot3_rn(nearc[0], nearc[1], nearc[2], nearc[0], nearc[1], nearc[2]);
    const float far2 = dot3_rn(farc[0], farc[1], farc[2], farc[0], farc[1], farc[2]);
    pass_bits = 0;
    if (!((near2 <= rout2) && (far2 >= rin2))) return false;
    if (brush.pmask) {
        // the box must meet every restricted coordinate range, and its radius range
        // [sqrt(near2), sqrt(far2)] the radius range (dot3_rn is monotone in each |coordinate|)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!((brush.pmask >> a) & 1u)) continue;
            float lo, hi;
            brick_box_axis(c[a], nb, sc, bs, lo, hi);
            if (!(hi >= brush.plo[a] && lo <= brush.phi[a])) return false;
        }
        if (((brush.pmask >> 3) & 1u) && !(__fsqrt_rn(far2) >= brush.plo[3] && __fsqrt_rn(near2) <= brush.phi[3]))
            return false;
    }
    bool all = true;
    for (int v = 0; v < nvars; ++v) {
        if (!((brush.mask >> v) & 1u)) continue;
        const float mn = bmin[b * nvars + v], mx = bmax[b * nvars + v];
        const float m = fmaxf(fabsf(mn), fabsf(mx));
        const float d = __fmaf_rn(m, 0x1p-20f, 0x1p-120f);
        const bool ok = m > 0x1p126f || ((__fadd_rn(mx, d) >= brush.lo[v]) && (__fsub_rn(mn, d) <= brush.hi[v]));
        if (ok) pass_bits |= 1u << v;
        all = all && ok;
    }
    return all;
}

// Skippable = brick b and its existing 26 neighbours are inactive.
__device__ __forceinline__ bool skippable_brick(size_t b, int nb, const uint32_t* active) {
    const int x = (int)(b % nb), y = (int)((b / nb) % nb), z = (int)(b / ((size_t)nb * nb));
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = x + dx, yy = y + dy, zz = z + dz;
                if (xx < 0 || yy < 0 || zz < 0 || xx >= nb || yy >= nb || zz >= nb) continue;
                const size_t id = ((size_t)zz * nb + yy) * nb + xx;
                if ((active[id >> 5] >> (id & 31)) & 1u) return false;
            }
    return true;
}

// Classification of all built levels of a volume in one launch per kernel.
// Entries 0..nbrick-1 are the 8^3 bricks of the levels (active, skippable,
// compacted list, selectivity counts); the entries after them are sub-brick
// grids (bs = kSub: active bits only; the other outputs are null).
struct ClassifyLevel {
    const float* bmin;
    const float* bmax;
    int n;                        // level edge
    int bs;                       // brick edge (kBrick or kSub)
    float sc;                     // 2 / n, set by the launcher
    size_t first;                 // first flat index of this entry (multiple of 32), set by the launcher
    uint32_t* active;
    uint32_t* skippable;
    uint32_t* list;
    uint32_t* n_active;
    unsigned* pass_count;
    uint32_t* alist;              // optional: active ids in no particular order ...
    uint32_t* acount;             // ... and their number (zeroed by the launcher)
};

struct ClassifyArgs {
    int nlev;                     // entries in lv
    int nbrick;                   // leading entries with bs = kBrick
    int nvars;
    float rin2, rout2;            // r_in * r_in, r_out * r_out rounded to FP32
    BrushArgs brush;
    size_t total;                 // set by the launcher: flat range of all entries
    size_t total_brick;           // set by the launcher: flat range of the kBrick entries
    ClassifyLevel lv[6];
};

// Cell classes under a brush: for the interpolation cell with lower corner
// (x, y, z) and each restricted variable v, over its 8 corner values: FAIL if
// a corner is NaN or, with m = max(|min|, |max|) <= 2^126 and the brick
// margin d, max + d < lo_v or min - d > hi_v (every sample value fails);
// INSIDE if m <= 2^126, min - d >= lo_v and max + d <= hi_v (every value
// passes); else the value must be interpolated. Word per cell: bit v = v must
// be interpolated, kCellFail = some restricted variable fails; [z][y][x] over
// n^3 (entries with an index of n-1 are not written).
constexpr unsigned kCellFail = 0x8000u;
struct CellClassArgs {
    const void* pairs;            // x-pair layout of the level (see Pair)
    int n;
    int nvars;
    BrushArgs brush;
    const uint32_t* slist;        // active sub-brick ids under this brush (any order) ...
    const uint32_t* scount;       // ... and their number (device)
    uint16_t* out;                // written for the cells of the listed sub-bricks only
};

// NaN-propagating max (a NaN operand gives NaN).
__device__ __forceinline__ float max_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// Restricted variables of a brush in increasing order: ids packed 4 bits
// each, bounds in the same order.
struct CellVars {
    int nr;
    unsigned ids;
    float lo[kMaxVars], hi[kMaxVars];
};

__host__ __device__ inline void cell_vars_of(const BrushArgs& b, int nvars, CellVars& R) {
    R.nr = 0;
    R.ids = 0;
    for (int v = 0; v < nvars && v < kMaxVars; ++v)
        if ((b.mask >> v) & 1u) {
            R.ids |= (unsigned)v << (4 * R.nr);
            R.lo[R.nr] = b.lo[v];
            R.hi[R.nr] = b.hi[v];
            ++R.nr;
        }
}

constexpr int kCellWarps = 4;                           // warps per block of the cell-class kernels

// Cell class words of the 4 x 4 x 4 cells of sub-brick `id` (see
// CellClassArgs), computed by one warp: lane (lx, ly, lz) takes the cells
// (4sx + lx, 4sy + ly, 4sz + 2lz + {0, 1}). Per restricted variable a lane
// loads its 2 x 3 corner x-pairs (the render's layout: one load gives both
// x-corners) at once; the corner max propagates NaN, so a NaN corner shows as
// a NaN cell max. Cells with an index of n-1 do not exist and are not written.
template <int DT>
__device__ __forceinline__ void cell_classes_of_subbrick(const void* __restrict__ pairs, int n, int nsb, uint32_t id,
                                                         int lane, const CellVars& R, uint16_t* __restrict__ out) {
    const int lx = lane & 3, ly = (lane >> 2) & 3, lz = lane >> 4;
    const size_t nn = (size_t)n * n;
    const int sx = (int)(id % nsb), sy = (int)((id / nsb) % nsb), sz = (int)(id / ((uint32_t)nsb * nsb));
    const int x = sx * kSub + lx, y = sy * kSub + ly, z = sz * kSub + 2 * lz;
    const int y0 = min(y, n - 1), y1 = min(y + 1, n - 1), x0 = min(x, n - 1);   // pair x0 = (c[x0], c[min(x0+1, n-1)])
    const int zc[3] = {min(z, n - 1), min(z + 1, n - 1), min(z + 2, n - 1)};
    unsigned word[2] = {0u, 0u};
#pragma unroll
    for (int j = 0; j < kMaxVars; ++j) {
        if (j >= R.nr) break;
        const int v = (R.ids >> (4 * j)) & 15u;
        const size_t pv = (size_t)v * nn * n;
        float mn3[3], mx3[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const size_t r0 = pv + zc[q] * nn + (size_t)y0 * n, r1 = pv + zc[q] * nn + (size_t)y1 * n;
            const float2 p0 = Pair<DT>::load(pairs, r0 + x0), p1 = Pair<DT>::load(pairs, r1 + x0);
            mn3[q] = fminf(fminf(p0.x, p0.y), fminf(p1.x, p1.y));
            mx3[q] = max_nan(max_nan(p0.x, p0.y), max_nan(p1.x, p1.y));
        }
        const float lo = R.lo[j], hi = R.hi[j];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float mn = fminf(mn3[c], mn3[c + 1]), mx = max_nan(mx3[c], mx3[c + 1]);
            unsigned w;
            if (mx != mx) {
                w = kCellFail;                                         // a NaN corner
            } else {
                const float m = fmaxf(fabsf(mn), fabsf(mx));
                const float d = __fmaf_rn(m, 0x1p-20f, 0x1p-120f);
                const float up = __fadd_rn(mx, d), dn = __fsub_rn(mn, d);
                if (m > 0x1p126f) w = 1u << v;
                else if (up < lo || dn > hi) w = kCellFail;
                else if (dn >= lo && up <= hi) w = 0u;
                else w = 1u << v;
            }
            word[c] |= w;
        }
    }
    if (x < n - 1 && y < n - 1) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (z + c < n - 1) out[((size_t)(z + c) * n + y) * n + x] = (uint16_t)word[c];
    }
}

// Process-wide count of launched kernels (defined in api.cu).
void count_launches(int k);

// Launchers (defined in the .cu files; all enqueue on `stream`).
// Ingest (level 0) and LOD (coarser level) also write the level's brick and
// sub-brick min/max (n <= kMaxRowsEdge).
constexpr int kMaxRowsEdge = 4096;
cudaError_t launch_ingest(const void* src, int src_dtype, void* cells, void* pairs, int dtype,
                          int n, int nvars, float* bmin, float* bmax, float* sbmin, float* sbmax,
                          cudaStream_t stream);
cudaError_t launch_lod(const void* fine, int n_fine, void* cells, void* pairs, int dtype, int nvars,
                       float* bmin, float* bmax, float* sbmin, float* sbmax, cudaStream_t stream);
// Ingest that also writes the next level's cells and x-pairs (edge n / 2, the same
// 2x2x2 means as launch_lod, from the values it stores) in the same pass over the
// source; that level's brick min/max then come from launch_level_bricks. Only when
// ingest_next_level_fits(src, n): n a multiple of 16 from 128 up, a 16-byte aligned source.
bool ingest_next_level_fits(const void* src, int n);
cudaError_t launch_ingest_next_level(const void* src, int src_dtype, void* cells, void* pairs, int dtype, int n,
                                     int nvars, float* bmin, float* bmax, float* sbmin, float* sbmax,
                                     void* next_cells, void* next_pairs, cudaStream_t stream);
// Brick and sub-brick min/max of a level from its own stored cells.
cudaError_t launch_level_bricks(const void* cells, int dtype, int n, int nvars, float* bmin, float* bmax,
                                float* sbmin, float* sbmax, cudaStream_t stream);
cudaError_t launch_classify(ClassifyArgs& c, cudaStream_t stream);
cudaError_t launch_cell_classes(const CellClassArgs& a, int dtype, cudaStream_t stream);
cudaError_t launch_render(const RenderArgs& a, int dtype, cudaStream_t stream);
// Batched render: per-view classification (bricks, sub-bricks and the cell
// classes of the active sub-bricks, into a.cls), then a persistent kernel that
// pulls (view, tile) work items from *tile_counter (zeroed by the caller).
// Grids are fixed by the caller (cls_blocks for the grid-stride classification,
// blocks for the persistent render) so the launch can be captured in a graph;
// launches are not counted here (the caller counts each replay).
cudaError_t launch_render_batch(const BatchHeader* hdr, const BatchView* views, unsigned* tile_counter, bool depth,
                                int dtype, int variant, unsigned cls_blocks, int blocks, cudaStream_t stream);
int render_batch_blocks_per_sm(int dtype, int variant, bool depth);
cudaError_t launch_histogram(const HistArgs& a, int dtype, cudaStream_t stream);

// Image warping (render_kernels.cu).
struct WarpArgs {
    float from_eye[3], from_target[3], from_up[3], from_tan_half;
    float to_eye[3], to_target[3], to_up[3], to_tan_half;
    int w, h;                     // both images (w * h < 2^32 pixels)
    const float4* src_rgba;       // [h][w]
    const float* src_depth;       // [h][w], +inf: no depth
    float bg[4];
    unsigned long long* keys;     // [h][w] scratch
    float4* out;                  // [h][w]
    int* out_src;                 // optional [h][w]: chosen source pixel or -1
    int fill_holes;               // unreached pixels take their nearest-z reached neighbour
};
cudaError_t launch_warp(const WarpArgs& a, cudaStream_t stream);

// TF-aware skipping (volume_kernels.cu): activity bits of the 8^3 bricks and
// 4^3 sub-bricks of a level ANDed with their TF visibility.
struct TfVisArgs {
    int n, nb, nsb, nvars, color_var;
    const float* bmin;            // [nb^3][nvars]
    const float* bmax;
    const float* sbmin;           // [nsb^3][nvars]
    const float* sbmax;
    const uint32_t* active;       // brush activity bits
    const uint32_t* sactive;
    const float4* tf;             // 256 entries (r, g, b, sigma)
    float tf_lo, tf_scale;
    uint32_t* out_active;         // nwords / nswords
    uint32_t* out_sactive;
};
cudaError_t launch_tf_visibility(const TfVisArgs& a, cudaStream_t stream);

// Empty-space distance of the nsb^3 sub-bricks under the activity bits sactive:
// Chebyshev distance in sub-bricks to the nearest active sub-brick, capped at
// kDistCap, 0 for active ones (volume_kernels.cu). tmp: nsb^3 bytes of scratch.
cudaError_t launch_subbrick_distance(const uint32_t* sactive, int nsb, uint8_t* dist, uint8_t* tmp,
                                     cudaStream_t stream);
// The same for every view of a batch that renders with skipping, from the view's
// own activity bits into its a.lv.sdist (with its stmp as scratch), after the
// per-view classification; `blocks` of 256 threads walk the views' ranges.
cudaError_t launch_subbrick_distance_views(const BatchHeader* hdr, const BatchView* views, unsigned blocks,
                                           cudaStream_t stream);

// PC line subsample (pcsub_kernels.cu).
constexpr int kSubMaxSegments = 8192;   // warp-owned row segments of the ordered compaction
struct SubsampleArgs {
    const void* cells;            // planar level values, storage dtype
    int n, nvars;
    int s_in, s_out;              // integer shell test on (2x+1-n)^2 + ..., clamped to int
    unsigned long long key;       // generator stream: seed * 2^32 + 2^32 - 1
    BrushArgs brush;              // for the per-cell brush flag (mask 0 / pmask 0: no restriction)
    int naxes;
    int axis[kMaxVars];           // stored variable or kPosAxisBase + position axis
    int use_pos;                  // position brush or a position axis in use
    unsigned long long m;         // cells to write, min(k, in-shell cells) < 2^31
    long long* out_cells;         // m
    float* out_values;            // m x naxes
    uint8_t* out_flags;           // m
};
size_t pc_subsample_scratch_bytes();

// Brush test of given points (points_kernels.cu).
struct PointFilterArgs {
    const void* pairs;            // render layout of the level, storage dtype
    int n, nvars;
    BrushArgs brush;              // variable brush and coordinate brushes (pmask bits 0..2)
    float keep_lo2, keep_hi2;     // |p|^2 range of the shell and the radius brush
    const float* pts;             // npts x 3 (x, y, z), device
    long long npts;
    uint8_t* out;                 // npts flags, device
};
cudaError_t launch_filter_points(const PointFilterArgs& a, int dtype, cudaStream_t stream);
cudaError_t launch_pc_subsample(const SubsampleArgs& a, int dtype, unsigned long long m, unsigned long long N,
                                void* scratch, cudaStream_t stream);

}  // namespace raypc

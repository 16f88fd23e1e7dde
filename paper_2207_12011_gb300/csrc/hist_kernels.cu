// Adjacent-axis parallel-coordinates density histograms (Section 2.1 PC data,
// Fig. 2): for every in-shell (and, optionally, in-brush) cell and every pair
// of adjacent axes (a, a+1), H[a][bin_a][bin_{a+1}] += 1.
//
// HBM-bound scan. A warp walks one x-row of cells so the planar loads are
// coalesced; rows whose cells all lie outside the shell are skipped without
// touching memory. The vector kernel gives each lane a 16-byte chunk of a
// row per variable (8 FP16 or 4 FP32 cells); the scalar kernel (ragged grid
// edges, unaligned fields) one cell per lane. A cell's axis values that are
// not brushed are loaded only after its brushed values pass. Position axes and
// the position brush use the cell centre, coordinate RN((2i + 1 - n) / n).
// With the volume's own brush the cells of inactive 4^3 sub-bricks are skipped
// without loads: every vertex of such a sub-brick fails the brush (its values
// lie between the sub-brick's min and max) or lies outside the shell (the
// sub-brick's widened box, which holds the vertex centres, misses the shell).
// The in-shell test is integer-exact. Bins come from a walk over the FP32 edges
// held in shared memory (comparisons only, so exact). Increments are
// aggregated per warp with __match_any_sync on the (bin_a, bin_{a+1}) key: one
// atomicAdd per distinct key per warp and pair.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "host_math.h"

namespace raypc {

namespace {

constexpr int kHistThreads = 256;
constexpr int kHistWarps = kHistThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// Number of interior edges e_1..e_{bins-1} that are <= v, for non-decreasing
// edges: j from an affine guess is the answer iff (j == 0 or v >= e_j) and
// (j == bins-1 or v < e_{j+1}) -- both edges are loaded at once; otherwise the
// guess is walked to the answer with comparisons only (exact for any edges;
// equally spaced edges rarely need a step). NaN compares false everywhere and
// lands in bin 0.
__device__ __forceinline__ int bin_of(const float* e, int bins, float v, float e0, float scale) {
    if (v != v) return 0;
    float g = (v - e0) * scale;
    g = fminf(fmaxf(g, 0.0f), (float)(bins - 1));
    int j = (int)g;
    const float lo = e[j], hi = e[j + 1];
    if ((j == 0 || v >= lo) && (j == bins - 1 || v < hi)) return j;
    while (j > 0 && !(v >= e[j])) --j;
    while (j < bins - 1 && v >= e[j + 1]) ++j;
    return j;
}

// Adds one count per kept lane to hist[key] (all 32 lanes call it, in x order of
// their cells; km = ballot of kept): a lane whose key differs from its left neighbour's, or whose left
// neighbour is not kept, starts a run and adds the run's length once. Neighbouring
// cells of a smooth field mostly share their bin pair, so few atomics remain.
__device__ __forceinline__ void add_runs(uint32_t* hist, unsigned key, bool kept, unsigned km, int lane) {
    const unsigned left = __shfl_up_sync(kFull, key, 1);
    const bool head = kept && (lane == 0 || !((km >> (lane - 1)) & 1u) || left != key);
    const unsigned hm = __ballot_sync(kFull, head);
    if (head) {
        const unsigned after = lane == 31 ? 0u : (kFull << (lane + 1));
        const unsigned stop = (hm | ~km) & after;            // next run start or next lane not kept
        const int end = stop ? __ffs(stop) - 1 : 32;
        atomicAdd(hist + key, (unsigned)(end - lane));
    }
}

// Largest integer m >= 0 with m * m <= a (0 <= a < 2^31).
__device__ __forceinline__ int isqrt_floor(int a) {
    int m = (int)sqrtf((float)a);
    while ((long long)m * m > a) --m;
    while ((long long)(m + 1) * (m + 1) <= a) ++m;
    return m;
}

// Kernel view of a histogram call: the brushed variables and the axes as
// compact lists (the host builds it from HistArgs). Edge tables of up to
// kInlineEdges floats travel in the launch parameters (no device copy);
// larger ones are read from `edges`.
constexpr int kInlineEdges = kHistInlineEdges;
struct HistLaunch {
    const void* cells;
    int n, bins;
    int nbr;                       // brushed variables tested per cell
    int bvar[kMaxVars];
    float blo[kMaxVars], bhi[kMaxVars];
    int naxes;
    int avar[kMaxVars];            // variable of each axis, or kPosAxisBase + position axis
    float plo[kNumPos], phi[kNumPos];
    uint32_t pmask;                // position brush at the cell centre (0: none)
    int use_pos;                   // the position brush or a position axis is in use
    // load slots of the vector kernel: slot a < naxes is axis a (loaded when it names a
    // stored variable), slots naxes..nslot-1 hold brushed variables that are no axis
    int nslot;
    int svar[kMaxVars];            // variable of each slot (-1: position axis, nothing to load)
    uint32_t sbr;                  // bit s: slot s is tested against the brush
    float slo[kMaxVars], shi[kMaxVars];
    uint32_t slo_h2[kMaxVars], shi_h2[kMaxVars];   // FP16 fields: the same bounds as binary16 pairs
    float guess_e0[kMaxVars], guess_scale[kMaxVars];
    int s_in, s_out;               // shell test on 2x+1-n etc., clamped to int
    uint32_t* out;
    const uint32_t* sactive;       // optional sub-brick activity (see HistArgs)
    int nsb;
    const float* edges;            // naxes x (bins + 1) on the device, or null: edges_inl
    float edges_inl[kInlineEdges];
};

// Copy the edge table into shared memory (all threads; the caller syncs).
__device__ __forceinline__ void stage_edges(const HistLaunch& A, float* s_edges) {
    const int ne = A.naxes * (A.bins + 1);
    if (A.edges)
        for (int i = threadIdx.x; i < ne; i += blockDim.x) s_edges[i] = __ldg(A.edges + i);
    else
        for (int i = threadIdx.x; i < ne; i += blockDim.x) s_edges[i] = A.edges_inl[i];
}

// Row geometry shared by both kernels: the x range of row r (y, z) inside the
// outer sphere, |2x + 1 - n| <= m; false when the whole row lies outside.
struct RowSpan {
    int y, z, syz, xa, xb;
    float cy, cz;
    size_t base;                   // r * n
    uint32_t srow;                 // first sub-brick id of the row's sub-brick row
};

__device__ __forceinline__ bool row_span(const HistLaunch& A, int r, RowSpan& R) {
    const int n = A.n;
    R.y = r % n;
    R.z = r / n;
    const int dy = 2 * R.y + 1 - n, dz = 2 * R.z + 1 - n;
    R.syz = dy * dy + dz * dz;                              // < 2^31 for n <= 4096
    if (R.syz > A.s_out) return false;
    const int m = isqrt_floor(A.s_out - R.syz);
    R.xa = max(0, (n - m) / 2);
    R.xb = min(n - 1, (n - 1 + m) / 2);
    R.cy = A.use_pos ? cell_centre_rn(R.y, n) : 0.0f;
    R.cz = A.use_pos ? cell_centre_rn(R.z, n) : 0.0f;
    R.base = (size_t)r * n;
    R.srow = ((uint32_t)(R.z >> 2) * A.nsb + (uint32_t)(R.y >> 2)) * A.nsb;
    return true;
}

// Whether cell x of row R is counted before any brushed value is read: in the
// shell (integers), in an active sub-brick when the activity is given (a vertex
// of an inactive sub-brick fails the brush or lies outside the shell), and
// inside the position brush at the cell centre.
__device__ __forceinline__ bool cell_geometry_passes(const HistLaunch& A, const RowSpan& R, int x) {
    const int dx = 2 * x + 1 - A.n;
    const int sh = dx * dx + R.syz;
    if (!(sh >= A.s_in && sh <= A.s_out)) return false;
    if (A.sactive) {
        const uint32_t sid = R.srow + (uint32_t)(x >> 2);
        if (!((__ldg(A.sactive + (sid >> 5)) >> (sid & 31)) & 1u)) return false;
    }
    if (A.pmask) {
        BrushArgs pb;
#pragma unroll
        for (int a = 0; a < kNumPos; ++a) { pb.plo[a] = A.plo[a]; pb.phi[a] = A.phi[a]; }
        pb.pmask = A.pmask;
        const float cx = cell_centre_rn(x, A.n);
        if (!pos_pass(cx, R.cy, R.cz, dot3_rn(cx, R.cy, R.cz, cx, R.cy, R.cz), pb)) return false;
    }
    return true;
}

// Scalar kernel: any grid edge, any alignment, any number of axes. A warp walks
// one x-row of cells (lanes over x, two cells per lane in flight); persistent
// grid, rows by warp stride.
template <int DT>
__global__ void __launch_bounds__(kHistThreads) k_hist_scalar(const __grid_constant__ HistLaunch A) {
    extern __shared__ float s_edges[];
    stage_edges(A, s_edges);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int n = A.n;
    const int rows = n * n;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int bins = A.bins;
    const size_t plane = (size_t)n * n * n;

    for (int r = gwarp; r < rows; r += nwarps) {
        RowSpan R;
        if (!row_span(A, r, R)) continue;
        for (int x0 = R.xa; x0 <= R.xb; x0 += 64) {
            bool keep[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int x = x0 + lane + 32 * j;
                keep[j] = x <= R.xb && cell_geometry_passes(A, R, x);
            }
            // brushed variables first, all loads in flight together
            float bv[2][kMaxVars];
#pragma unroll
            for (int k = 0; k < kMaxVars; ++k) {
                if (k >= A.nbr) break;
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    bv[j][k] = keep[j] ? load_cell<DT>(A.cells, A.bvar[k] * plane + R.base + x0 + lane + 32 * j) : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < kMaxVars; ++k) {
                if (k >= A.nbr) break;
#pragma unroll
                for (int j = 0; j < 2; ++j) keep[j] = keep[j] && bv[j][k] >= A.blo[k] && bv[j][k] <= A.bhi[k];
            }
            if (__ballot_sync(kFull, keep[0] || keep[1]) == 0u) continue;
            // axis values of the cells that pass (brushed ones come back from L1), binned and
            // added in x order
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const unsigned km = __ballot_sync(kFull, keep[j]);
                if (km == 0u) continue;
                const int x = x0 + lane + 32 * j;
                float cx = 0.0f, cr2 = 0.0f;
                if (A.use_pos && keep[j]) {
                    cx = cell_centre_rn(x, n);
                    cr2 = dot3_rn(cx, R.cy, R.cz, cx, R.cy, R.cz);
                }
                unsigned prev = 0u;
#pragma unroll
                for (int a = 0; a < kMaxVars; ++a) {
                    if (a >= A.naxes) break;
                    const int av = A.avar[a];
                    unsigned b = 0u;
                    if (keep[j]) {
                        const float v = av >= kPosAxisBase ? pos_axis(cx, R.cy, R.cz, cr2, av - kPosAxisBase)
                                                           : load_cell<DT>(A.cells, av * plane + R.base + x);
                        b = (unsigned)bin_of(s_edges + a * (bins + 1), bins, v, A.guess_e0[a], A.guess_scale[a]);
                    }
                    if (a > 0) add_runs(A.out + (size_t)(a - 1) * bins * bins, prev * (unsigned)bins + b, keep[j], km, lane);
                    prev = b;
                }
            }
        }
    }
}

__device__ __forceinline__ __half2 u32_as_half2(unsigned u) {
    __half2 h;
    memcpy(&h, &u, sizeof(h));
    return h;
}

// Element j of a 16-byte chunk of FP32 values.
template <int DT> __device__ __forceinline__ float chunk_elem(const uint4& c, int j);
template <> __device__ __forceinline__ float chunk_elem<kF32>(const uint4& c, int j) {
    return __uint_as_float(j == 0 ? c.x : j == 1 ? c.y : j == 2 ? c.z : c.w);
}

// Per-warp shared staging of the vector kernel: the axis values of one chunk row
// (32 lanes x 16 bytes per axis) and the list of its surviving cells (up to 256).
constexpr int kStageBytes = kMaxVars * 512 + 256;

// Vector kernel (grid edge a multiple of the chunk, 16-byte aligned planes, at most
// kMaxVars load slots). A warp walks one x-row; each lane takes a chunk of VEC
// consecutive cells (16 bytes per variable: 8 FP16 or 4 FP32 values), so one
// load instruction brings 512 bytes per warp. The chunk's cells are tested
// against the shell (integers), the sub-brick activity and the position brush;
// then all brushed slots of a chunk with a surviving cell are loaded together
// and tested, then the axis slots that are not brushed. The axis values go to
// the warp's shared staging and the surviving cells into a compact list in x
// order (warp prefix sum), from which the warp bins 32 surviving cells per
// round: a selective brush needs one round per chunk row instead of one per
// chunk position, and neighbouring lanes hold neighbouring cells for the
// run-length adds. Persistent grid, rows by warp stride; the edge table is
// staged once per resident block.
template <int DT>
__global__ void __launch_bounds__(kHistThreads, 4) k_hist(const __grid_constant__ HistLaunch A) {
    constexpr int VEC = DT == kF16 ? 8 : 4;
    constexpr int CH = 32 * VEC;                           // cells per warp and chunk row
    extern __shared__ __align__(16) unsigned char s_raw[];
    float* s_edges = reinterpret_cast<float*>(s_raw);
    const int ne16 = (A.naxes * (A.bins + 1) + 3) & ~3;
    unsigned char* s_stage = s_raw + sizeof(float) * ne16 + (size_t)(threadIdx.x >> 5) * kStageBytes;
    unsigned char* s_list = s_stage + kMaxVars * 512;
    stage_edges(A, s_edges);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int n = A.n;
    const int rows = n * n;                                   // n <= 4096
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int bins = A.bins;
    const size_t plane = (size_t)n * n * n;
    const uint32_t sbr = A.sbr;
    const int nslot = A.nslot, naxes = A.naxes;

    for (int r = gwarp; r < rows; r += nwarps) {
        RowSpan R;
        if (!row_span(A, r, R)) continue;
        const int xa = R.xa & ~(VEC - 1);                    // first chunk holding a cell inside the outer sphere
        for (int xw = xa; xw <= R.xb; xw += CH) {
            const int x0 = xw + lane * VEC;                 // this lane's chunk; x0 + VEC <= n when x0 <= xb
            unsigned kb = 0u;                               // bit j: cell x0 + j is still counted
            if (x0 <= R.xb) {
                if (A.sactive && !A.pmask) {
                    // whole sub-bricks at once (a chunk covers VEC / 4 of them)
#pragma unroll
                    for (int q = 0; q < VEC / 4; ++q) {
                        const uint32_t sid = R.srow + (uint32_t)((x0 >> 2) + q);
                        if (!((__ldg(A.sactive + (sid >> 5)) >> (sid & 31)) & 1u)) continue;
#pragma unroll
                        for (int j = 4 * q; j < 4 * q + 4; ++j) {
                            const int dx = 2 * (x0 + j) + 1 - n;
                            const int sh = dx * dx + R.syz;
                            if (sh >= A.s_in && sh <= A.s_out) kb |= 1u << j;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < VEC; ++j)
                        if (cell_geometry_passes(A, R, x0 + j)) kb |= 1u << j;
                }
            }
            // brushed slots: all loads of the chunk in flight together
            uint4 val[kMaxVars];
#pragma unroll
            for (int s = 0; s < kMaxVars; ++s) {
                val[s] = make_uint4(0u, 0u, 0u, 0u);
                if (s < nslot && ((sbr >> s) & 1u) && kb)
                    val[s] = __ldg(reinterpret_cast<const uint4*>(
                        static_cast<const char*>(A.cells) + ((size_t)A.svar[s] * plane + R.base + x0) * (16 / VEC)));
            }
            if constexpr (DT == kF16) {
                // two cells per comparison against the exact binary16 bounds (h >= lo iff
                // h >= lo_h, h <= hi iff h <= hi_h; NaN fails both)
                unsigned acc[4] = {kFull, kFull, kFull, kFull};
#pragma unroll
                for (int s = 0; s < kMaxVars; ++s) {
                    if (s < nslot && ((sbr >> s) & 1u)) {
                        const __half2 lo2 = u32_as_half2(A.slo_h2[s]), hi2 = u32_as_half2(A.shi_h2[s]);
                        const unsigned w[4] = {val[s].x, val[s].y, val[s].z, val[s].w};
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            acc[q] &= __hge2_mask(u32_as_half2(w[q]), lo2) & __hle2_mask(u32_as_half2(w[q]), hi2);
                    }
                }
                unsigned pass = 0u;
#pragma unroll
                for (int q = 0; q < 4; ++q) pass |= ((acc[q] & 1u) | ((acc[q] >> 15) & 2u)) << (2 * q);
                kb &= pass;
            } else {
#pragma unroll
                for (int s = 0; s < kMaxVars; ++s) {
                    if (s < nslot && ((sbr >> s) & 1u)) {
                        const float lo = A.slo[s], hi = A.shi[s];
#pragma unroll
                        for (int j = 0; j < VEC; ++j) {
                            const float v = chunk_elem<DT>(val[s], j);
                            if (!(v >= lo && v <= hi)) kb &= ~(1u << j);
                        }
                    }
                }
            }
            if (__ballot_sync(kFull, kb != 0u) == 0u) continue;
            // axis slots that are not brushed, for chunks with a surviving cell; then every
            // stored axis slot and the keep bits to the warp's staging
#pragma unroll
            for (int s = 0; s < kMaxVars; ++s) {
                if (s < naxes && A.svar[s] >= 0) {
                    if (!((sbr >> s) & 1u) && kb)
                        val[s] = __ldg(reinterpret_cast<const uint4*>(
                            static_cast<const char*>(A.cells) + ((size_t)A.svar[s] * plane + R.base + x0) * (16 / VEC)));
                    *reinterpret_cast<uint4*>(s_stage + s * 512 + lane * 16) = val[s];
                }
            }
            // compact list of the surviving cells (chunk-row offsets) in x order
            const unsigned cnt = (unsigned)__popc(kb);
            unsigned incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = (int)__shfl_sync(kFull, incl, 31);
            int pos = (int)(incl - cnt);
#pragma unroll
            for (int j = 0; j < VEC; ++j)
                if ((kb >> j) & 1u) s_list[pos++] = (unsigned char)(lane * VEC + j);
            __syncwarp();
            // bin 32 surviving cells per round
#pragma unroll 1
            for (int base = 0; base < total; base += 32) {
                const bool kept = base + lane < total;
                const unsigned km = total - base >= 32 ? kFull : (1u << (total - base)) - 1u;
                const int c = kept ? s_list[base + lane] : 0;       // cell xw + c
                float cx = 0.0f, cr2 = 0.0f;
                if (A.use_pos && kept) {
                    cx = cell_centre_rn(xw + c, n);
                    cr2 = dot3_rn(cx, R.cy, R.cz, cx, R.cy, R.cz);
                }
                unsigned prev = 0u;
#pragma unroll
                for (int a = 0; a < kMaxVars; ++a) {
                    if (a >= naxes) break;
                    const int av = A.avar[a];
                    unsigned b = 0u;
                    if (kept) {
                        float v;
                        if (av >= kPosAxisBase) {
                            v = pos_axis(cx, R.cy, R.cz, cr2, av - kPosAxisBase);
                        } else if (DT == kF16) {
                            v = __half2float(__ushort_as_half(reinterpret_cast<const unsigned short*>(s_stage + a * 512)[c]));
                        } else {
                            v = reinterpret_cast<const float*>(s_stage + a * 512)[c];
                        }
                        b = (unsigned)bin_of(s_edges + a * (bins + 1), bins, v, A.guess_e0[a], A.guess_scale[a]);
                    }
                    if (a > 0) add_runs(A.out + (size_t)(a - 1) * bins * bins, prev * (unsigned)bins + b, kept, km, lane);
                    prev = b;
                }
            }
            __syncwarp();                                       // staging is rewritten by the next chunk row
        }
    }
}

template <int DT>
cudaError_t launch_t(const HistArgs& h, cudaStream_t stream) {
    HistLaunch a{};                      // about 8.6 KB with the inline edges (host stack)
    a.cells = h.cells;
    a.n = h.n;
    a.bins = h.bins;
    if (h.use_brush)
        for (int v = 0; v < h.nvars && v < kMaxVars; ++v)
            if ((h.brush.mask >> v) & 1u) {
                a.bvar[a.nbr] = v;
                a.blo[a.nbr] = h.brush.lo[v];
                a.bhi[a.nbr] = h.brush.hi[v];
                ++a.nbr;
            }
    if (h.use_brush && h.brush.pmask) {
        for (int i = 0; i < kNumPos; ++i) { a.plo[i] = h.brush.plo[i]; a.phi[i] = h.brush.phi[i]; }
        a.pmask = h.brush.pmask;
        a.use_pos = 1;
    }
    a.naxes = h.naxes;
    for (int i = 0; i < h.naxes && i < kMaxVars; ++i) {
        a.avar[i] = h.axis[i];
        if (h.axis[i] >= kPosAxisBase) a.use_pos = 1;
        a.guess_e0[i] = h.guess_e0[i];
        a.guess_scale[i] = h.guess_scale[i];
    }
    // load slots of the vector kernel: the axes, then the brushed variables that are no axis
    bool vec_slots = true;
    a.nslot = h.naxes;
    for (int i = 0; i < h.naxes && i < kMaxVars; ++i) {
        a.svar[i] = h.axis[i] >= kPosAxisBase ? -1 : h.axis[i];
        a.slo[i] = -INFINITY;
        a.shi[i] = INFINITY;
    }
    for (int k = 0; k < a.nbr; ++k) {
        int s = -1;
        for (int i = 0; i < h.naxes; ++i)
            if (a.svar[i] == a.bvar[k]) { s = i; break; }
        if (s < 0) {
            if (a.nslot >= kMaxVars) { vec_slots = false; break; }
            s = a.nslot++;
            a.svar[s] = a.bvar[k];
        }
        a.sbr |= 1u << s;
        a.slo[s] = a.blo[k];
        a.shi[s] = a.bhi[k];
    }
    if (DT == kF16)
        for (int s = 0; s < a.nslot && s < kMaxVars; ++s) {
            const uint32_t lo = half_ceil_bits(a.slo[s]), hi = half_floor_bits(a.shi[s]);
            a.slo_h2[s] = lo | (lo << 16);
            a.shi_h2[s] = hi | (hi << 16);
        }
    const int64_t imax = 0x7fffffff;
    a.s_in = (int)std::min<int64_t>(std::max<int64_t>(h.s_in, 0), imax);
    a.s_out = (int)std::min<int64_t>(h.s_out, imax);
    a.out = h.out;
    a.sactive = h.sactive;
    a.nsb = h.nsb;
    const int ne = h.naxes * (h.bins + 1);
    if (h.edges_host && ne <= kInlineEdges) {
        for (int i = 0; i < ne; ++i) a.edges_inl[i] = h.edges_host[i];
        a.edges = nullptr;
    } else if (h.edges) {
        a.edges = h.edges;
    } else {
        return cudaErrorInvalidValue;
    }
    if (h.s_out < 0) return cudaSuccess;                 // no cell in the shell: the zeroed output is the answer
    constexpr int VEC = DT == kF16 ? 8 : 4;
    const bool vec = vec_slots && h.n % VEC == 0 && (reinterpret_cast<uintptr_t>(h.cells) & 15u) == 0;
    const size_t smem = vec ? sizeof(float) * (size_t)((ne + 3) & ~3) + (size_t)kHistWarps * kStageBytes
                            : sizeof(float) * (size_t)ne;
    // persistent grid: as many blocks as fit at once (rows by warp stride)
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && vec && smem > 48 * 1024)
        e = cudaFuncSetAttribute(k_hist<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist<DT>, kHistThreads, smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist_scalar<DT>, kHistThreads, smem);
    if (e != cudaSuccess) return e;
    const long long rows = (long long)a.n * a.n;
    const long long want_blocks = (rows + kHistWarps - 1) / kHistWarps;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(want_blocks, (long long)sms * std::max(1, per_sm)));
    if (vec) k_hist<DT><<<blocks, kHistThreads, smem, stream>>>(a);
    else k_hist_scalar<DT><<<blocks, kHistThreads, smem, stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_histogram(const HistArgs& a, int dtype, cudaStream_t stream) {
    if (dtype == kF16) return launch_t<kF16>(a, stream);
    return launch_t<kF32>(a, stream);
}

}  // namespace raypc

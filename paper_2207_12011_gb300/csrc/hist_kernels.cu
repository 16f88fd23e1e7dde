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

namespace raypc {

namespace {

constexpr int kHistThreads = 256;

// Number of interior edges e_1..e_{bins-1} that are <= v, for non-decreasing
// edges: start from an affine guess and walk to the answer with comparisons
// only (exact for any edges; one or two steps for equally spaced ones). NaN
// compares false everywhere and lands in bin 0.
__device__ __forceinline__ int bin_of(const float* e, int bins, float v, float e0, float scale) {
    if (v != v) return 0;
    float g = (v - e0) * scale;
    g = fminf(fmaxf(g, 0.0f), (float)(bins - 1));
    int j = (int)g;
    while (j > 0 && !(v >= e[j])) --j;
    while (j < bins - 1 && v >= e[j + 1]) ++j;
    return j;
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

// Scalar kernel: any grid edge, any alignment, any number of axes. A warp walks
// one x-row of cells (lanes over x, two cells per lane in flight).
template <int DT>
__global__ void __launch_bounds__(kHistThreads) k_hist_scalar(const __grid_constant__ HistLaunch A) {
    extern __shared__ float s_edges[];
    stage_edges(A, s_edges);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int n = A.n;
    const long long rows = (long long)n * n;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int bins = A.bins;
    const size_t plane = (size_t)n * n * n;

    for (long long r = gwarp; r < rows; r += nwarps) {
        const int y = (int)(r % n), z = (int)(r / n);
        const int dy = 2 * y + 1 - n, dz = 2 * z + 1 - n;
        const float cy = A.use_pos ? cell_centre_rn(y, n) : 0.0f, cz = A.use_pos ? cell_centre_rn(z, n) : 0.0f;
        const int syz = dy * dy + dz * dz;                  // < 2^31 for n <= 4096
        if (syz > A.s_out) continue;                        // whole row outside the outer sphere
        // x range of the row inside the outer sphere: |2x + 1 - n| <= m
        const int m = isqrt_floor(A.s_out - syz);
        const int xa = max(0, (n - m) / 2);
        const int xb = min(n - 1, (n - 1 + m) / 2);
        const size_t row_base = (size_t)r * n;
        const uint32_t srow = ((uint32_t)(z >> 2) * A.nsb + (uint32_t)(y >> 2)) * A.nsb;
        // two cells per lane and iteration: their loads are in flight together
        for (int x0 = xa; x0 <= xb; x0 += 64) {
            bool keep[2];
            float cx[2], cr2[2];           // centre x and squared radius (position axes)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int x = x0 + lane + 32 * j;
                keep[j] = false;
                cx[j] = cr2[j] = 0.0f;
                if (x <= xb) {
                    const int dx = 2 * x + 1 - n;
                    const int s = dx * dx + syz;
                    keep[j] = s >= A.s_in && s <= A.s_out;
                    if (keep[j] && A.sactive) {
                        // a vertex of an inactive sub-brick fails the brush or lies outside the shell
                        const uint32_t sid = srow + (uint32_t)(x >> 2);
                        keep[j] = (__ldg(A.sactive + (sid >> 5)) >> (sid & 31)) & 1u;
                    }
                    if (keep[j] && A.use_pos) {
                        cx[j] = cell_centre_rn(x, n);
                        cr2[j] = dot3_rn(cx[j], cy, cz, cx[j], cy, cz);
                        if (A.pmask) {
                            BrushArgs pb;
#pragma unroll
                            for (int a = 0; a < kNumPos; ++a) { pb.plo[a] = A.plo[a]; pb.phi[a] = A.phi[a]; }
                            pb.pmask = A.pmask;
                            keep[j] = pos_pass(cx[j], cy, cz, cr2[j], pb);
                        }
                    }
                }
            }
            // brushed variables first
            float bv[2][kMaxVars];
#pragma unroll
            for (int k = 0; k < kMaxVars; ++k) {
                if (k >= A.nbr) break;
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    bv[j][k] = keep[j] ? load_cell<DT>(A.cells, A.bvar[k] * plane + row_base + x0 + lane + 32 * j) : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < kMaxVars; ++k) {
                if (k >= A.nbr) break;
#pragma unroll
                for (int j = 0; j < 2; ++j) keep[j] = keep[j] && bv[j][k] >= A.blo[k] && bv[j][k] <= A.bhi[k];
            }
            if (__ballot_sync(0xffffffffu, keep[0] || keep[1]) == 0u) continue;
            // axis values of the cells that pass (brushed ones come back from L1)
            int bn[2][kMaxVars];
#pragma unroll
            for (int a = 0; a < kMaxVars; ++a) {
                if (a >= A.naxes) break;
                float va[2];
                const int av = A.avar[a];
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    va[j] = !keep[j] ? 0.0f
                          : av >= kPosAxisBase ? pos_axis(cx[j], cy, cz, cr2[j], av - kPosAxisBase)
                                               : load_cell<DT>(A.cells, av * plane + row_base + x0 + lane + 32 * j);
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    bn[j][a] = keep[j] ? bin_of(s_edges + a * (bins + 1), bins, va[j], A.guess_e0[a], A.guess_scale[a]) : 0;
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const unsigned km = __ballot_sync(0xffffffffu, keep[j]);
                if (km == 0u) continue;
                if (keep[j]) {
#pragma unroll
                    for (int p = 0; p + 1 < kMaxVars; ++p) {
                        if (p + 1 >= A.naxes) break;
                        const unsigned key = (unsigned)bn[j][p] * (unsigned)bins + (unsigned)bn[j][p + 1];
                        const unsigned peers = __match_any_sync(km, key);
                        if (lane == __ffs(peers) - 1)
                            atomicAdd(A.out + (size_t)p * bins * bins + key, (unsigned)__popc(peers));
                    }
                }
            }
        }
    }
}

// Element j of a 16-byte chunk of stored values, as FP32 (exact).
template <int DT> __device__ __forceinline__ float chunk_elem(const uint4& c, int j);
template <> __device__ __forceinline__ float chunk_elem<kF32>(const uint4& c, int j) {
    return __uint_as_float(j == 0 ? c.x : j == 1 ? c.y : j == 2 ? c.z : c.w);
}
template <> __device__ __forceinline__ float chunk_elem<kF16>(const uint4& c, int j) {
    const unsigned w = (j >> 1) == 0 ? c.x : (j >> 1) == 1 ? c.y : (j >> 1) == 2 ? c.z : c.w;
    return __half2float(__ushort_as_half((unsigned short)(w >> (16 * (j & 1)))));
}

// Vector kernel (grid edge a multiple of the chunk, 16-byte aligned planes, at most
// kMaxVars load slots). A warp walks one x-row; each lane takes a chunk of VEC
// consecutive cells (16 bytes per variable: 8 FP16 or 4 FP32 values), so one
// load instruction brings 512 bytes per warp. The chunk's cells are tested
// against the shell (integers), the sub-brick activity and the position brush;
// then all brushed slots of a chunk with a surviving cell are loaded together
// and tested, then the axis slots that are not brushed; the surviving cells are
// binned one chunk position at a time. The grid is persistent (rows by warp
// stride), so the edge table is staged once per resident block.
template <int DT>
__global__ void __launch_bounds__(kHistThreads) k_hist(const __grid_constant__ HistLaunch A) {
    constexpr int VEC = DT == kF16 ? 8 : 4;
    extern __shared__ float s_edges[];
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
        const int y = r % n, z = r / n;
        const int dy = 2 * y + 1 - n, dz = 2 * z + 1 - n;
        const int syz = dy * dy + dz * dz;
        if (syz > A.s_out) continue;                        // whole row outside the outer sphere
        const int m = isqrt_floor(A.s_out - syz);
        const int xa = max(0, (n - m) / 2) & ~(VEC - 1);    // first chunk holding a cell inside the outer sphere
        const int xb = min(n - 1, (n - 1 + m) / 2);
        const float cy = A.use_pos ? cell_centre_rn(y, n) : 0.0f, cz = A.use_pos ? cell_centre_rn(z, n) : 0.0f;
        const size_t row_base = (size_t)r * n;
        const uint32_t srow = ((uint32_t)(z >> 2) * A.nsb + (uint32_t)(y >> 2)) * A.nsb;
        for (int xw = xa; xw <= xb; xw += 32 * VEC) {
            const int x0 = xw + lane * VEC;                 // this lane's chunk; x0 + VEC <= n when x0 <= xb
            unsigned kb = 0u;                               // bit j: cell x0 + j is still counted
            if (x0 <= xb) {
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    const int dx = 2 * (x0 + j) + 1 - n;
                    const int sh = dx * dx + syz;
                    if (sh >= A.s_in && sh <= A.s_out) kb |= 1u << j;
                }
                if (kb && A.sactive) {
                    // cells of inactive 4^3 sub-bricks are never counted
#pragma unroll
                    for (int q = 0; q < VEC / 4; ++q) {
                        const uint32_t sid = srow + (uint32_t)((x0 >> 2) + q);
                        if (!((__ldg(A.sactive + (sid >> 5)) >> (sid & 31)) & 1u)) kb &= ~(0xfu << (4 * q));
                    }
                }
                if (kb && A.pmask) {
                    BrushArgs pb;
#pragma unroll
                    for (int a = 0; a < kNumPos; ++a) { pb.plo[a] = A.plo[a]; pb.phi[a] = A.phi[a]; }
                    pb.pmask = A.pmask;
#pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        if (!((kb >> j) & 1u)) continue;
                        const float cx = cell_centre_rn(x0 + j, n);
                        if (!pos_pass(cx, cy, cz, dot3_rn(cx, cy, cz, cx, cy, cz), pb)) kb &= ~(1u << j);
                    }
                }
            }
            // brushed slots: all loads of the chunk in flight together
            uint4 val[kMaxVars];
#pragma unroll
            for (int s = 0; s < kMaxVars; ++s) {
                val[s] = make_uint4(0u, 0u, 0u, 0u);
                if (s < nslot && ((sbr >> s) & 1u) && kb)
                    val[s] = __ldg(reinterpret_cast<const uint4*>(
                        static_cast<const char*>(A.cells) + ((size_t)A.svar[s] * plane + row_base + x0) * (16 / VEC)));
            }
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
            if (__ballot_sync(0xffffffffu, kb != 0u) == 0u) continue;
            // axis slots that are not brushed, for chunks with a surviving cell
#pragma unroll
            for (int s = 0; s < kMaxVars; ++s)
                if (s < naxes && !((sbr >> s) & 1u) && A.svar[s] >= 0 && kb)
                    val[s] = __ldg(reinterpret_cast<const uint4*>(
                        static_cast<const char*>(A.cells) + ((size_t)A.svar[s] * plane + row_base + x0) * (16 / VEC)));
            // bin the surviving cells, one chunk position at a time (warp-aggregated atomics)
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                const bool kj = (kb >> j) & 1u;
                const unsigned km = __ballot_sync(0xffffffffu, kj);
                if (km == 0u) continue;
                if (kj) {
                    float cx = 0.0f, cr2 = 0.0f;
                    if (A.use_pos) {
                        cx = cell_centre_rn(x0 + j, n);
                        cr2 = dot3_rn(cx, cy, cz, cx, cy, cz);
                    }
                    unsigned prev = 0u;
#pragma unroll
                    for (int a = 0; a < kMaxVars; ++a) {
                        if (a >= naxes) break;
                        const int av = A.avar[a];
                        const float v = av >= kPosAxisBase ? pos_axis(cx, cy, cz, cr2, av - kPosAxisBase)
                                                           : chunk_elem<DT>(val[a], j);
                        const unsigned b = (unsigned)bin_of(s_edges + a * (bins + 1), bins, v, A.guess_e0[a], A.guess_scale[a]);
                        if (a > 0) {
                            const unsigned key = prev * (unsigned)bins + b;
                            const unsigned peers = __match_any_sync(km, key);
                            if (lane == __ffs(peers) - 1)
                                atomicAdd(A.out + (size_t)(a - 1) * bins * bins + key, (unsigned)__popc(peers));
                        }
                        prev = b;
                    }
                }
            }
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
    const size_t smem = sizeof(float) * ne;
    constexpr int VEC = DT == kF16 ? 8 : 4;
    const bool vec = vec_slots && h.n % VEC == 0 && (reinterpret_cast<uintptr_t>(h.cells) & 15u) == 0;
    const long long rows = (long long)a.n * a.n;
    const long long want_blocks = (rows + (kHistThreads / 32) - 1) / (kHistThreads / 32);
    int blocks;
    if (vec) {
        // persistent grid: as many blocks as fit at once (rows by warp stride)
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist<DT>, kHistThreads, smem);
        if (e != cudaSuccess) return e;
        blocks = (int)std::min<long long>(want_blocks, (long long)std::max(1, sms * std::max(1, per_sm)));
        k_hist<DT><<<blocks, kHistThreads, smem, stream>>>(a);
    } else {
        // one row per warp (rows differ in length; the hardware balances blocks)
        blocks = (int)std::max<long long>(1, std::min<long long>(want_blocks, 0x7fffffffLL));
        k_hist_scalar<DT><<<blocks, kHistThreads, smem, stream>>>(a);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_histogram(const HistArgs& a, int dtype, cudaStream_t stream) {
    if (dtype == kF16) return launch_t<kF16>(a, stream);
    return launch_t<kF32>(a, stream);
}

}  // namespace raypc

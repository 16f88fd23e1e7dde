// Adjacent-axis parallel-coordinates density histograms (Section 2.1 PC data,
// Fig. 2): for every in-shell (and, optionally, in-brush) cell and every pair
// of adjacent axes (a, a+1), H[a][bin_a][bin_{a+1}] += 1.
//
// A scan over HBM plus the binning of the kept cells. A warp walks one x-row
// of cells at a time so the planar loads are coalesced; rows whose cells all
// lie outside the shell are skipped without touching memory. The vector kernel
// streams 16-byte chunks of a row per variable (8 FP16 or 4 FP32 cells per
// lane) through a cp.async double buffer in shared memory; the scalar kernel
// (ragged grid edges, unaligned fields) takes one cell per lane. A cell's axis
// values that are not brushed are loaded only after its brushed values pass.
// Position axes and the position brush use the cell centre, coordinate
// RN((2i + 1 - n) / n). With the volume's own brush the cells of inactive 4^3
// sub-bricks are skipped without loads: every vertex of such a sub-brick fails
// the brush (its values lie between the sub-brick's min and max) or lies
// outside the shell (the sub-brick's widened box, which holds the vertex
// centres, misses the shell). The in-shell test is integer-exact. Bins come
// from the FP32 edges held in shared memory (comparisons only, so exact).
// Increments are aggregated over runs of neighbouring cells that share their
// bins (one atomicAdd per run), and on large grids spread over partial
// histograms that a reduction sums, so the hot bins of a smooth field do not
// serialise in L2.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "host_math.h"

namespace raypc {

namespace {

constexpr int kHistThreads = 256;                    // scalar kernel
constexpr int kHistWarps = kHistThreads / 32;
constexpr int kHistVecThreads = 512;                 // vector kernel (two resident blocks per SM)
constexpr int kHistVecWarps = kHistVecThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// Number of interior edges e_1..e_{bins-1} that are <= v, for non-decreasing
// edges, from the staged table whose first and last entries are -inf and +inf
// (stage_edges): j from an affine guess is the answer iff e[j] <= v < e[j+1]
// (both loaded at once); otherwise the guess is walked to the answer with
// comparisons of interior edges only (exact for any edges; equally spaced
// edges rarely need a step). NaN compares false everywhere and lands in bin 0;
// +inf fails only the last check of bin bins-1 and walks back to it.
__device__ __forceinline__ int bin_of(const float* e, int bins, float v, float scale, float off) {
    float g = fmaf(v, scale, off);                         // any guess is verified below
    g = fminf(fmaxf(g, 0.0f), (float)(bins - 1));          // a NaN guess becomes 0
    int j = __float_as_int(__fadd_rd(g, 0x1p23f)) - 0x4b000000;   // floor(g): 0 <= g < 2^23
    const float lo = e[j], hi = e[j + 1];
    if ((v >= lo) & (v < hi)) return j;
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
    float guess_scale[kMaxVars], guess_off[kMaxVars];   // bin guess fma(v, scale, off)
    long long soff[kMaxVars];      // byte offset of each load slot's plane (vector kernel)
    int rot;                       // row order: plane z is rotated in y by z * rot (mod n)
    uint32_t* rowctr;              // zeroed row counter, or null: rows by warp stride
    int s_in, s_out;               // shell test on 2x+1-n etc., clamped to int
    uint32_t* out;                 // nout histograms; block b adds to copy b % nout
    int nout;
    const uint32_t* sactive;       // optional sub-brick activity (see HistArgs)
    int nsb;
    const float* edges;            // naxes x (bins + 1) on the device, or null: edges_inl
    float edges_inl[kInlineEdges];
};

// Copy the edge table into shared memory (all threads; the caller syncs), with
// each axis's outer edges e_0 and e_bins, which no count depends on, replaced by
// -inf and +inf so that bin_of checks a guess with two comparisons.
__device__ __forceinline__ void stage_edges(const HistLaunch& A, float* s_edges) {
    const int ne = A.naxes * (A.bins + 1);
    for (int i = threadIdx.x; i < ne; i += blockDim.x) {
        const int k = i % (A.bins + 1);
        s_edges[i] = k == 0 ? -INFINITY : k == A.bins ? INFINITY : A.edges ? __ldg(A.edges + i) : A.edges_inl[i];
    }
}

// Row geometry shared by both kernels: the x range of the r-th row (y, z) inside the
// outer sphere, |2x + 1 - n| <= m, and the range [ca, cb] of its cells inside the
// inner sphere (empty when ca > cb); false when the whole row lies outside.
// Rows are taken in z-planes whose y order is rotated by z * rot. With a row
// counter the vector kernel's warps take the next untaken rows whenever they
// finish (rot = 0): they finish together whatever the brush leaves in each row.
// Without one they take rows by warp stride, and rot is a golden-ratio fraction
// of n: a stride that is a multiple of n would otherwise give every warp one y
// -- all its rows long chords through the shell or all short ones near the
// outer sphere. The scalar kernel keeps the plain order (rot = 0).
struct RowSpan {
    int y, z, syz, xa, xb, ca, cb;
    float cy, cz;
    size_t base;                   // (z n + y) n
    uint32_t srow;                 // first sub-brick id of the row's sub-brick row
};

__device__ __forceinline__ bool row_span(const HistLaunch& A, int r, RowSpan& R) {
    const int n = A.n;
    R.z = r / n;
    R.y = r - R.z * n + (R.z * A.rot) % n;                  // z * rot < 2^24 for n <= 4096
    if (R.y >= n) R.y -= n;
    const int dy = 2 * R.y + 1 - n, dz = 2 * R.z + 1 - n;
    R.syz = dy * dy + dz * dz;                              // < 2^31 for n <= 4096
    if (R.syz > A.s_out) return false;
    const int m = isqrt_floor(A.s_out - R.syz);
    R.xa = max(0, (n - m) / 2);
    R.xb = min(n - 1, (n - 1 + m) / 2);
    R.ca = 1;
    R.cb = 0;
    const int din = A.s_in - R.syz;                         // cells with dx^2 < din fail the shell test
    if (din > 0) {
        const int mi = isqrt_floor(din - 1);                // |2x + 1 - n| <= mi
        R.ca = max(0, (n - mi) / 2);
        R.cb = min(n - 1, (n - 1 + mi) / 2);
    }
    R.cy = A.use_pos ? cell_centre_rn(R.y, n) : 0.0f;
    R.cz = A.use_pos ? cell_centre_rn(R.z, n) : 0.0f;
    R.base = ((size_t)R.z * n + R.y) * n;
    R.srow = ((uint32_t)(R.z >> 2) * A.nsb + (uint32_t)(R.y >> 2)) * A.nsb;
    return true;
}

// The warp's row after r (r = its warp index - nwarps: its first row). With a
// row counter, warps take batches of kRowBatch neighbouring rows: warp w starts
// with batch w, and every later batch is nwarps + the counter's next value,
// taken one batch ahead in lane 0's rq (first_batch gives its initial value) so
// that the atomic's latency hides behind a batch's work, and few enough atomics
// meet at the one address. Without one, rows go by warp stride. Every lane calls
// it; the result is the same in all of them.
constexpr int kRowBatch = 2;

__device__ __forceinline__ unsigned first_batch(const HistLaunch& A, int gwarp) {
    return A.rowctr ? (unsigned)gwarp : 0u;
}

__device__ __forceinline__ int take_row(const HistLaunch& A, int r, int rows, int nwarps, int lane, unsigned& rq) {
    if (!A.rowctr) return r + nwarps;
    if (r >= 0 && (r + 1) % kRowBatch != 0) return r + 1;
    const int t = (int)__shfl_sync(kFull, rq, 0) * kRowBatch;
    if (t < rows && lane == 0) rq = (unsigned)nwarps + atomicAdd(A.rowctr, 1u);
    return t;
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
// grid, rows by warp stride in their plain order (the launch gives it rot = 0 and
// no row counter: either costs this latency-bound kernel registers and time).
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
    uint32_t* const out = A.out + (size_t)(blockIdx.x % (unsigned)A.nout) * (A.naxes - 1) * bins * bins;

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
                        b = (unsigned)bin_of(s_edges + a * (bins + 1), bins, v, A.guess_scale[a], A.guess_off[a]);
                    }
                    if (a > 0) add_runs(out + (size_t)(a - 1) * bins * bins, prev * (unsigned)bins + b, keep[j], km, lane);
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

// Asynchronous 16-byte global -> shared copies (no registers held while in
// flight); a group is waited for with cp.async.wait_group, a hardware wait.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// One chunk row of the vector kernel: 32 lanes x VEC consecutive cells of row r
// starting at xw, and this lane's cells that pass the geometric tests.
struct ChunkRow {
    int r, xw;                     // r = -1: none
    RowSpan R;
    unsigned kb;
    unsigned rq;                   // with a row counter, lane 0: the row to take after this one
};


// Bits j of [0, VEC) with lo <= j <= hi.
template <int VEC>
__device__ __forceinline__ unsigned span_bits(int lo, int hi) {
    const int l = max(lo, 0), h = min(hi, VEC - 1);
    return l > h ? 0u : (2u << h) - (1u << l);
}

// Geometric keep bits of this lane's chunk (x0 .. x0 + VEC - 1; x0 and n multiples
// of VEC): in the shell (the row's ranges), in an active sub-brick when the
// activity is given, inside the position brush. A chunk with a cell in the shell
// lies inside the row, so its sub-brick ids are valid.
template <int VEC>
__device__ __forceinline__ unsigned chunk_geometry(const HistLaunch& A, const RowSpan& R, int x0) {
    unsigned kb = span_bits<VEC>(R.xa - x0, R.xb - x0) & ~span_bits<VEC>(R.ca - x0, R.cb - x0);
    if (kb && A.sactive) {
        // the chunk's VEC / 4 sub-bricks sit in one activity word unless the first is bit 31
        const uint32_t sid = R.srow + (uint32_t)(x0 >> 2);
        unsigned act = __ldg(A.sactive + (sid >> 5)) >> (sid & 31);
        if (VEC > 4 && (sid & 31) > 32 - VEC / 4) act |= __ldg(A.sactive + (sid >> 5) + 1) << (32 - (sid & 31));
#pragma unroll
        for (int q = 0; q < VEC / 4; ++q)
            if (!((act >> q) & 1u)) kb &= ~(0xfu << (4 * q));
    }
    if (kb && A.pmask) {
        BrushArgs pb;
#pragma unroll
        for (int a = 0; a < kNumPos; ++a) { pb.plo[a] = A.plo[a]; pb.phi[a] = A.phi[a]; }
        pb.pmask = A.pmask;
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            const float cx = cell_centre_rn(x0 + j, A.n);
            if (((kb >> j) & 1u) && !pos_pass(cx, R.cy, R.cz, dot3_rn(cx, R.cy, R.cz, cx, R.cy, R.cz), pb))
                kb &= ~(1u << j);
        }
    }
    return kb;
}

// The warp's next chunk row after (r, xw): the next chunk of the same row, else the
// first chunk of the next row (by warp stride) that meets the outer sphere and holds
// a cell passing the geometric tests in some lane.
template <int VEC>
__device__ __forceinline__ void next_chunk_row(const HistLaunch& A, int nwarps, int lane, ChunkRow& C) {
    constexpr int CH = 32 * VEC;
    const int rows = A.n * A.n;
    int r = C.r, xw = C.xw + CH;
    bool have_row = r >= 0;
    for (;;) {
        if (!have_row || xw > C.R.xb) {
            r = take_row(A, r, rows, nwarps, lane, C.rq);
            if (r >= rows) { C.r = -1; C.kb = 0u; return; }
            if (!row_span(A, r, C.R)) { have_row = false; continue; }
            have_row = true;
            xw = C.R.xa & ~(VEC - 1);
        }
        const unsigned kb = chunk_geometry<VEC>(A, C.R, xw + lane * VEC);
        if (__ballot_sync(kFull, kb != 0u) != 0u) {
            C.r = r;
            C.xw = xw;
            C.kb = kb;
            return;
        }
        xw += CH;
    }
}

// One binning round of the vector kernel: lane l holds a cell iff kept (the kept lanes
// are a prefix, km their mask) with its axis values val[a]. Bins come from the FP32 edges in
// shared memory; a lane whose bin tuple differs from its left neighbour's starts a run and
// adds the run's length to each adjacent-axis pair (one atomic per pair and run).
__device__ __forceinline__ void bin_round(const HistLaunch& A, const float* s_edges, uint32_t* out,
                                          const float (&val)[kMaxVars], bool kept, unsigned km, int lane) {
    const int naxes = A.naxes, bins = A.bins;
    unsigned bn[kMaxVars];
    unsigned packed[3] = {0u, 0u, 0u};                      // three bins per word, 10 bits each
#pragma unroll
    for (int a = 0; a < kMaxVars; ++a) {
        bn[a] = 0u;
        if (a >= naxes || !kept) continue;
        bn[a] = (unsigned)bin_of(s_edges + a * (bins + 1), bins, val[a], A.guess_scale[a], A.guess_off[a]);
        packed[a / 3] |= bn[a] << (10 * (a % 3));
    }
    bool same = lane > 0;
#pragma unroll
    for (int w = 0; w < 3; ++w) {
        if (3 * w >= naxes) break;
        const unsigned left = __shfl_up_sync(kFull, packed[w], 1);   // every lane takes part
        same = same && left == packed[w];
    }
    const bool head = kept && !same;
    const unsigned hm = __ballot_sync(kFull, head);
    if (head) {
        const unsigned after = lane == 31 ? 0u : (kFull << (lane + 1));
        const unsigned stop = (hm | ~km) & after;            // next run start or the last kept lane
        const unsigned len = (unsigned)((stop ? __ffs(stop) - 1 : 32) - lane);
#pragma unroll
        for (int a = 1; a < kMaxVars; ++a) {
            if (a >= naxes) break;
            atomicAdd(out + (size_t)(a - 1) * bins * bins + bn[a - 1] * (unsigned)bins + bn[a], len);
        }
    }
}

// Vector kernel (grid edge a multiple of the chunk, 16-byte aligned planes, at most
// kMaxVars load slots). A warp walks x-rows in chunk rows of 32 lanes x 16 bytes
// (8 FP16 or 4 FP32 cells per lane). While it tests and bins one chunk row it has
// the next one's slots copied into its other shared buffer with cp.async (only
// chunks with a cell that passes the shell, sub-brick and position tests), so
// HBM latency hides behind the binning and no registers wait on loads. All
// brushed slots are tested (FP16: two cells at a time against exact binary16
// bounds); the surviving cells go into a compact list in x order (warp prefix
// sum) from which the warp bins 32 cells per round, reading the axis values
// from the buffer. Neighbouring lanes then hold neighbouring cells, whose bin
// tuples mostly agree on a smooth field: a lane whose tuple differs from its
// left neighbour's starts a run and adds the run's length to each
// adjacent-axis pair (one atomic per pair and run). Persistent grid, rows from
// the row counter or by warp stride; the edge table is staged once per resident
// block.
template <int DT>
__global__ void __launch_bounds__(kHistVecThreads, 2) k_hist(const __grid_constant__ HistLaunch A) {
    constexpr int VEC = DT == kF16 ? 8 : 4;
    extern __shared__ __align__(16) unsigned char s_raw[];
    float* s_edges = reinterpret_cast<float*>(s_raw);
    const int ne16 = (A.naxes * (A.bins + 1) + 3) & ~3;
    const int nslot = A.nslot, naxes = A.naxes;
    const int buf_bytes = nslot * 512;                          // one chunk row of every slot
    unsigned char* s_warp = s_raw + sizeof(float) * ne16 + (size_t)(threadIdx.x >> 5) * (2 * buf_bytes + 256);
    unsigned char* s_list = s_warp + 2 * buf_bytes;
    stage_edges(A, s_edges);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int n = A.n;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int bins = A.bins;
    const uint32_t sbr = A.sbr;
    uint32_t* const out = A.out + (size_t)(blockIdx.x % (unsigned)A.nout) * (naxes - 1) * bins * bins;

    // copies of chunk row C into buffer b (lanes whose chunk has no passing cell copy nothing)
    auto prefetch = [&](const ChunkRow& C, int b) {
        if (C.r >= 0 && C.kb) {
            const int x0 = C.xw + lane * VEC;
            unsigned char* dst = s_warp + b * buf_bytes + lane * 16;
            const char* src = static_cast<const char*>(A.cells) + (C.R.base + x0) * (16 / VEC);
#pragma unroll
            for (int s = 0; s < kMaxVars; ++s)
                if (s < nslot && A.svar[s] >= 0) cp_async16(dst + s * 512, src + A.soff[s]);
        }
        cp_async_commit();
    };

    const bool carry = DT == kF16 && !A.use_pos;
    int q = 0;                                                  // carried cells, in lanes 0..q-1
    unsigned cpk[kMaxVars / 2] = {0u, 0u, 0u, 0u};              // a carried cell's values, binary16 pairs

    ChunkRow cur;
    cur.r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) - nwarps;
    cur.xw = 0;
    cur.rq = first_batch(A, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5));
    next_chunk_row<VEC>(A, nwarps, lane, cur);
    prefetch(cur, 0);
    int b = 0;
    while (cur.r >= 0) {
        ChunkRow nxt = cur;
        next_chunk_row<VEC>(A, nwarps, lane, nxt);
        prefetch(nxt, b ^ 1);
        cp_async_wait_prev();                                   // this chunk row's copies have landed
        __syncwarp();
        const unsigned char* buf = s_warp + b * buf_bytes;
        unsigned kb = cur.kb;
        // brushed slots
        if constexpr (DT == kF16) {
            unsigned acc[4] = {kFull, kFull, kFull, kFull};
#pragma unroll
            for (int s = 0; s < kMaxVars; ++s) {
                if (s < nslot && ((sbr >> s) & 1u)) {
                    const uint4 v = *reinterpret_cast<const uint4*>(buf + s * 512 + lane * 16);
                    const __half2 lo2 = u32_as_half2(A.slo_h2[s]), hi2 = u32_as_half2(A.shi_h2[s]);
                    const unsigned w[4] = {v.x, v.y, v.z, v.w};
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
                    const uint4 v = *reinterpret_cast<const uint4*>(buf + s * 512 + lane * 16);
                    const float lo = A.slo[s], hi = A.shi[s];
#pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        const float x = chunk_elem<DT>(v, j);
                        if (!(x >= lo && x <= hi)) kb &= ~(1u << j);
                    }
                }
            }
        }
        // compact list of the surviving cells (chunk-row offsets) in x order: the exclusive
        // prefix of the per-lane counts from an inclusive shuffle scan
        const unsigned cnt = (unsigned)__popc(kb);
        unsigned inc = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned t = __shfl_up_sync(kFull, inc, d);
            if (lane >= d) inc += t;
        }
        int pos = (int)(inc - cnt);
        const int total = (int)__shfl_sync(kFull, inc, 31);
#pragma unroll
        for (int j = 0; j < VEC; ++j)
            if ((kb >> j) & 1u) s_list[pos++] = (unsigned char)(lane * VEC + j);
        __syncwarp();
        // bin the surviving cells 32 per round. FP16 without position axes carries a remainder
        // of fewer than 32 cells to the next chunk row (their values in the lanes' registers),
        // so that sparse chunk rows still fill whole rounds
        int consumed = 0;
#pragma unroll 1
        for (;;) {
            const int avail = q + total - consumed;
            if (avail == 0) break;
            if (carry && avail < 32) {
                if (lane >= q && lane < avail) {
                    const int c = s_list[consumed + lane - q];
#pragma unroll
                    for (int a = 0; a < kMaxVars; ++a) {
                        if (a >= naxes) break;
                        const unsigned hb = reinterpret_cast<const unsigned short*>(buf + a * 512)[c];
                        cpk[a >> 1] = (cpk[a >> 1] & (0xffff0000u >> (16 * (a & 1)))) | (hb << (16 * (a & 1)));
                    }
                }
                q = avail;
                break;
            }
            const int take = min(32, avail);
            const bool kept = lane < take;
            const unsigned km = take == 32 ? kFull : (1u << take) - 1u;
            float val[kMaxVars];
#pragma unroll
            for (int a = 0; a < kMaxVars; ++a) val[a] = 0.0f;
            if (kept && lane < q) {                             // a carried cell
#pragma unroll
                for (int a = 0; a < kMaxVars; ++a)
                    if (a < naxes)
                        val[a] = __half2float(__ushort_as_half((unsigned short)(cpk[a >> 1] >> (16 * (a & 1)))));
            } else if (kept) {
                const int c = s_list[consumed + lane - q];       // cell cur.xw + c
                float cx = 0.0f, cr2 = 0.0f;
                if (A.use_pos) {
                    cx = cell_centre_rn(cur.xw + c, n);
                    cr2 = dot3_rn(cx, cur.R.cy, cur.R.cz, cx, cur.R.cy, cur.R.cz);
                }
#pragma unroll
                for (int a = 0; a < kMaxVars; ++a) {
                    if (a >= naxes) break;
                    const int av = A.avar[a];
                    if (av >= kPosAxisBase)
                        val[a] = pos_axis(cx, cur.R.cy, cur.R.cz, cr2, av - kPosAxisBase);
                    else if (DT == kF16)
                        val[a] = __half2float(__ushort_as_half(reinterpret_cast<const unsigned short*>(buf + a * 512)[c]));
                    else
                        val[a] = reinterpret_cast<const float*>(buf + a * 512)[c];
                }
            }
            bin_round(A, s_edges, out, val, kept, km, lane);
            consumed += take - q;
            q = 0;
        }
        __syncwarp();                                           // buffer b and the list are reused next
        cur = nxt;
        b ^= 1;
    }
    if (q > 0) {                                                // the last carried cells
        const bool kept = lane < q;
        float val[kMaxVars];
#pragma unroll
        for (int a = 0; a < kMaxVars; ++a)
            val[a] = kept && a < naxes ? __half2float(__ushort_as_half((unsigned short)(cpk[a >> 1] >> (16 * (a & 1)))))
                                       : 0.0f;
        bin_round(A, s_edges, out, val, kept, (1u << q) - 1u, lane);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// out[i] = sum over the copies of copy[c][i] (count a multiple of 4, 16-byte aligned).
__global__ void __launch_bounds__(256) k_hist_reduce(const uint4* __restrict__ copies, int ncopies, size_t count4,
                                                     uint4* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count4; i += (size_t)gridDim.x * blockDim.x) {
        uint4 s = __ldcs(copies + i);
        for (int c = 1; c < ncopies; ++c) {
            const uint4 v = __ldcs(copies + (size_t)c * count4 + i);
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        out[i] = s;
    }
}

// Kernel view of h. False when the edge table is neither small enough for the
// launch parameters nor on the device; vec_slots reports whether the load
// slots fit the vector kernel.
template <int DT>
bool fill_launch(const HistArgs& h, HistLaunch& a, bool& vec_slots) {
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
        a.guess_scale[i] = h.guess_scale[i];
        a.guess_off[i] = -h.guess_e0[i] * h.guess_scale[i];
    }
    // load slots of the vector kernel: the axes, then the brushed variables that are no axis
    vec_slots = true;
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
    const long long plane_bytes = (long long)h.n * h.n * h.n * (DT == kF16 ? 2 : 4);
    for (int s = 0; s < a.nslot && s < kMaxVars; ++s) a.soff[s] = a.svar[s] >= 0 ? a.svar[s] * plane_bytes : 0;
    a.rowctr = h.rowctr;
    a.rot = h.rowctr ? 0 : (int)(0.6180339887498949 * h.n);
    if (DT == kF16)
        for (int s = 0; s < a.nslot && s < kMaxVars; ++s) {
            const uint32_t lo = half_ceil_bits(a.slo[s]), hi = half_floor_bits(a.shi[s]);
            a.slo_h2[s] = lo | (lo << 16);
            a.shi_h2[s] = hi | (hi << 16);
        }
    const int64_t imax = 0x7fffffff;
    a.s_in = (int)std::min<int64_t>(std::max<int64_t>(h.s_in, 0), imax);
    a.s_out = (int)std::min<int64_t>(h.s_out, imax);
    a.out = h.ncopies > 1 ? h.copies : h.out;
    a.nout = h.ncopies > 1 ? h.ncopies : 1;
    a.sactive = h.sactive;
    a.nsb = h.nsb;
    const int ne = h.naxes * (h.bins + 1);
    if (h.edges_host && ne <= kInlineEdges) {
        for (int i = 0; i < ne; ++i) a.edges_inl[i] = h.edges_host[i];
        a.edges = nullptr;
    } else if (h.edges) {
        a.edges = h.edges;
    } else {
        return false;
    }
    return true;
}

template <int DT>
cudaError_t launch_t(const HistArgs& h, cudaStream_t stream) {
    HistLaunch a{};                      // about 8.6 KB with the inline edges (host stack)
    bool vec_slots = true;
    if (!fill_launch<DT>(h, a, vec_slots)) return cudaErrorInvalidValue;
    const int ne = h.naxes * (h.bins + 1);
    if (h.s_out < 0) return cudaSuccess;                 // no cell in the shell: the zeroed output is the answer
    constexpr int VEC = DT == kF16 ? 8 : 4;
    const bool vec = vec_slots && h.n % VEC == 0 && (reinterpret_cast<uintptr_t>(h.cells) & 15u) == 0;
    const size_t smem = vec ? sizeof(float) * (size_t)((ne + 3) & ~3) + (size_t)kHistVecWarps * (2 * a.nslot * 512 + 256)
                            : sizeof(float) * (size_t)ne;
    // persistent grid: as many blocks as fit at once
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && vec && smem > 48 * 1024)
        e = cudaFuncSetAttribute(k_hist<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist<DT>, kHistVecThreads, smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist_scalar<DT>, kHistThreads, smem);
    if (e != cudaSuccess) return e;
    const long long rows = (long long)a.n * a.n;
    const int warps_per_block = vec ? kHistVecWarps : kHistWarps;
    const long long want_blocks = (rows + warps_per_block - 1) / warps_per_block;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(want_blocks, (long long)sms * std::max(1, per_sm)));
    if (!vec) {
        a.rot = 0;
        a.rowctr = nullptr;
    }
    if (vec) k_hist<DT><<<blocks, kHistVecThreads, smem, stream>>>(a);
    else k_hist_scalar<DT><<<blocks, kHistThreads, smem, stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

int hist_copies(int n, int naxes, int bins) {
    const size_t bytes = sizeof(uint32_t) * (size_t)(naxes - 1) * bins * bins;
    if ((long long)n * n * n < (1LL << 21) || bytes % 16) return 1;      // small grids: not worth a pass
    const size_t fit = kHistCopyBytes / bytes;
    return (int)std::min<size_t>(kHistMaxCopies, fit);
}

cudaError_t launch_histogram_reduce(const uint32_t* copies, int ncopies, size_t count, uint32_t* out,
                                    cudaStream_t stream) {
    const size_t count4 = count / 4;
    const unsigned blocks = (unsigned)std::min<size_t>((count4 + 255) / 256, 4096);
    k_hist_reduce<<<blocks, 256, 0, stream>>>(reinterpret_cast<const uint4*>(copies), ncopies, count4,
                                               reinterpret_cast<uint4*>(out));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_histogram(const HistArgs& a, int dtype, cudaStream_t stream) {
    if (dtype == kF16) return launch_t<kF16>(a, stream);
    return launch_t<kF32>(a, stream);
}

}  // namespace raypc

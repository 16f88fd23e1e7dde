// Adjacent-axis parallel-coordinates density histograms (Section 2.1 PC data,
// Fig. 2): for every in-shell (and, optionally, in-brush) cell and every pair
// of adjacent axes (a, a+1), H[a][bin_a][bin_{a+1}] += 1.
//
// HBM-bound scan. A warp walks one x-row of cells (lanes over x, two cells per
// lane in flight), so the planar loads of the needed variables are coalesced; rows whose cells all lie
// outside the shell are skipped without touching memory. The in-shell test is
// integer-exact. Bins come from a binary search over the FP32 edges held in
// shared memory (comparisons only, so exact). Increments are aggregated per
// warp with __match_any_sync on the (bin_a, bin_{a+1}) key: one atomicAdd per
// distinct key per warp and pair.
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

// Largest integer m >= 0 with m * m <= a (a >= 0).
__device__ __forceinline__ long long isqrt_floor(long long a) {
    long long m = (long long)sqrt((double)a);
    while (m * m > a) --m;
    while ((m + 1) * (m + 1) <= a) ++m;
    return m;
}

template <int DT>
__global__ void __launch_bounds__(kHistThreads) k_hist(HistArgs A) {
    extern __shared__ float s_edges[];
    const int ne = A.naxes * (A.bins + 1);
    for (int i = threadIdx.x; i < ne; i += blockDim.x) s_edges[i] = A.edges[i];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int n = A.n;
    const long long rows = (long long)n * n;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int bins = A.bins;
    const size_t plane = (size_t)n * n * n;
    const unsigned brush_mask = A.use_brush ? A.brush.mask : 0u;
    const unsigned rest_mask = A.need_mask & ~brush_mask;

    for (long long r = gwarp; r < rows; r += nwarps) {
        const int y = (int)(r % n), z = (int)(r / n);
        const long long dy = 2 * y + 1 - n, dz = 2 * z + 1 - n;
        const long long syz = dy * dy + dz * dz;
        if (syz > A.s_out) continue;                       // whole row outside the outer sphere
        // x range of the row inside the outer sphere: |2x + 1 - n| <= m
        const long long m = isqrt_floor(A.s_out - syz);
        const int xa = (int)max(0LL, (n - 1 - m + 1) / 2);
        const int xb = (int)min((long long)n - 1, (n - 1 + m) / 2);
        const size_t row_base = (size_t)r * n;
        // two cells per lane and iteration: their loads are in flight together
        for (int x0 = xa; x0 <= xb; x0 += 64) {
            bool keep[2];
            int bn[2][kMaxVars];
            float val[2][kMaxVars];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int x = x0 + lane + 32 * j;
                keep[j] = false;
                if (x <= xb) {
                    const long long dx = 2 * x + 1 - n;
                    const long long s = dx * dx + syz;
                    keep[j] = s >= A.s_in && s <= A.s_out;
                }
            }
            // brushed variables first; the rest only for cells that pass
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const size_t off = row_base + x0 + lane + 32 * j;
#pragma unroll
                for (int v = 0; v < kMaxVars; ++v)
                    val[j][v] = (keep[j] && ((brush_mask >> v) & 1u)) ? load_cell<DT>(A.cells, v * plane + off) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int v = 0; v < kMaxVars; ++v)
                    if ((brush_mask >> v) & 1u)
                        keep[j] = keep[j] && (val[j][v] >= A.brush.lo[v]) && (val[j][v] <= A.brush.hi[v]);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const size_t off = row_base + x0 + lane + 32 * j;
#pragma unroll
                for (int v = 0; v < kMaxVars; ++v)
                    if (keep[j] && ((rest_mask >> v) & 1u)) val[j][v] = load_cell<DT>(A.cells, v * plane + off);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (keep[j]) {
#pragma unroll
                    for (int a = 0; a < kMaxVars; ++a) {
                        if (a < A.naxes) {
                            float va = val[j][0];
#pragma unroll
                            for (int v = 1; v < kMaxVars; ++v)
                                if (A.axis[a] == v) va = val[j][v];
                            bn[j][a] = bin_of(s_edges + a * (bins + 1), bins, va, A.guess_e0[a], A.guess_scale[a]);
                        }
                    }
                }
                const unsigned km = __ballot_sync(0xffffffffu, keep[j]);
                if (km == 0u) continue;
                if (keep[j]) {
#pragma unroll
                    for (int p = 0; p + 1 < kMaxVars; ++p) {
                        if (p + 1 < A.naxes) {
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
}

template <int DT>
cudaError_t launch_t(const HistArgs& a, cudaStream_t stream) {
    // one row per warp (rows differ in length; the hardware balances blocks)
    long long rows = (long long)a.n * a.n;
    long long want_blocks = (rows + (kHistThreads / 32) - 1) / (kHistThreads / 32);
    int blocks = (int)(want_blocks < 0x7fffffffLL ? want_blocks : 0x7fffffffLL);
    if (blocks < 1) blocks = 1;
    size_t smem = sizeof(float) * a.naxes * (a.bins + 1);
    k_hist<DT><<<blocks, kHistThreads, smem, stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_histogram(const HistArgs& a, int dtype, cudaStream_t stream) {
    if (dtype == kF16) return launch_t<kF16>(a, stream);
    return launch_t<kF32>(a, stream);
}

}  // namespace raypc

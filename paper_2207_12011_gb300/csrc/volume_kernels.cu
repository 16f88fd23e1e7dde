// Volume preparation kernels: ingest/relayout and level-of-detail mean fused
// with brick min/max, and brush classification of bricks.
//
// Section 2.1 of the paper prepares the data once (levels of detail, derived
// variables); Section 2.2 relies on that preparation not depending on the
// restrictions, so a brush edit only re-runs the (cheap) classification.
#include "common.cuh"

namespace raypc {

namespace {

constexpr int kRowThreads = 256;

__device__ __forceinline__ float load_src(const void* src, int dtype, size_t i) {
    if (dtype == kF16) return __half2float(__ldg(reinterpret_cast<const __half*>(src) + i));
    return __ldg(reinterpret_cast<const float*>(src) + i);
}

// Round to the storage dtype (the stored value, as a float).
template <int DT> __device__ __forceinline__ float to_stored(float v);
template <> __device__ __forceinline__ float to_stored<kF32>(float v) { return v; }
template <> __device__ __forceinline__ float to_stored<kF16>(float v) { return __half2float(__float2half_rn(v)); }

template <int DT> __device__ __forceinline__ void store_cell(void* cells, size_t i, float v);
template <> __device__ __forceinline__ void store_cell<kF32>(void* cells, size_t i, float v) {
    reinterpret_cast<float*>(cells)[i] = v;
}
template <> __device__ __forceinline__ void store_cell<kF16>(void* cells, size_t i, float v) {
    reinterpret_cast<__half*>(cells)[i] = __float2half_rn(v);
}

template <int DT> __device__ __forceinline__ void store_pair(void* pairs, size_t i, float a, float b);
template <> __device__ __forceinline__ void store_pair<kF32>(void* pairs, size_t i, float a, float b) {
    reinterpret_cast<float2*>(pairs)[i] = make_float2(a, b);
}
template <> __device__ __forceinline__ void store_pair<kF16>(void* pairs, size_t i, float a, float b) {
    reinterpret_cast<__half2*>(pairs)[i] = __floats2half2_rn(a, b);
}

struct RowsArgs {
    const void* src;      // ingest: planar source (src_dtype); LOD: planar cells of the finer level
    int src_dtype;        // ingest only
    int n_src;            // LOD: edge of the finer level
    void* cells;          // this level, planar
    void* pairs;          // this level, x-pairs
    int n;                // edge of this level
    int nvars;
    float* bmin;          // [nb^3][nvars]
    float* bmax;
};

// Value of cell (x, y, z) of variable v of the level being produced, rounded
// to the storage dtype.
//   MODE 0 (ingest): the converted source value.
//   MODE 1 (LOD):    FP32 mean of the 2x2x2 fine cells, fine indices clamped,
//                    ((c000 + c100) + (c010 + c110)) + ((c001 + c101) + (c011 + c111)), x 1/8.
template <int DT, int MODE>
__device__ __forceinline__ float produce(const RowsArgs& A, int x, int y, int z, int v) {
    if (MODE == 0) {
        const size_t n = (size_t)A.n;
        return to_stored<DT>(load_src(A.src, A.src_dtype, ((v * n + z) * n + y) * n + x));
    } else {
        const int nf = A.n_src;
        const int x0 = 2 * x, y0 = 2 * y, z0 = 2 * z;
        const int x1 = min(x0 + 1, nf - 1), y1 = min(y0 + 1, nf - 1), z1 = min(z0 + 1, nf - 1);
        const size_t plane = (size_t)v * nf * nf * nf;
        auto at = [&](int a, int b, int c) { return load_cell<DT>(A.src, plane + ((size_t)c * nf + b) * nf + a); };
        float s0 = __fadd_rn(__fadd_rn(at(x0, y0, z0), at(x1, y0, z0)), __fadd_rn(at(x0, y1, z0), at(x1, y1, z0)));
        float s1 = __fadd_rn(__fadd_rn(at(x0, y0, z1), at(x1, y0, z1)), __fadd_rn(at(x0, y1, z1), at(x1, y1, z1)));
        return to_stored<DT>(__fmul_rn(__fadd_rn(s0, s1), 0.125f));
    }
}

// One block per (brick row (by, bz), variable), up to 256 threads (one per x
// column, striding when the level is wider). Threads own x columns; the
// block streams the (up to) 9 x 9 x-rows y in [8by, 8by+8], z in [8bz, 8bz+8]
// of the level, writes the 8 x 8 rows it owns (cells and x-pairs; the right
// element of a pair comes from the neighbouring lane) and folds every row,
// apron rows included, into per-column NaN-ignoring min/max. Columns are then
// reduced to bricks in shared memory. Brick (bx, by, bz) covers vertices
// 8b..min(8b+8, n-1) on each axis.
template <int DT, int MODE>
__global__ void __launch_bounds__(kRowThreads) k_rows(RowsArgs A) {
    extern __shared__ float s_col[];          // [2][n]: column min, column max
    const int n = A.n;
    const int nb = (n + kBrick - 1) / kBrick;
    const int by = blockIdx.x % nb, bz = blockIdx.x / nb, v = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const float qnan = __int_as_float(0x7fffffff);
    for (int xc = 0; xc < n; xc += blockDim.x) {
        const int x = xc + threadIdx.x;
        const bool valid = x < n;
        float mn = qnan, mx = qnan;
        for (int dz = 0; dz <= kBrick; ++dz) {
            const int z = bz * kBrick + dz;
            if (z >= n) break;
            // Ingest: issue the (up to) 9 row loads of this z-slice before using
            // any of them (9 loads in flight per thread). LOD: one row at a time
            // (each value already costs 8 loads).
            constexpr int kAhead = MODE == 0 ? kBrick + 1 : 1;
            for (int dy0 = 0; dy0 <= kBrick; dy0 += kAhead) {
                float val[kAhead];
#pragma unroll
                for (int j = 0; j < kAhead; ++j) {
                    const int y = by * kBrick + dy0 + j;
                    val[j] = (valid && dy0 + j <= kBrick && y < n) ? produce<DT, MODE>(A, x, y, z, v) : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < kAhead; ++j) {
                    const int dy = dy0 + j;
                    const int y = by * kBrick + dy;
                    if (dy > kBrick || y >= n) break;
                    if (valid) {
                        mn = fminf(mn, val[j]);
                        mx = fmaxf(mx, val[j]);
                    }
                    if (dy < kBrick && dz < kBrick) {
                        float right = __shfl_down_sync(0xffffffffu, val[j], 1);
                        if (valid) {
                            if (x == n - 1) right = val[j];
                            else if (lane == 31) right = produce<DT, MODE>(A, x + 1, y, z, v);
                            const size_t i = (((size_t)v * n + z) * n + y) * n + x;
                            store_cell<DT>(A.cells, i, val[j]);
                            store_pair<DT>(A.pairs, i, val[j], right);
                        }
                    }
                }
            }
        }
        if (valid) {
            s_col[x] = mn;
            s_col[n + x] = mx;
        }
    }
    __syncthreads();
    for (int bx = threadIdx.x; bx < nb; bx += blockDim.x) {
        const int x0 = bx * kBrick, x1 = min(x0 + kBrick, n - 1);
        float mn = qnan, mx = qnan;
        for (int x = x0; x <= x1; ++x) {
            mn = fminf(mn, s_col[x]);
            mx = fmaxf(mx, s_col[n + x]);
        }
        const size_t b = ((size_t)bz * nb + by) * nb + bx;
        A.bmin[b * A.nvars + v] = mn;
        A.bmax[b * A.nvars + v] = mx;
    }
}

// Locate the level of a flat brick index over all levels (<= 3 levels).
__device__ __forceinline__ int level_of(const ClassifyArgs& C, size_t g, size_t& b) {
    int l = 0;
    while (l + 1 < C.nlev && g >= C.lv[l + 1].first) ++l;
    b = g - C.lv[l].first;
    return l;
}

// One thread per brick of every level: shell test of the widened box and brush
// test with the rounding margin d = max(|min|, |max|) * 2^-20 + 2^-120. Writes
// the active bitmask (one ballot word per warp; level ranges start on
// multiples of 32) and counts, per restricted variable, the in-shell bricks
// that pass that variable alone (a selectivity hint for the render).
__global__ void k_classify(ClassifyArgs C) {
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    size_t b = 0;
    const int l = level_of(C, g, b);
    const ClassifyLevel& L = C.lv[l];
    const int nb = (L.n + kBrick - 1) / kBrick;
    const size_t nbricks = (size_t)nb * nb * nb;
    const bool in_range = g < C.total;
    const bool valid = in_range && b < nbricks;
    bool act = false;
    unsigned pass_bits = 0;
    if (valid)
        act = classify_brick(b, nb, L.sc, C.rin2, C.rout2, C.brush, C.nvars, L.bmin, L.bmax, pass_bits);
    const unsigned word = __ballot_sync(0xffffffffu, act);
    if (lane == 0 && in_range && b < ((nbricks + 31) & ~(size_t)31)) L.active[b >> 5] = word;
    for (int v = 0; v < C.nvars; ++v) {
        const unsigned cnt = __popc(__ballot_sync(0xffffffffu, (pass_bits >> v) & 1u));
        if (lane == 0 && cnt) atomicAdd(&L.pass_count[v], cnt);
    }
}

// Skippable = this brick and its existing 26 neighbours are inactive.
__global__ void k_skippable(ClassifyArgs C) {
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    size_t b = 0;
    const int l = level_of(C, g, b);
    const ClassifyLevel& L = C.lv[l];
    const int nb = (L.n + kBrick - 1) / kBrick;
    const size_t nbricks = (size_t)nb * nb * nb;
    const bool in_range = g < C.total;
    const bool valid = in_range && b < nbricks;
    const bool s = valid && skippable_brick(b, nb, L.active);
    const unsigned word = __ballot_sync(0xffffffffu, s);
    if (lane == 0 && in_range && b < ((nbricks + 31) & ~(size_t)31)) L.skippable[b >> 5] = word;
}

// Ordered compaction of the active brick ids, one block of 1024 threads per
// level: each thread owns a contiguous run of bitmask words; a block-wide
// exclusive scan of the per-thread popcounts gives every thread its offset.
__global__ void __launch_bounds__(1024) k_compact(ClassifyArgs C) {
    __shared__ unsigned s_sum[1024];
    const ClassifyLevel& L = C.lv[blockIdx.x];
    const int nb = (L.n + kBrick - 1) / kBrick;
    const size_t nbricks = (size_t)nb * nb * nb;
    const size_t nwords = (nbricks + 31) / 32;
    const size_t per = (nwords + blockDim.x - 1) / blockDim.x;
    const size_t w0 = min(nwords, threadIdx.x * per), w1 = min(nwords, w0 + per);
    unsigned cnt = 0;
    for (size_t w = w0; w < w1; ++w) cnt += __popc(L.active[w]);
    s_sum[threadIdx.x] = cnt;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const unsigned add = threadIdx.x >= (unsigned)off ? s_sum[threadIdx.x - off] : 0u;
        __syncthreads();
        s_sum[threadIdx.x] += add;
        __syncthreads();
    }
    unsigned pos = s_sum[threadIdx.x] - cnt;
    for (size_t w = w0; w < w1; ++w) {
        uint32_t bits = L.active[w];
        while (bits) {
            const int j = __ffs(bits) - 1;
            bits &= bits - 1;
            const size_t id = w * 32 + j;
            if (id < nbricks) L.list[pos++] = (uint32_t)id;
        }
    }
    if (threadIdx.x == blockDim.x - 1) *L.n_active = s_sum[threadIdx.x];
}

inline unsigned blocks_for(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <int MODE>
cudaError_t launch_rows(const RowsArgs& a, int dtype, cudaStream_t stream) {
    const int nb = (a.n + kBrick - 1) / kBrick;
    dim3 grid((unsigned)(nb * nb), (unsigned)a.nvars);
    const size_t smem = sizeof(float) * 2 * (size_t)a.n;
    if (smem > 48 * 1024) {
        cudaError_t e = dtype == kF16
            ? cudaFuncSetAttribute(k_rows<kF16, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(k_rows<kF32, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // one thread per x column up to kRowThreads (narrow levels use narrow blocks)
    const int threads = min(kRowThreads, max(32, (a.n + 31) / 32 * 32));
    if (dtype == kF16)
        k_rows<kF16, MODE><<<grid, threads, smem, stream>>>(a);
    else
        k_rows<kF32, MODE><<<grid, threads, smem, stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ingest(const void* src, int src_dtype, void* cells, void* pairs, int dtype, int n,
                          int nvars, float* bmin, float* bmax, cudaStream_t stream) {
    RowsArgs a{};
    a.src = src;
    a.src_dtype = src_dtype;
    a.cells = cells;
    a.pairs = pairs;
    a.n = n;
    a.nvars = nvars;
    a.bmin = bmin;
    a.bmax = bmax;
    return launch_rows<0>(a, dtype, stream);
}

cudaError_t launch_lod(const void* fine, int n_fine, void* cells, void* pairs, int dtype, int nvars,
                       float* bmin, float* bmax, cudaStream_t stream) {
    RowsArgs a{};
    a.src = fine;
    a.n_src = n_fine;
    a.cells = cells;
    a.pairs = pairs;
    a.n = (n_fine + 1) / 2;
    a.nvars = nvars;
    a.bmin = bmin;
    a.bmax = bmax;
    return launch_rows<1>(a, dtype, stream);
}

cudaError_t launch_classify(ClassifyArgs& c, cudaStream_t stream) {
    size_t total = 0;
    for (int l = 0; l < c.nlev; ++l) {
        ClassifyLevel& L = c.lv[l];
        const int nb = (L.n + kBrick - 1) / kBrick;
        L.first = total;
        L.sc = 2.0f / (float)L.n;
        total += ((size_t)nb * nb * nb + 31) / 32 * 32;      // level ranges start on warp boundaries
        cudaError_t e = cudaMemsetAsync(L.pass_count, 0, sizeof(unsigned) * kMaxVars, stream);
        if (e != cudaSuccess) return e;
    }
    c.total = total;
    k_classify<<<blocks_for(total, 256), 256, 0, stream>>>(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_skippable<<<blocks_for(total, 256), 256, 0, stream>>>(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_compact<<<c.nlev, 1024, 0, stream>>>(c);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace raypc

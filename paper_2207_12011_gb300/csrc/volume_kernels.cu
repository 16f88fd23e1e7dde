// Volume preparation kernels: ingest/relayout, level-of-detail mean,
// brick min/max and brush classification of bricks.
//
// Section 2.1 of the paper prepares the data once (levels of detail, derived
// variables); Section 2.2 relies on that preparation not depending on the
// restrictions, so a brush edit only re-runs the (cheap) classification.
#include "common.cuh"

namespace raypc {

namespace {

__device__ __forceinline__ float load_src(const void* src, int dtype, size_t i) {
    if (dtype == kF16) return __half2float(reinterpret_cast<const __half*>(src)[i]);
    return reinterpret_cast<const float*>(src)[i];
}

// Store one value of a level: planar cell plus its two pair slots (as the
// left element of its own pair and the right element of the pair at x-1;
// the last x also fills its own right element).
template <int DT>
__device__ __forceinline__ void store_value(void* cells, void* pairs, size_t i, int x, int n, float v);

template <>
__device__ __forceinline__ void store_value<kF32>(void* cells, void* pairs, size_t i, int x, int n, float v) {
    reinterpret_cast<float*>(cells)[i] = v;
    float* p = reinterpret_cast<float*>(pairs);
    p[2 * i] = v;
    if (x > 0) p[2 * (i - 1) + 1] = v;
    if (x == n - 1) p[2 * i + 1] = v;
}

template <>
__device__ __forceinline__ void store_value<kF16>(void* cells, void* pairs, size_t i, int x, int n, float v) {
    __half h = __float2half_rn(v);
    reinterpret_cast<__half*>(cells)[i] = h;
    __half* p = reinterpret_cast<__half*>(pairs);
    p[2 * i] = h;
    if (x > 0) p[2 * (i - 1) + 1] = h;
    if (x == n - 1) p[2 * i + 1] = h;
}

// One thread per (variable, cell): convert the source value to the storage
// dtype and write the planar cell and both pair slots. Reads and writes are
// coalesced along x.
template <int DT>
__global__ void k_ingest(const void* __restrict__ src, int src_dtype, void* __restrict__ cells,
                         void* __restrict__ pairs, int n, size_t total) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int x = (int)(i % n);
    store_value<DT>(cells, pairs, i, x, n, load_src(src, src_dtype, i));
}

// Coarse cell = FP32 mean of its 2x2x2 fine cells (fine indices clamped):
// ((c000 + c100) + (c010 + c110)) + ((c001 + c101) + (c011 + c111)), x 1/8,
// then rounded to the storage dtype. One thread per (variable, coarse cell).
template <int DT>
__global__ void k_lod(const void* __restrict__ fine, int n, void* __restrict__ cells,
                      void* __restrict__ pairs, int nvars) {
    const int m = (n + 1) / 2;
    const size_t mm = (size_t)m * m * m;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mm * nvars) return;
    const int v = (int)(i / mm);
    const size_t c = i % mm;
    const int x = (int)(c % m), y = (int)((c / m) % m), z = (int)(c / ((size_t)m * m));
    const int x0 = 2 * x, y0 = 2 * y, z0 = 2 * z;
    const int x1 = min(x0 + 1, n - 1), y1 = min(y0 + 1, n - 1), z1 = min(z0 + 1, n - 1);
    const size_t plane = (size_t)v * n * n * n;
    auto at = [&](int a, int b, int cz) { return load_cell<DT>(fine, plane + ((size_t)cz * n + b) * n + a); };
    float s0 = __fadd_rn(__fadd_rn(at(x0, y0, z0), at(x1, y0, z0)), __fadd_rn(at(x0, y1, z0), at(x1, y1, z0)));
    float s1 = __fadd_rn(__fadd_rn(at(x0, y0, z1), at(x1, y0, z1)), __fadd_rn(at(x0, y1, z1), at(x1, y1, z1)));
    store_value<DT>(cells, pairs, i, x, m, __fmul_rn(__fadd_rn(s0, s1), 0.125f));
}

// One warp per brick: the 32 lanes stride over the brick's (up to) 9^3
// vertices, keep running NaN-ignoring min/max per variable, then reduce.
template <int DT>
__global__ void k_brick_minmax(const void* __restrict__ cells, int n, int nvars,
                               float* __restrict__ bmin, float* __restrict__ bmax) {
    int nb = (n + kBrick - 1) / kBrick;
    size_t nbricks = (size_t)nb * nb * nb;
    size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= nbricks) return;
    int bx = (int)(warp % nb), by = (int)((warp / nb) % nb), bz = (int)(warp / ((size_t)nb * nb));
    int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    int ex = min(x0 + kBrick, n - 1) - x0 + 1;
    int ey = min(y0 + kBrick, n - 1) - y0 + 1;
    int ez = min(z0 + kBrick, n - 1) - z0 + 1;
    int cnt = ex * ey * ez;
    const size_t plane = (size_t)n * n * n;
    for (int v = 0; v < nvars; ++v) {
        float mn = __int_as_float(0x7fffffff), mx = mn;
        for (int j = lane; j < cnt; j += 32) {
            int dx = j % ex, dy = (j / ex) % ey, dz = j / (ex * ey);
            float a = load_cell<DT>(cells, v * plane + ((size_t)(z0 + dz) * n + (y0 + dy)) * n + (x0 + dx));
            mn = fminf(mn, a);
            mx = fmaxf(mx, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            bmin[warp * nvars + v] = mn;
            bmax[warp * nvars + v] = mx;
        }
    }
}

// World box that the samples assigned to brick b (lower interpolation index in
// [8b, 8b+8)) can occupy along one axis, widened by 2^-10; the first and
// last bricks also own the clamped border.
__device__ __forceinline__ void brick_box_axis(int b, int nb, float sc, float& lo, float& hi) {
    lo = __fsub_rn(__fmaf_rn(__fadd_rn((float)(b * kBrick), 0.5f), sc, -1.0f), 0x1p-10f);
    hi = __fadd_rn(__fmaf_rn(__fadd_rn((float)(b * kBrick + kBrick), 0.5f), sc, -1.0f), 0x1p-10f);
    if (b == 0) lo = -2.0f;
    if (b == nb - 1) hi = 2.0f;
}

// One thread per brick: shell test of the widened box and brush test with the
// rounding margin d = max(|min|, |max|) * 2^-20 + 2^-120. Writes the active
// bitmask (one ballot word per warp) and counts, per restricted variable, the
// in-shell bricks that pass that variable alone (a selectivity hint).
__global__ void k_classify(const float* __restrict__ bmin, const float* __restrict__ bmax, int n,
                           int nvars, float sc, float rin2, float rout2, BrushArgs brush,
                           uint32_t* __restrict__ active, unsigned* __restrict__ pass_count) {
    int nb = (n + kBrick - 1) / kBrick;
    size_t nbricks = (size_t)nb * nb * nb;
    size_t b = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    bool valid = b < nbricks;
    bool act = false;
    unsigned pass_bits = 0;
    if (valid) {
        int c[3] = {(int)(b % nb), (int)((b / nb) % nb), (int)(b / ((size_t)nb * nb))};
        float nearc[3], farc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float lo, hi;
            brick_box_axis(c[a], nb, sc, lo, hi);
            nearc[a] = (lo > 0.0f) ? lo : ((hi < 0.0f) ? -hi : 0.0f);
            farc[a] = fmaxf(fabsf(lo), fabsf(hi));
        }
        float near2 = dot3_rn(nearc[0], nearc[1], nearc[2], nearc[0], nearc[1], nearc[2]);
        float far2 = dot3_rn(farc[0], farc[1], farc[2], farc[0], farc[1], farc[2]);
        act = (near2 <= rout2) && (far2 >= rin2);
        if (act) {
            bool all = true;
            for (int v = 0; v < nvars; ++v) {
                if (!((brush.mask >> v) & 1u)) continue;
                float mn = bmin[b * nvars + v], mx = bmax[b * nvars + v];
                float m = fmaxf(fabsf(mn), fabsf(mx));
                float d = __fmaf_rn(m, 0x1p-20f, 0x1p-120f);
                bool ok = (__fadd_rn(mx, d) >= brush.lo[v]) && (__fsub_rn(mn, d) <= brush.hi[v]);
                if (ok) pass_bits |= 1u << v;
                all = all && ok;
            }
            act = all;
        }
    }
    unsigned word = __ballot_sync(0xffffffffu, act);
    if (lane == 0 && (b >> 5) < (nbricks + 31) / 32) active[b >> 5] = word;
    for (int v = 0; v < nvars; ++v) {
        unsigned cnt = __popc(__ballot_sync(0xffffffffu, (pass_bits >> v) & 1u));
        if (lane == 0 && cnt) atomicAdd(&pass_count[v], cnt);
    }
}

// Skippable = this brick and its existing 26 neighbours are inactive.
__global__ void k_skippable(const uint32_t* __restrict__ active, int nb, uint32_t* __restrict__ skippable) {
    size_t nbricks = (size_t)nb * nb * nb;
    size_t b = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    bool s = false;
    if (b < nbricks) {
        int x = (int)(b % nb), y = (int)((b / nb) % nb), z = (int)(b / ((size_t)nb * nb));
        s = true;
        for (int dz = -1; dz <= 1 && s; ++dz)
            for (int dy = -1; dy <= 1 && s; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int xx = x + dx, yy = y + dy, zz = z + dz;
                    if (xx < 0 || yy < 0 || zz < 0 || xx >= nb || yy >= nb || zz >= nb) continue;
                    size_t id = ((size_t)zz * nb + yy) * nb + xx;
                    if ((active[id >> 5] >> (id & 31)) & 1u) { s = false; break; }
                }
    }
    unsigned word = __ballot_sync(0xffffffffu, s);
    if (lane == 0 && (b >> 5) < (nbricks + 31) / 32) skippable[b >> 5] = word;
}

// Ordered compaction of the active brick ids: one block of 1024 threads, each
// owning a contiguous run of bitmask words; block-wide exclusive scan of the
// per-thread popcounts gives every thread its output offset.
__global__ void __launch_bounds__(1024) k_compact(const uint32_t* __restrict__ active, size_t nwords,
                                                  size_t nbricks, uint32_t* __restrict__ list,
                                                  uint32_t* __restrict__ n_active) {
    __shared__ unsigned s_sum[1024];
    size_t per = (nwords + blockDim.x - 1) / blockDim.x;
    size_t w0 = threadIdx.x * per, w1 = min(nwords, w0 + per);
    unsigned cnt = 0;
    for (size_t w = w0; w < w1; ++w) cnt += __popc(active[w]);
    s_sum[threadIdx.x] = cnt;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        unsigned add = threadIdx.x >= (unsigned)off ? s_sum[threadIdx.x - off] : 0u;
        __syncthreads();
        s_sum[threadIdx.x] += add;
        __syncthreads();
    }
    unsigned pos = s_sum[threadIdx.x] - cnt;
    if (list) {
        for (size_t w = w0; w < w1; ++w) {
            uint32_t bits = active[w];
            while (bits) {
                int j = __ffs(bits) - 1;
                bits &= bits - 1;
                size_t id = w * 32 + j;
                if (id < nbricks) list[pos++] = (uint32_t)id;
            }
        }
    }
    if (threadIdx.x == blockDim.x - 1 && n_active) *n_active = s_sum[threadIdx.x];
}

inline unsigned blocks_for(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_ingest(const void* src, int src_dtype, void* cells, void* pairs, int dtype, int n,
                          int nvars, cudaStream_t stream) {
    size_t total = (size_t)n * n * n * nvars;
    if (dtype == kF16)
        k_ingest<kF16><<<blocks_for(total, 256), 256, 0, stream>>>(src, src_dtype, cells, pairs, n, total);
    else
        k_ingest<kF32><<<blocks_for(total, 256), 256, 0, stream>>>(src, src_dtype, cells, pairs, n, total);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lod(const void* fine, int n_fine, void* cells, void* pairs, int dtype, int nvars,
                       cudaStream_t stream) {
    size_t m = (size_t)(n_fine + 1) / 2;
    size_t total = m * m * m * nvars;
    if (dtype == kF16)
        k_lod<kF16><<<blocks_for(total, 256), 256, 0, stream>>>(fine, n_fine, cells, pairs, nvars);
    else
        k_lod<kF32><<<blocks_for(total, 256), 256, 0, stream>>>(fine, n_fine, cells, pairs, nvars);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_brick_minmax(const void* cells, int dtype, int n, int nvars, float* bmin, float* bmax,
                                cudaStream_t stream) {
    size_t nb = (size_t)(n + kBrick - 1) / kBrick;
    size_t threads = nb * nb * nb * 32;
    if (dtype == kF16)
        k_brick_minmax<kF16><<<blocks_for(threads, 256), 256, 0, stream>>>(cells, n, nvars, bmin, bmax);
    else
        k_brick_minmax<kF32><<<blocks_for(threads, 256), 256, 0, stream>>>(cells, n, nvars, bmin, bmax);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_classify(const float* bmin, const float* bmax, int n, int nvars, float r_in,
                            float r_out, const BrushArgs& brush, uint32_t* active,
                            uint32_t* skippable, uint32_t* list, uint32_t* n_active,
                            unsigned* pass_count, cudaStream_t stream) {
    int nb = (n + kBrick - 1) / kBrick;
    size_t nbricks = (size_t)nb * nb * nb;
    size_t nwords = (nbricks + 31) / 32;
    cudaError_t e = cudaMemsetAsync(pass_count, 0, sizeof(unsigned) * kMaxVars, stream);
    if (e != cudaSuccess) return e;
    float sc = 2.0f / (float)n;
    float rin2 = r_in * r_in, rout2 = r_out * r_out;
    k_classify<<<blocks_for(nbricks, 256), 256, 0, stream>>>(bmin, bmax, n, nvars, sc, rin2, rout2,
                                                             brush, active, pass_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_skippable<<<blocks_for(nbricks, 256), 256, 0, stream>>>(active, nb, skippable);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_compact<<<1, 1024, 0, stream>>>(active, nwords, nbricks, list, n_active);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace raypc

// Volume preparation kernels: ingest/relayout and level-of-detail mean fused
// with brick min/max, and brush classification of bricks.
//
// Section 2.1 of the paper prepares the data once (levels of detail, derived
// variables); Section 2.2 relies on that preparation not depending on the
// restrictions, so a brush edit only re-runs the (cheap) classification.
#include <algorithm>

#include "common.cuh"

namespace raypc {

namespace {

// Round to the storage dtype (the stored value, as a float).
template <int DT> __device__ __forceinline__ float to_stored(float v);
template <> __device__ __forceinline__ float to_stored<kF32>(float v) { return v; }
template <> __device__ __forceinline__ float to_stored<kF16>(float v) { return __half2float(__float2half_rn(v)); }

struct RowsArgs {
    const void* src;      // ingest: planar source (src_dtype); LOD: planar cells of the finer level;
                          // bricks only: planar cells of this level
    int src_dtype;        // ingest only
    int n_src;            // LOD: edge of the finer level
    void* cells;          // this level, planar
    void* pairs;          // this level, x-pairs
    int n;                // edge of this level
    int nvars;
    float* bmin;          // [nb^3][nvars]
    float* bmax;
    float* sbmin;         // [nsb^3][nvars], sub-bricks of edge kSub
    float* sbmax;
    void* ccells;         // ingest with the next level: its planar cells (edge n / 2) ...
    void* cpairs;         // ... and x-pairs
};

__device__ __forceinline__ void fold(float& mn, float& mx, float a_mn, float a_mx) {
    mn = fminf(mn, a_mn);
    mx = fmaxf(mx, a_mx);
}

// VEC consecutive values of a planar array of element type T (kF32 / kF16)
// starting at element i (aligned to VEC elements when VEC > 1), as floats.
template <int T, int VEC> __device__ __forceinline__ void load_run(const void* base, size_t i, float* out);
template <> __device__ __forceinline__ void load_run<kF32, 1>(const void* base, size_t i, float* out) {
    out[0] = __ldg(reinterpret_cast<const float*>(base) + i);
}
template <> __device__ __forceinline__ void load_run<kF16, 1>(const void* base, size_t i, float* out) {
    out[0] = __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(base) + i)));
}
template <> __device__ __forceinline__ void load_run<kF32, 2>(const void* base, size_t i, float* out) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(base) + i));
    out[0] = a.x; out[1] = a.y;
}
template <> __device__ __forceinline__ void load_run<kF16, 2>(const void* base, size_t i, float* out) {
    const unsigned w = __ldg(reinterpret_cast<const unsigned*>(reinterpret_cast<const __half*>(base) + i));
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
    out[0] = f.x; out[1] = f.y;
}
template <> __device__ __forceinline__ void load_run<kF32, 4>(const void* base, size_t i, float* out) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(base) + i));
    out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
}
template <> __device__ __forceinline__ void load_run<kF16, 4>(const void* base, size_t i, float* out) {
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const __half*>(base) + i));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
template <> __device__ __forceinline__ void load_run<kF32, 8>(const void* base, size_t i, float* out) {
    load_run<kF32, 4>(base, i, out);
    load_run<kF32, 4>(base, i + 4, out + 4);
}
template <> __device__ __forceinline__ void load_run<kF16, 8>(const void* base, size_t i, float* out) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const __half*>(base) + i));
    const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&ws[q]));
        out[2 * q] = f.x;
        out[2 * q + 1] = f.y;
    }
}

// Store VEC stored values (already rounded to DT) of one row run: the cells
// and their x-pairs (c[x], c[x+1]); val[VEC] is the value right of the run.
template <int DT, int VEC>
__device__ __forceinline__ void store_run(void* cells, void* pairs, size_t i, const float* val) {
    if (DT == kF32) {
        float* c = reinterpret_cast<float*>(cells) + i;
        float2* p = reinterpret_cast<float2*>(pairs) + i;
        if (VEC == 4) {
            *reinterpret_cast<float4*>(c) = make_float4(val[0], val[1], val[2], val[3]);
            reinterpret_cast<float4*>(p)[0] = make_float4(val[0], val[1], val[1], val[2]);
            reinterpret_cast<float4*>(p)[1] = make_float4(val[2], val[3], val[3], val[4]);
        } else {
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                c[q] = val[q];
                p[q] = make_float2(val[q], val[q + 1]);
            }
        }
    } else {
        __half h[VEC + 1];
#pragma unroll
        for (int q = 0; q <= VEC; ++q) h[q] = __float2half_rn(val[q]);   // exact: values are stored halves
        __half* c = reinterpret_cast<__half*>(cells) + i;
        __half2* p = reinterpret_cast<__half2*>(pairs) + i;
        if (VEC == 4) {
            __half2 c01 = __halves2half2(h[0], h[1]), c23 = __halves2half2(h[2], h[3]);
            uint2 cw;
            cw.x = *reinterpret_cast<unsigned*>(&c01);
            cw.y = *reinterpret_cast<unsigned*>(&c23);
            *reinterpret_cast<uint2*>(c) = cw;
            __half2 p0 = __halves2half2(h[0], h[1]), p1 = __halves2half2(h[1], h[2]);
            __half2 p2 = __halves2half2(h[2], h[3]), p3 = __halves2half2(h[3], h[4]);
            uint4 pw;
            pw.x = *reinterpret_cast<unsigned*>(&p0);
            pw.y = *reinterpret_cast<unsigned*>(&p1);
            pw.z = *reinterpret_cast<unsigned*>(&p2);
            pw.w = *reinterpret_cast<unsigned*>(&p3);
            *reinterpret_cast<uint4*>(p) = pw;
        } else {
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                c[q] = h[q];
                p[q] = __halves2half2(h[q], h[q + 1]);
            }
        }
    }
}

// Values of columns X .. X+VEC of row (y, z) of variable v of the level being
// produced, rounded to the storage dtype DT; column X+VEC is clamped to n-1.
//   MODE 0 (ingest): the converted source value (source element type SRC).
//   MODE 1 (LOD):    FP32 mean of the 2x2x2 fine cells, fine indices clamped,
//                    ((c000 + c100) + (c010 + c110)) + ((c001 + c101) + (c011 + c111)), x 1/8.
//   MODE 2 (ingest and the next level): as MODE 0; the kernel also forms the next
//                    level's means from the values it produced (n a multiple of 16).
//   MODE 3 (bricks only): the level's own stored cells, for its brick min/max.
// With VEC > 1 the caller guarantees n % VEC == 0 and, for LOD, an even fine edge.
template <int DT, int MODE, int SRC, int VEC>
__device__ __forceinline__ void produce_run(const RowsArgs& A, int X, int y, int z, int v, float* val) {
    const int n = A.n;
    const bool right = X + VEC < n;
    if (MODE != 1) {
        const size_t row = (((size_t)v * n + z) * n + y) * n;
        load_run<SRC, VEC>(A.src, row + X, val);
        load_run<SRC, 1>(A.src, row + (right ? X + VEC : X + VEC - 1), val + VEC);
#pragma unroll
        for (int q = 0; q <= VEC; ++q) val[q] = to_stored<DT>(val[q]);
    } else {
        const int nf = A.n_src;
        const int y0 = 2 * y, y1 = min(y0 + 1, nf - 1), z0 = 2 * z, z1 = min(z0 + 1, nf - 1);
        const size_t plane = (size_t)v * nf * nf * nf;
        const size_t r00 = plane + ((size_t)z0 * nf + y0) * nf, r10 = plane + ((size_t)z0 * nf + y1) * nf;
        const size_t r01 = plane + ((size_t)z1 * nf + y0) * nf, r11 = plane + ((size_t)z1 * nf + y1) * nf;
        // fine columns 2X .. 2X+2VEC+1 (the last two for the right neighbour), clamped
        constexpr int W = 2 * VEC + 2;
        float f00[W], f10[W], f01[W], f11[W];
        const int fx = 2 * X;
        if (VEC > 1) {
            load_run<DT, 2 * VEC>(A.src, r00 + fx, f00);
            load_run<DT, 2 * VEC>(A.src, r10 + fx, f10);
            load_run<DT, 2 * VEC>(A.src, r01 + fx, f01);
            load_run<DT, 2 * VEC>(A.src, r11 + fx, f11);
            const int e0 = right ? fx + 2 * VEC : fx + 2 * VEC - 2;    // even: a 2-run stays in the row
            load_run<DT, 2>(A.src, r00 + e0, f00 + 2 * VEC);
            load_run<DT, 2>(A.src, r10 + e0, f10 + 2 * VEC);
            load_run<DT, 2>(A.src, r01 + e0, f01 + 2 * VEC);
            load_run<DT, 2>(A.src, r11 + e0, f11 + 2 * VEC);
        } else {
            // fine columns of X, then of the right neighbour X+1 (of X itself at the edge)
            const int g = right ? fx + 2 : fx;
            const int cc[4] = {fx, min(fx + 1, nf - 1), g, min(g + 1, nf - 1)};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                load_run<DT, 1>(A.src, r00 + cc[q], f00 + q);
                load_run<DT, 1>(A.src, r10 + cc[q], f10 + q);
                load_run<DT, 1>(A.src, r01 + cc[q], f01 + q);
                load_run<DT, 1>(A.src, r11 + cc[q], f11 + q);
            }
        }
#pragma unroll
        for (int q = 0; q <= VEC; ++q) {
            const int a = 2 * q, b = 2 * q + 1;
            const float s0 = __fadd_rn(__fadd_rn(f00[a], f00[b]), __fadd_rn(f10[a], f10[b]));
            const float s1 = __fadd_rn(__fadd_rn(f01[a], f01[b]), __fadd_rn(f11[a], f11[b]));
            val[q] = to_stored<DT>(__fmul_rn(__fadd_rn(s0, s1), 0.125f));
        }
    }
}

// One block per (brick row (by, bz), variable), threads (t, dz): thread t owns
// the VEC columns X = VEC t .. VEC t + VEC-1 (striding over the level when it
// is wider than the block) of z-slice z = 8bz + dz, dz in 0..8, and also reads
// column X+VEC, the right element of its last pair. Each thread streams the
// (up to) 9 x-rows y in [8by, 8by+8] of its slice, writes the rows it owns
// (dy, dz < 8: cells and x-pairs) and folds every row, apron rows included,
// with the right column, into NaN-ignoring min/max for the two y halves of
// the brick (half 0 is rows 0..4, half 1 rows 4..8; row 4 is in both). The
// slices are folded into the two z halves in shared memory, then lanes are
// reduced with shuffles: 4/VEC lanes make a sub-brick of edge 4 (x in
// 4s..min(4s+4, n-1)), two sub-bricks a brick (x in 8b..min(8b+8, n-1)).
constexpr int kRowCols = 64;                            // column threads per block (blockDim.x)
constexpr int kRowSlices = kBrick + 1;                  // blockDim.y

// The next level's two cells (2 t, 2 t + 1) of one row, from the per-slice sums in
// shared memory, stored with their x-pairs at flat index i (even). The pair of cell
// 2 t + 1 needs cell 2 t + 2: from the neighbouring thread, the cell itself at the
// row's end, or -- at the end of a column chunk -- from the next chunk's first
// thread, which writes that half (`whole` false: only the first half here).
template <int DT>
__device__ __forceinline__ void store_next_level(void* cells, void* pairs, size_t i, float v0, float v1, float r,
                                                 bool whole) {
    if (DT == kF32) {
        float* c = reinterpret_cast<float*>(cells) + i;
        float* p = reinterpret_cast<float*>(pairs) + 2 * i;
        *reinterpret_cast<float2*>(c) = make_float2(v0, v1);
        if (whole) {
            *reinterpret_cast<float4*>(p) = make_float4(v0, v1, v1, r);
        } else {
            *reinterpret_cast<float2*>(p) = make_float2(v0, v1);
            p[2] = v1;
        }
    } else {
        const __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1), hr = __float2half_rn(r);   // exact
        __half2 c01 = __halves2half2(h0, h1), c1r = __halves2half2(h1, hr);
        *reinterpret_cast<__half2*>(reinterpret_cast<__half*>(cells) + i) = c01;
        __half* p = reinterpret_cast<__half*>(pairs) + 2 * i;
        if (whole) {
            uint2 w;
            w.x = *reinterpret_cast<unsigned*>(&c01);
            w.y = *reinterpret_cast<unsigned*>(&c1r);
            *reinterpret_cast<uint2*>(p) = w;
        } else {
            *reinterpret_cast<__half2*>(p) = c01;
            p[2] = h1;
        }
    }
}

template <int DT>
__device__ __forceinline__ void store_pair_second(void* pairs, size_t i, float v) {
    if (DT == kF32) reinterpret_cast<float*>(pairs)[2 * i + 1] = v;
    else reinterpret_cast<__half*>(pairs)[2 * i + 1] = __float2half_rn(v);
}

template <int DT, int MODE, int SRC, int VEC>
__global__ void __launch_bounds__(kRowCols * kRowSlices, 2) k_rows(RowsArgs A) {
    constexpr int G = kSub / VEC;                       // lanes per sub-brick column
    constexpr int kBatch = MODE == 1 ? 1 : 3;          // rows whose loads are issued together
    constexpr int kHalf = kBrick / 2;
    __shared__ float s_half[kRowSlices][4][kRowCols];  // per slice: min, max of y half 0, then of half 1
    // MODE 2: per fine slice and coarse row, the sums over the row pair of the x-pair sums
    __shared__ float s_next[MODE == 2 ? kBrick : 1][kHalf][2][kRowCols];
    const int n = A.n;
    const int nb = (n + kBrick - 1) / kBrick;
    const int nsb = (n + kSub - 1) / kSub;
    const int ncol = (n + VEC - 1) / VEC;
    const int by = blockIdx.x % nb, bz = blockIdx.x / nb, v = blockIdx.y;
    const int dz = threadIdx.y, tx = threadIdx.x;
    const int z = bz * kBrick + dz;
    const float qnan = __int_as_float(0x7fffffff);
    for (int c0 = 0; c0 < ncol; c0 += blockDim.x) {
        const int t = c0 + tx;
        const bool valid = t < ncol && z < n;
        const int X = t * VEC;
        float ymn[2] = {qnan, qnan}, ymx[2] = {qnan, qnan};
        float even0 = 0.0f, even1 = 0.0f;                // MODE 2: x-pair sums of the even row
#pragma unroll
        for (int dy0 = 0; dy0 <= kBrick; dy0 += kBatch) {
            float val[kBatch][VEC + 1];
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const int y = by * kBrick + dy0 + j;
                if (valid && dy0 + j <= kBrick && y < n) produce_run<DT, MODE, SRC, VEC>(A, X, y, z, v, val[j]);
            }
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const int dy = dy0 + j;
                const int y = by * kBrick + dy;
                if (!valid || dy > kBrick || y >= n) continue;
                float rmn = val[j][0], rmx = val[j][0];
#pragma unroll
                for (int q = 1; q <= VEC; ++q) fold(rmn, rmx, val[j][q], val[j][q]);
                if (dy <= kSub) fold(ymn[0], ymx[0], rmn, rmx);
                if (dy >= kSub) fold(ymn[1], ymx[1], rmn, rmx);
                if (MODE != 3 && dy < kBrick && dz < kBrick)
                    store_run<DT, VEC>(A.cells, A.pairs, (((size_t)v * n + z) * n + y) * n + X, val[j]);
                if (MODE == 2 && dy < kBrick && dz < kBrick) {
                    // the next level's mean, in its order: (c000 + c100) + (c010 + c110) per fine slice
                    const float p0 = __fadd_rn(val[j][0], val[j][1]), p1 = __fadd_rn(val[j][2], val[j][3]);
                    if ((dy & 1) == 0) {
                        even0 = p0;
                        even1 = p1;
                    } else {
                        s_next[MODE == 2 ? dz : 0][dy >> 1][0][tx] = __fadd_rn(even0, p0);
                        s_next[MODE == 2 ? dz : 0][dy >> 1][1][tx] = __fadd_rn(even1, p1);
                    }
                }
            }
        }
        s_half[dz][0][tx] = ymn[0];
        s_half[dz][1][tx] = ymx[0];
        s_half[dz][2][tx] = ymn[1];
        s_half[dz][3][tx] = ymx[1];
        __syncthreads();
        if (dz == 0) {
            // (y half, z half) h = j + 2i: slices 0..4 make z half 0, slices 4..8 z half 1
            float mn[4] = {qnan, qnan, qnan, qnan}, mx[4] = {qnan, qnan, qnan, qnan};
#pragma unroll
            for (int sl = 0; sl < kRowSlices; ++sl) {
                const float a0 = s_half[sl][0][tx], b0 = s_half[sl][1][tx];
                const float a1 = s_half[sl][2][tx], b1 = s_half[sl][3][tx];
                if (sl <= kSub) { fold(mn[0], mx[0], a0, b0); fold(mn[1], mx[1], a1, b1); }
                if (sl >= kSub) { fold(mn[2], mx[2], a0, b0); fold(mn[3], mx[3], a1, b1); }
            }
            // sub-bricks: reduce over the G lanes of a sub-brick column
#pragma unroll
            for (int m = 1; m < G; m <<= 1)
#pragma unroll
                for (int h = 0; h < 4; ++h)
                    fold(mn[h], mx[h], __shfl_xor_sync(0xffffffffu, mn[h], m), __shfl_xor_sync(0xffffffffu, mx[h], m));
            const bool tcol = t < ncol;
            const int sx = t / G;
            if (tcol && t % G == 0) {
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int sy = 2 * by + (h & 1), sz = 2 * bz + (h >> 1);
                    if (sy < nsb && sz < nsb && sx < nsb) {
                        const size_t sb = ((size_t)sz * nsb + sy) * nsb + sx;
                        A.sbmin[sb * A.nvars + v] = mn[h];
                        A.sbmax[sb * A.nvars + v] = mx[h];
                    }
                }
            }
            // bricks: all four halves of two neighbouring sub-brick columns
            float bmn = mn[0], bmx = mx[0];
#pragma unroll
            for (int h = 1; h < 4; ++h) fold(bmn, bmx, mn[h], mx[h]);
            fold(bmn, bmx, __shfl_xor_sync(0xffffffffu, bmn, G), __shfl_xor_sync(0xffffffffu, bmx, G));
            const int bx = t / (2 * G);
            if (tcol && t % (2 * G) == 0 && bx < nb) {
                const size_t b = ((size_t)bz * nb + by) * nb + bx;
                A.bmin[b * A.nvars + v] = bmn;
                A.bmax[b * A.nvars + v] = bmx;
            }
        }
        if (MODE == 2 && dz < kHalf && t < ncol) {
            // the next level's cells 2t, 2t+1 of its rows 4 by .. 4 by + 3 in slice 4 bz + dz:
            // ((fine slice 2 dz) + (fine slice 2 dz + 1)) / 8
            const int m = n >> 1;
            const bool row_end = t + 1 >= ncol, chunk_end = tx + 1 >= (int)blockDim.x;
            const int s0 = MODE == 2 ? 2 * dz : 0, s1 = MODE == 2 ? 2 * dz + 1 : 0;
#pragma unroll
            for (int k = 0; k < kHalf; ++k) {
                const float v0 = to_stored<DT>(__fmul_rn(__fadd_rn(s_next[s0][k][0][tx], s_next[s1][k][0][tx]), 0.125f));
                const float v1 = to_stored<DT>(__fmul_rn(__fadd_rn(s_next[s0][k][1][tx], s_next[s1][k][1][tx]), 0.125f));
                float r = v1;                            // the row's last cell pairs with itself
                if (!row_end && !chunk_end)
                    r = to_stored<DT>(__fmul_rn(__fadd_rn(s_next[s0][k][0][tx + 1], s_next[s1][k][0][tx + 1]), 0.125f));
                const size_t i = (((size_t)v * m + (size_t)(bz * kHalf + dz)) * m + (size_t)(by * kHalf + k)) * m + 2 * t;
                store_next_level<DT>(A.ccells, A.cpairs, i, v0, v1, r, row_end || !chunk_end);
                if (tx == 0 && t > 0) store_pair_second<DT>(A.cpairs, i - 1, v0);   // the previous chunk's last pair
            }
        }
        __syncthreads();                                 // s_half is rewritten by the next column chunk
    }
}

// Locate the level of a flat brick index over all levels (<= 3 levels).
__device__ __forceinline__ int level_of(const ClassifyArgs& C, size_t g, size_t& b) {
    int l = 0;
    while (l + 1 < C.nlev && g >= C.lv[l + 1].first) ++l;
    b = g - C.lv[l].first;
    return l;
}

// One thread per brick of every entry (8^3 bricks and 4^3 sub-bricks of every
// level): shell test of the widened box and brush test with the rounding
// margin d = max(|min|, |max|) * 2^-20 + 2^-120. Writes the active bitmask
// (one ballot word per warp; entry ranges start on multiples of 32) and, for
// the 8^3 bricks, counts per restricted variable the in-shell bricks that pass
// that variable alone (a selectivity hint for the render).
__global__ void k_classify(ClassifyArgs C) {
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    size_t b = 0;
    const int l = level_of(C, g, b);
    const ClassifyLevel& L = C.lv[l];
    const int nb = (L.n + L.bs - 1) / L.bs;
    const size_t nbricks = (size_t)nb * nb * nb;
    const bool in_range = g < C.total;
    const bool valid = in_range && b < nbricks;
    bool act = false;
    unsigned pass_bits = 0;
    if (valid)
        act = classify_brick(b, nb, L.bs, L.sc, C.rin2, C.rout2, C.brush, C.nvars, L.bmin, L.bmax, pass_bits);
    const unsigned word = __ballot_sync(0xffffffffu, act);
    if (lane == 0 && in_range && b < ((nbricks + 31) & ~(size_t)31)) L.active[b >> 5] = word;
    if (L.alist && word) {                      // uniform per warp: entry ranges are warp-aligned
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(L.acount, (unsigned)__popc(word));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (act) L.alist[base + __popc(word & ((1u << lane) - 1u))] = (uint32_t)b;
    }
    if (L.pass_count == nullptr) return;
    for (int v = 0; v < C.nvars; ++v) {
        const unsigned cnt = __popc(__ballot_sync(0xffffffffu, (pass_bits >> v) & 1u));
        if (lane == 0 && cnt) atomicAdd(&L.pass_count[v], cnt);
    }
}

// Skippable = this 8^3 brick and its existing 26 neighbours are inactive.
__global__ void k_skippable(ClassifyArgs C) {
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    size_t b = 0;
    const int l = level_of(C, g, b);
    const ClassifyLevel& L = C.lv[l];
    const int nb = (L.n + kBrick - 1) / kBrick;
    const size_t nbricks = (size_t)nb * nb * nb;
    const bool in_range = g < C.total_brick;
    const bool valid = in_range && b < nbricks;
    const bool s = valid && skippable_brick(b, nb, L.active);
    const unsigned word = __ballot_sync(0xffffffffu, s);
    if (lane == 0 && in_range && b < ((nbricks + 31) & ~(size_t)31)) L.skippable[b >> 5] = word;
}

// Ordered compaction of the active 8^3 brick ids, one block of 1024 threads per
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

// Cell classes (see CellClassArgs) of the cells of the active sub-bricks only
// (the render consults a cell's class only for samples in an active
// sub-brick): one warp per listed sub-brick (see cell_classes_of_subbrick).
template <int DT>
__global__ void __launch_bounds__(32 * kCellWarps) k_cell_classes(const void* __restrict__ pairs, int n,
                                                                 const uint32_t* __restrict__ slist,
                                                                 const uint32_t* __restrict__ scount,
                                                                 uint16_t* __restrict__ out, CellVars R) {
    const int lane = threadIdx.x & 31;
    const int nsb = (n + kSub - 1) / kSub;
    const unsigned count = *scount;
    for (unsigned i = blockIdx.x * kCellWarps + (threadIdx.x >> 5); i < count; i += gridDim.x * kCellWarps)
        cell_classes_of_subbrick<DT>(pairs, n, nsb, __ldg(slist + i), lane, R, out);
}

inline unsigned blocks_for(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <int DT, int MODE, int SRC, int VEC>
void launch_rows_t(const RowsArgs& a, dim3 grid, cudaStream_t stream) {
    const int ncol = (a.n + VEC - 1) / VEC;
    // one thread per column run up to kRowCols (narrow levels use narrow blocks), per z-slice
    const dim3 block(min(kRowCols, max(32, (ncol + 31) / 32 * 32)), kRowSlices);
    k_rows<DT, MODE, SRC, VEC><<<grid, block, 0, stream>>>(a);
}

template <int MODE>
cudaError_t launch_rows(const RowsArgs& a, int dtype, cudaStream_t stream) {
    if (a.n < 2 || a.n > kMaxRowsEdge) return cudaErrorInvalidValue;
    const int nb = (a.n + kBrick - 1) / kBrick;
    dim3 grid((unsigned)(nb * nb), (unsigned)a.nvars);
    // 4-column runs when every run is aligned -- n % 4 == 0, a 16-byte aligned
    // source (ingest) or an even fine edge (LOD; n % 4 == 0 makes it 8k) -- and
    // the level is wide enough to fill a warp with runs.
    bool vec = a.n % 4 == 0 && a.n >= 128;
    if (MODE == 1) vec = vec && a.n_src == 2 * a.n;
    else vec = vec && ((uintptr_t)a.src % 16 == 0);
    if (MODE == 2) {
        // the fused next level needs 4-column runs and whole bricks of both levels
        if (!vec || a.n % 16 != 0 || !a.ccells || !a.cpairs) return cudaErrorInvalidValue;
        const bool s16 = a.src_dtype == kF16;
        if (dtype == kF16) { if (s16) launch_rows_t<kF16, 2, kF16, 4>(a, grid, stream); else launch_rows_t<kF16, 2, kF32, 4>(a, grid, stream); }
        else               { if (s16) launch_rows_t<kF32, 2, kF16, 4>(a, grid, stream); else launch_rows_t<kF32, 2, kF32, 4>(a, grid, stream); }
    } else if (MODE == 3) {
        if (dtype == kF16) { if (vec) launch_rows_t<kF16, 3, kF16, 4>(a, grid, stream); else launch_rows_t<kF16, 3, kF16, 1>(a, grid, stream); }
        else               { if (vec) launch_rows_t<kF32, 3, kF32, 4>(a, grid, stream); else launch_rows_t<kF32, 3, kF32, 1>(a, grid, stream); }
    } else if (MODE == 0) {
        const bool s16 = a.src_dtype == kF16;
        if (dtype == kF16) {
            if (vec) { if (s16) launch_rows_t<kF16, 0, kF16, 4>(a, grid, stream); else launch_rows_t<kF16, 0, kF32, 4>(a, grid, stream); }
            else     { if (s16) launch_rows_t<kF16, 0, kF16, 1>(a, grid, stream); else launch_rows_t<kF16, 0, kF32, 1>(a, grid, stream); }
        } else {
            if (vec) { if (s16) launch_rows_t<kF32, 0, kF16, 4>(a, grid, stream); else launch_rows_t<kF32, 0, kF32, 4>(a, grid, stream); }
            else     { if (s16) launch_rows_t<kF32, 0, kF16, 1>(a, grid, stream); else launch_rows_t<kF32, 0, kF32, 1>(a, grid, stream); }
        }
    } else {
        if (dtype == kF16) { if (vec) launch_rows_t<kF16, 1, kF16, 4>(a, grid, stream); else launch_rows_t<kF16, 1, kF16, 1>(a, grid, stream); }
        else               { if (vec) launch_rows_t<kF32, 1, kF32, 4>(a, grid, stream); else launch_rows_t<kF32, 1, kF32, 1>(a, grid, stream); }
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ingest(const void* src, int src_dtype, void* cells, void* pairs, int dtype, int n,
                          int nvars, float* bmin, float* bmax, float* sbmin, float* sbmax,
                          cudaStream_t stream) {
    RowsArgs a{};
    a.src = src;
    a.src_dtype = src_dtype;
    a.cells = cells;
    a.pairs = pairs;
    a.n = n;
    a.nvars = nvars;
    a.bmin = bmin;
    a.bmax = bmax;
    a.sbmin = sbmin;
    a.sbmax = sbmax;
    return launch_rows<0>(a, dtype, stream);
}

bool ingest_next_level_fits(const void* src, int n) {
    return n % 16 == 0 && n >= 128 && n <= kMaxRowsEdge && (uintptr_t)src % 16 == 0;
}

cudaError_t launch_ingest_next_level(const void* src, int src_dtype, void* cells, void* pairs, int dtype, int n,
                                     int nvars, float* bmin, float* bmax, float* sbmin, float* sbmax,
                                     void* next_cells, void* next_pairs, cudaStream_t stream) {
    RowsArgs a{};
    a.src = src;
    a.src_dtype = src_dtype;
    a.cells = cells;
    a.pairs = pairs;
    a.n = n;
    a.nvars = nvars;
    a.bmin = bmin;
    a.bmax = bmax;
    a.sbmin = sbmin;
    a.sbmax = sbmax;
    a.ccells = next_cells;
    a.cpairs = next_pairs;
    return launch_rows<2>(a, dtype, stream);
}

cudaError_t launch_level_bricks(const void* cells, int dtype, int n, int nvars, float* bmin, float* bmax,
                                float* sbmin, float* sbmax, cudaStream_t stream) {
    RowsArgs a{};
    a.src = cells;
    a.src_dtype = dtype;
    a.n = n;
    a.nvars = nvars;
    a.bmin = bmin;
    a.bmax = bmax;
    a.sbmin = sbmin;
    a.sbmax = sbmax;
    return launch_rows<3>(a, dtype, stream);
}

cudaError_t launch_lod(const void* fine, int n_fine, void* cells, void* pairs, int dtype, int nvars,
                       float* bmin, float* bmax, float* sbmin, float* sbmax, cudaStream_t stream) {
    RowsArgs a{};
    a.src = fine;
    a.n_src = n_fine;
    a.cells = cells;
    a.pairs = pairs;
    a.n = (n_fine + 1) / 2;
    a.nvars = nvars;
    a.bmin = bmin;
    a.bmax = bmax;
    a.sbmin = sbmin;
    a.sbmax = sbmax;
    return launch_rows<1>(a, dtype, stream);
}

cudaError_t launch_cell_classes(const CellClassArgs& a, int dtype, cudaStream_t stream) {
    if (a.n < 2 || !a.slist || !a.scount) return cudaErrorInvalidValue;
    CellVars R;
    cell_vars_of(a.brush, a.nvars, R);
    // grid fixed on the host (the list length is on the device): enough warps
    // for every listed sub-brick of a small level, a few waves for a large one
    const size_t nsb = (size_t)((a.n + kSub - 1) / kSub);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned blocks = (unsigned)std::min<size_t>(blocks_for(nsb * nsb * nsb, kCellWarps), (size_t)sms * 16);
    if (dtype == kF16) k_cell_classes<kF16><<<blocks, 32 * kCellWarps, 0, stream>>>(a.pairs, a.n, a.slist, a.scount, a.out, R);
    else k_cell_classes<kF32><<<blocks, 32 * kCellWarps, 0, stream>>>(a.pairs, a.n, a.slist, a.scount, a.out, R);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_classify(ClassifyArgs& c, cudaStream_t stream) {
    size_t total = 0;
    for (int l = 0; l < c.nlev; ++l) {
        ClassifyLevel& L = c.lv[l];
        if (L.bs != (l < c.nbrick ? kBrick : kSub)) return cudaErrorInvalidValue;
        const int nb = (L.n + L.bs - 1) / L.bs;
        L.first = total;
        L.sc = 2.0f / (float)L.n;
        total += ((size_t)nb * nb * nb + 31) / 32 * 32;      // entry ranges start on warp boundaries
        if (l + 1 == c.nbrick) c.total_brick = total;
        if (L.pass_count) {
            cudaError_t e = cudaMemsetAsync(L.pass_count, 0, sizeof(unsigned) * kMaxVars, stream);
            if (e != cudaSuccess) return e;
        }
        if (L.alist) {
            cudaError_t e = cudaMemsetAsync(L.acount, 0, sizeof(uint32_t), stream);
            if (e != cudaSuccess) return e;
        }
    }
    c.total = total;
    k_classify<<<blocks_for(total, 256), 256, 0, stream>>>(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (c.nbrick == 0) {             // sub-bricks only: no skippable bits, no brick list
        count_launches(1);
        return cudaSuccess;
    }
    k_skippable<<<blocks_for(c.total_brick, 256), 256, 0, stream>>>(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_compact<<<c.nbrick, 1024, 0, stream>>>(c);
    count_launches(3);
    return cudaGetLastError();
}

namespace {

// One thread per brick (entries 0..nbricks-1, padded to whole words) and per
// sub-brick (the entries after them): activity AND TF visibility
// (tf_range_visible). A brick's range holds its sub-bricks' ranges, so an
// invisible brick has only invisible sub-bricks.
__global__ void __launch_bounds__(256) k_tf_visibility(TfVisArgs A) {
    __shared__ int s_pre[kTF + 1];             // s_pre[j] = entries < j with sigma > 0
    if (threadIdx.x < 32) {
        int run = 0;
        for (int base = 0; base < kTF; base += 32) {
            const bool nz = A.tf[base + threadIdx.x].w > 0.0f;
            const unsigned b = __ballot_sync(0xffffffffu, nz);
            s_pre[base + threadIdx.x] = run + __popc(b & ((1u << threadIdx.x) - 1u));
            run += __popc(b);
        }
        if (threadIdx.x == 0) s_pre[kTF] = run;
    }
    __syncthreads();
    const size_t nbr = (size_t)A.nb * A.nb * A.nb, nsub = (size_t)A.nsb * A.nsb * A.nsb;
    const size_t nbr_pad = (nbr + 31) & ~(size_t)31;
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool is_sub = g >= nbr_pad;
    const size_t b = is_sub ? g - nbr_pad : g;
    const size_t cnt = is_sub ? nsub : nbr;
    bool bit = false;
    if (b < cnt) {
        const uint32_t* act = is_sub ? A.sactive : A.active;
        bit = (act[b >> 5] >> (b & 31)) & 1u;
        if (bit) {
            const float mn = (is_sub ? A.sbmin : A.bmin)[b * A.nvars + A.color_var];
            const float mx = (is_sub ? A.sbmax : A.bmax)[b * A.nvars + A.color_var];
            bit = tf_range_visible(mn, mx, s_pre, A.tf_lo, A.tf_scale);
        }
    }
    const unsigned word = __ballot_sync(0xffffffffu, bit);
    if ((threadIdx.x & 31) == 0 && b < ((cnt + 31) & ~(size_t)31)) (is_sub ? A.out_sactive : A.out_active)[b >> 5] = word;
}

}  // namespace

// Empty-space distance of the 4^3 sub-bricks: the Chebyshev distance, in
// sub-bricks, to the nearest active one, capped at kDistCap (0: active). The L-inf
// distance transform is separable: d(p) = min over qz of max(|dz|, min over qy of
// max(|dy|, min over active qx of |dx|)), each 1D pass a window of +-kDistCap.
// pass 0: x from the activity bits into a; 1: y from a into b; 2: z from b into a.
// One sub-brick id < nsb^3 of one pass.
__device__ __forceinline__ uint8_t subbrick_distance_at(const uint32_t* __restrict__ act, int nsb, int pass,
                                                      const uint8_t* __restrict__ in, size_t id) {
    const int x = (int)(id % nsb), y = (int)((id / nsb) % nsb), z = (int)(id / ((size_t)nsb * nsb));
    int d = kDistCap;
    if (pass == 0) {
        for (int o = -kDistCap; o <= kDistCap; ++o) {
            const int xx = x + o;
            if (xx < 0 || xx >= nsb) continue;
            const size_t q = id - x + xx;
            if ((__ldg(act + (q >> 5)) >> (q & 31)) & 1u) d = min(d, abs(o));
        }
    } else {
        const int c = pass == 1 ? y : z;
        const size_t stride = pass == 1 ? (size_t)nsb : (size_t)nsb * nsb;
        for (int o = -kDistCap; o <= kDistCap; ++o) {
            const int cc = c + o;
            if (cc < 0 || cc >= nsb) continue;
            d = min(d, max(abs(o), (int)__ldg(in + (size_t)((long long)id + (long long)o * (long long)stride))));
        }
    }
    return (uint8_t)d;
}

__global__ void __launch_bounds__(256) k_subbrick_distance(const uint32_t* __restrict__ act, int nsb, int pass,
                                                           const uint8_t* __restrict__ in, uint8_t* __restrict__ out) {
    const size_t total = (size_t)nsb * nsb * nsb;
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= total) return;
    out[id] = subbrick_distance_at(act, nsb, pass, in, id);
}

// Every view of a batch: the threads walk the views' concatenated distance ranges (a
// warp's 32 consecutive flat indices always belong to one view); pass 0 writes the
// view's distance buffer, 1 its scratch, 2 the distance buffer again.
__global__ void __launch_bounds__(256) k_subbrick_distance_views(const BatchHeader* __restrict__ hdr,
                                                                 const BatchView* __restrict__ views, int pass) {
    const unsigned long long total = hdr->dist_total;
    const int nviews = hdr->nviews;
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const unsigned long long g0 = g - lane;
        int lo = 0, hi = nviews - 1;                 // the last view whose range starts at or before g0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (views[mid].dist_begin <= g0) lo = mid; else hi = mid - 1;
        }
        const BatchView& V = views[lo];
        const int nsb = V.a.lv.nsb;
        const size_t id = (size_t)(g - V.dist_begin);
        if (id >= (size_t)nsb * nsb * nsb) continue;   // the padding of the view's range
        uint8_t* dist = const_cast<uint8_t*>(V.a.lv.sdist);
        const uint8_t* in = pass == 1 ? dist : V.stmp;
        uint8_t* out = pass == 1 ? V.stmp : dist;
        out[id] = subbrick_distance_at(V.a.lv.sactive, nsb, pass, in, id);
    }
}

cudaError_t launch_subbrick_distance(const uint32_t* sactive, int nsb, uint8_t* dist, uint8_t* tmp,
                                     cudaStream_t stream) {
    const size_t total = (size_t)nsb * nsb * nsb;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    k_subbrick_distance<<<blocks, 256, 0, stream>>>(sactive, nsb, 0, nullptr, dist);
    k_subbrick_distance<<<blocks, 256, 0, stream>>>(sactive, nsb, 1, dist, tmp);
    k_subbrick_distance<<<blocks, 256, 0, stream>>>(sactive, nsb, 2, tmp, dist);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_subbrick_distance_views(const BatchHeader* hdr, const BatchView* views, unsigned blocks,
                                           cudaStream_t stream) {
    for (int pass = 0; pass < 3; ++pass) {
        k_subbrick_distance_views<<<blocks, 256, 0, stream>>>(hdr, views, pass);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_tf_visibility(const TfVisArgs& a, cudaStream_t stream) {
    const size_t nbr = (size_t)a.nb * a.nb * a.nb, nsub = (size_t)a.nsb * a.nsb * a.nsb;
    const size_t total = ((nbr + 31) & ~(size_t)31) + nsub;
    k_tf_visibility<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace raypc

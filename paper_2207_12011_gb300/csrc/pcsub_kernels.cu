// PC line data (Section 2.1: the parallel-coordinates plot draws the polylines
// of a random subsample of at most 100 000 cells).
//
// Every in-shell cell c (linear index (z*n + y)*n + x; the integer shell test
// of the histograms) has the 64-bit key splitmix64_at(seed * 2^32 + 2^32 - 1, c).
// Keys are distinct: the output function is a bijection and the state
// increment is odd. The subsample is the m = min(k, N) cells with the smallest
// keys, written in increasing c with their PC axis values and a brush flag.
//
// Exact radix select, 12 bits per round, with no field data read: a round
// histograms the next 12-bit digit of the keys that share the prefix resolved
// so far (keys are recomputed from the cell index), then one block finds the
// digit whose bucket holds the m-th smallest key. When the cells still needed
// fill that bucket exactly, the select is done: the subsample is every cell
// whose key's resolved top bits are <= the prefix. Distinct keys guarantee
// this by 64 bits, i.e. within six rounds; rounds after the select is done
// return at once. An ordered compaction follows: warps own contiguous row
// segments, count their selected cells, one block scans the counts, and each
// warp writes its cells' indices in cell order from its segment's offset; one
// thread per line then gathers the line's axis values and brush flag.
#include "common.cuh"

namespace raypc {

namespace {

constexpr int kDigitBits = 12;
constexpr int kDigits = 1 << kDigitBits;
constexpr int kRounds = 6;             // 6 x 12 >= 64 bits
constexpr int kSubThreads = 256;

struct SubState {
    unsigned long long prefix;         // resolved top bits of the m-th smallest key
    unsigned long long need;           // cells still to take among keys sharing the prefix
    int nbits;                         // resolved bits, 0..64
    int done;                          // selection final: top nbits bits <= prefix (nbits 0: all)
    unsigned long long hist[kDigits];
    unsigned seg_cnt[kSubMaxSegments];   // selected cells per compaction segment
    unsigned seg_off[kSubMaxSegments];   // their exclusive prefix sums
};

// Largest integer m >= 0 with m * m <= a (0 <= a < 2^31).
__device__ __forceinline__ int isqrt_floor_dev(int a) {
    int m = (int)sqrtf((float)a);
    while ((long long)m * m > a) --m;
    while ((long long)(m + 1) * (m + 1) <= a) ++m;
    return m;
}

// x range [xa, xb] of row (y, z) whose cells can lie inside the outer sphere;
// false if none can. syz = dy^2 + dz^2 of the row.
__device__ __forceinline__ bool row_range(const SubsampleArgs& A, long long r, int& xa, int& xb, int& syz) {
    const int n = A.n;
    const int y = (int)(r % n), z = (int)(r / n);
    const int dy = 2 * y + 1 - n, dz = 2 * z + 1 - n;
    syz = dy * dy + dz * dz;
    if (syz > A.s_out) return false;
    const int m = isqrt_floor_dev(A.s_out - syz);
    xa = max(0, (n - m) / 2);
    xb = min(n - 1, (n - 1 + m) / 2);
    return xa <= xb;
}

__device__ __forceinline__ bool in_shell(const SubsampleArgs& A, int x, int syz) {
    const int dx = 2 * x + 1 - A.n;
    const int s = dx * dx + syz;
    return s >= A.s_in && s <= A.s_out;
}

__device__ __forceinline__ bool selected(unsigned long long key, int nbits, unsigned long long prefix) {
    return nbits == 0 || (key >> (64 - nbits)) <= prefix;
}

__global__ void k_sub_init(SubState* S, unsigned long long m, int all) {
    for (int i = threadIdx.x; i < kDigits; i += blockDim.x) S->hist[i] = 0ull;
    if (threadIdx.x == 0) {
        S->prefix = 0ull;
        S->need = m;
        S->nbits = 0;
        S->done = all;
    }
}

// One round: histogram of the next digit of the keys that share the prefix.
__global__ void __launch_bounds__(kSubThreads) k_sub_hist(SubsampleArgs A, SubState* S) {
    __shared__ unsigned h[kDigits];
    if (S->done) return;
    const int nbits = S->nbits;
    const unsigned long long prefix = S->prefix;
    const int width = min(kDigitBits, 64 - nbits);
    const int shift = 64 - nbits - width;
    const unsigned dmask = (1u << width) - 1u;
    for (int i = threadIdx.x; i < kDigits; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long rows = (long long)A.n * A.n;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = gwarp; r < rows; r += nwarps) {
        int xa, xb, syz;
        if (!row_range(A, r, xa, xb, syz)) continue;
        for (int x = xa + lane; x <= xb; x += 32) {
            if (!in_shell(A, x, syz)) continue;
            const unsigned long long key = splitmix64_at(A.key, (unsigned long long)r * A.n + x);
            if (nbits != 0 && (key >> (64 - nbits)) != prefix) continue;
            atomicAdd(&h[(unsigned)(key >> shift) & dmask], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kDigits; i += blockDim.x)
        if (h[i]) atomicAdd(&S->hist[i], (unsigned long long)h[i]);
}

// One block of 1024 threads: the digit whose bucket holds the next needed key.
__global__ void __launch_bounds__(1024) k_sub_pick(SubState* S) {
    __shared__ unsigned long long s_sum[1024];
    if (S->done) return;
    constexpr int kPer = kDigits / 1024;
    const int t = threadIdx.x;
    // the state is read before the first barrier: the owner thread rewrites it after the last one
    const int width = min(kDigitBits, 64 - S->nbits);
    const unsigned long long need = S->need;
    unsigned long long loc[kPer], tot = 0ull;
#pragma unroll
    for (int i = 0; i < kPer; ++i) { loc[i] = S->hist[t * kPer + i]; tot += loc[i]; }
    s_sum[t] = tot;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned long long add = t >= off ? s_sum[t - off] : 0ull;
        __syncthreads();
        s_sum[t] += add;
        __syncthreads();
    }
    unsigned long long before = s_sum[t] - tot;
    // exactly one thread owns the digit with before < need <= before + count
    if (before < need && need <= s_sum[t]) {
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            if (need <= before + loc[i]) {
                const unsigned long long rest = need - before;
                S->prefix = (S->nbits == 0 ? 0ull : (S->prefix << width)) | (unsigned long long)(t * kPer + i);
                S->nbits += width;
                S->need = rest;
                if (rest == loc[i]) S->done = 1;
                break;
            }
            before += loc[i];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPer; ++i) S->hist[t * kPer + i] = 0ull;
}

// Rows [r0, r1) of compaction segment g (one warp per segment, segments in row order).
__device__ __forceinline__ void segment_rows(const SubsampleArgs& A, long long g, int nseg, long long& r0, long long& r1) {
    const long long rows = (long long)A.n * A.n;
    const long long per = (rows + nseg - 1) / nseg;
    r0 = min(rows, g * per);
    r1 = min(rows, r0 + per);
}

__global__ void __launch_bounds__(kSubThreads) k_sub_count(SubsampleArgs A, SubState* S, int nseg) {
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= nseg) return;                                     // whole warps
    const int lane = threadIdx.x & 31;
    const int nbits = S->nbits;
    const unsigned long long prefix = S->prefix;
    long long r0, r1;
    segment_rows(A, g, nseg, r0, r1);
    unsigned cnt = 0;
    for (long long r = r0; r < r1; ++r) {
        int xa, xb, syz;
        if (!row_range(A, r, xa, xb, syz)) continue;
        for (int x = xa + lane; x <= xb; x += 32)
            if (in_shell(A, x, syz) && selected(splitmix64_at(A.key, (unsigned long long)r * A.n + x), nbits, prefix))
                ++cnt;
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) S->seg_cnt[g] = cnt;
}

// One block of 1024 threads: exclusive scan of the segment counts (m < 2^31).
__global__ void __launch_bounds__(1024) k_sub_scan(SubState* S, int nseg) {
    __shared__ unsigned s_sum[1024];
    constexpr int kPer = kSubMaxSegments / 1024;
    const int t = threadIdx.x;
    unsigned loc[kPer], tot = 0u;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int g = t * kPer + i;
        loc[i] = g < nseg ? S->seg_cnt[g] : 0u;
        tot += loc[i];
    }
    s_sum[t] = tot;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned add = t >= off ? s_sum[t - off] : 0u;
        __syncthreads();
        s_sum[t] += add;
        __syncthreads();
    }
    unsigned run = s_sum[t] - tot;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int g = t * kPer + i;
        if (g < nseg) S->seg_off[g] = run;
        run += loc[i];
    }
}

__global__ void __launch_bounds__(kSubThreads) k_sub_write(SubsampleArgs A, SubState* S, int nseg) {
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= nseg) return;                                     // whole warps
    const int lane = threadIdx.x & 31;
    const int nbits = S->nbits;
    const unsigned long long prefix = S->prefix;
    unsigned long long base = S->seg_off[g];
    long long r0, r1;
    segment_rows(A, g, nseg, r0, r1);
    const int n = A.n;
    for (long long r = r0; r < r1; ++r) {
        int xa, xb, syz;
        if (!row_range(A, r, xa, xb, syz)) continue;        // uniform over the warp
        for (int x0 = xa; x0 <= xb; x0 += 32) {
            const int x = x0 + lane;
            const unsigned long long c = (unsigned long long)r * n + x;
            const bool sel = x <= xb && in_shell(A, x, syz) && selected(splitmix64_at(A.key, c), nbits, prefix);
            const unsigned ball = __ballot_sync(0xffffffffu, sel);
            const unsigned long long pos = base + __popc(ball & ((1u << lane) - 1u));
            base += __popc(ball);
            if (sel && pos < A.m) A.out_cells[pos] = (long long)c;   // the select yields exactly m cells
        }
    }
}

// One thread per written line: PC axis values and the brush flag of its cell.
template <int DT>
__global__ void __launch_bounds__(kSubThreads) k_sub_gather(SubsampleArgs A) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.m) return;
    const int n = A.n;
    const size_t plane = (size_t)n * n * n;
    const unsigned long long c = (unsigned long long)A.out_cells[i];
    if (c >= (unsigned long long)plane) return;              // written by k_sub_write; never out of range
    const int x = (int)(c % n), y = (int)((c / n) % n), z = (int)(c / ((unsigned long long)n * n));
    float cx = 0.0f, cy = 0.0f, cz = 0.0f, r2 = 0.0f;
    if (A.use_pos) {
        cx = cell_centre_rn(x, n);
        cy = cell_centre_rn(y, n);
        cz = cell_centre_rn(z, n);
        r2 = dot3_rn(cx, cy, cz, cx, cy, cz);
    }
    for (int a = 0; a < A.naxes; ++a) {
        const int av = A.axis[a];
        A.out_values[i * A.naxes + a] = av >= kPosAxisBase ? pos_axis(cx, cy, cz, r2, av - kPosAxisBase)
                                                           : load_cell<DT>(A.cells, av * plane + c);
    }
    bool pass = true;
    for (int v = 0; v < A.nvars && pass; ++v) {
        if (!((A.brush.mask >> v) & 1u)) continue;
        const float sv = load_cell<DT>(A.cells, v * plane + c);
        pass = sv >= A.brush.lo[v] && sv <= A.brush.hi[v];
    }
    if (pass && A.brush.pmask) pass = pos_pass(cx, cy, cz, r2, A.brush);
    A.out_flags[i] = pass ? 1u : 0u;
}

}  // namespace

cudaError_t launch_pc_subsample(const SubsampleArgs& a, int dtype, unsigned long long m, unsigned long long N,
                                void* scratch, cudaStream_t stream) {
    SubState* S = reinterpret_cast<SubState*>(scratch);
    if (m == 0) return cudaSuccess;
    k_sub_init<<<1, 1024, 0, stream>>>(S, m, m >= N ? 1 : 0);
    const long long rows = (long long)a.n * a.n;
    const long long want = (rows + (kSubThreads / 32) - 1) / (kSubThreads / 32);
    const int hist_blocks = (int)(want < 1024 ? want : 1024);
    for (int round = 0; round < kRounds; ++round) {
        k_sub_hist<<<hist_blocks, kSubThreads, 0, stream>>>(a, S);
        k_sub_pick<<<1, 1024, 0, stream>>>(S);
    }
    const int nseg = (int)(rows < kSubMaxSegments ? rows : kSubMaxSegments);
    const int seg_blocks = (nseg + kSubThreads / 32 - 1) / (kSubThreads / 32);
    k_sub_count<<<seg_blocks, kSubThreads, 0, stream>>>(a, S, nseg);
    k_sub_scan<<<1, 1024, 0, stream>>>(S, nseg);
    k_sub_write<<<seg_blocks, kSubThreads, 0, stream>>>(a, S, nseg);
    const int gblocks = (int)((m + kSubThreads - 1) / kSubThreads);
    if (dtype == kF16)
        k_sub_gather<kF16><<<gblocks, kSubThreads, 0, stream>>>(a);
    else
        k_sub_gather<kF32><<<gblocks, kSubThreads, 0, stream>>>(a);
    count_launches(5 + 2 * kRounds);
    return cudaGetLastError();
}

size_t pc_subsample_scratch_bytes() { return sizeof(SubState); }

}  // namespace raypc

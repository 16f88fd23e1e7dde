// Brush test of given points (Section 3: only the pathlines whose seed lies in
// the current selection are shown). One thread per point runs exactly the
// per-sample test of the ray march: FP32 |p|^2 against the shell and radius
// range, the coordinate brushes, then every restricted variable's FP32
// trilinear value (x-pair loads of the render layout, lerps along x, y, z)
// against the brush, stopping at the first failure. Gather-bound: at most
// four 8- or 4-byte pair loads per restricted variable and point.
#include "common.cuh"

namespace raypc {

namespace {

constexpr int kPointThreads = 256;

template <int DT>
__global__ void __launch_bounds__(kPointThreads) k_filter_points(PointFilterArgs A) {
    const int n = A.n;
    const float hn = 0.5f * (float)n, off = hn - 0.5f, nm1 = (float)(n - 1);
    const size_t sy = (size_t)n, sz = (size_t)n * n, plane = sz * n;
    const size_t pair_bytes = DT == kF16 ? 4 : 8;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < A.npts;
         q += (long long)gridDim.x * blockDim.x) {
        const float x = A.pts[3 * q], y = A.pts[3 * q + 1], z = A.pts[3 * q + 2];
        const float r2 = dot3_rn(x, y, z, x, y, z);
        bool keep = r2 >= A.keep_lo2 && r2 <= A.keep_hi2;
        if (keep && (A.brush.pmask & 7u)) keep = pos_pass(x, y, z, r2, A.brush);
        if (keep && A.brush.mask) {
            float ux, uy, uz;
            const int ix = grid_index_rn(x, n, hn, off, ux);
            const int iy = grid_index_rn(y, n, hn, off, uy);
            const int iz = grid_index_rn(z, n, hn, off, uz);
            const float fx = grid_weight_rn(ux, ix, nm1), fy = grid_weight_rn(uy, iy, nm1), fz = grid_weight_rn(uz, iz, nm1);
            const size_t base = ((size_t)iz * n + iy) * n + ix;
            for (int v = 0; v < A.nvars && keep; ++v) {
                if (!((A.brush.mask >> v) & 1u)) continue;
                const void* pl = reinterpret_cast<const char*>(A.pairs) + pair_bytes * plane * (size_t)v;
                const float2 a = Pair<DT>::load(pl, base), b = Pair<DT>::load(pl, base + sy);
                const float2 c = Pair<DT>::load(pl, base + sz), d = Pair<DT>::load(pl, base + sz + sy);
                const float s = trilerp_rn(a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y, fx, fy, fz);
                keep = s >= A.brush.lo[v] && s <= A.brush.hi[v];
            }
        }
        A.out[q] = keep ? 1u : 0u;
    }
}

}  // namespace

cudaError_t launch_filter_points(const PointFilterArgs& a, int dtype, cudaStream_t stream) {
    if (a.npts <= 0) return cudaSuccess;
    const long long want = (a.npts + kPointThreads - 1) / kPointThreads;
    const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
    if (dtype == kF16)
        k_filter_points<kF16><<<blocks, kPointThreads, 0, stream>>>(a);
    else
        k_filter_points<kF32><<<blocks, kPointThreads, 0, stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace raypc

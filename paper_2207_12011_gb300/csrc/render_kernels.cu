// Brushed emission-absorption ray marching (Section 2.2 of the paper).
//
// One thread per ray; a warp covers a small pixel tile (8x4, 16x2 or 4x8: the
// launch variant) so that neighbouring rays fetch neighbouring vertices, and a
// 128-thread block covers 2x2 warp tiles. The per-pixel march is one device function shared by the
// single-frame kernel and the persistent batched kernel, so a view renders
// bit-identically alone and inside a batch. Per lattice sample: position,
// interpolation cell (exactly rounded FP32), the activity bit of the 4^3
// sub-brick that holds the cell (samples in inactive sub-bricks cannot pass
// the brush or the shell test), shell and radius test, then the restricted
// variables in increasing order of how many bricks pass them alone (most
// selective first; the order cannot change the result) that the sample's cell
// class does not already decide, each as an FP32
// trilinear interpolation from four x-pair loads of that variable only, with
// exit on the first failure. Kept samples are coloured by the transfer function (from shared
// memory) and composited front to back with early ray termination.
//
// The samples inside the inner core are jumped over analytically (exactly: see
// the march). Empty-space skipping: every sample reads its sub-brick's
// empty-space distance D (the Chebyshev distance, in sub-bricks, to the nearest
// active one; 0 for active ones). When the samples of all lanes running
// together have D >= 2 (or >= 4, or 8), every lane's next floor((4 (D - 1) - 1/16) /
// (dt n/2)) samples stay in its box of inactive sub-bricks -- the lattice moves
// a cell index by at most dt n/2 cells per sample on any axis, and 1/16 cell
// covers the FP32 rounding of t, the position and the grid coordinate -- so the
// lanes skip that many samples together (one warp vote) and stay on
// neighbouring samples. The lattice itself (t_k = t0 + (k + j) dt, j = 1/2 except in
// jittered progressive passes) is never shifted by a skip.
#include "common.cuh"

namespace raypc {

namespace {

constexpr int kThreads = kRenderThreads;

__device__ __forceinline__ bool bit_of(const uint32_t* bits, uint32_t id) {
    return (__ldg(bits + (id >> 5)) >> (id & 31)) & 1u;
}

// FP32 trilinear value of one variable: four pair loads give the 8 corners
// (x0, x0+1) at (y0,z0), (y1,z0), (y0,z1), (y1,z1).
template <int DT>
__device__ __forceinline__ float interp_var(const void* plane, size_t base, size_t sy, size_t sz,
                                            float fx, float fy, float fz) {
    const float2 a = Pair<DT>::load(plane, base);
    const float2 b = Pair<DT>::load(plane, base + sy);
    const float2 c = Pair<DT>::load(plane, base + sz);
    const float2 d = Pair<DT>::load(plane, base + sz + sy);
    return trilerp_rn(a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y, fx, fy, fz);
}

__device__ __forceinline__ const void* plane_ptr(const void* pairs, int DT, int v, size_t plane_elems) {
    const size_t bytes = (DT == kF16 ? 4 : 8) * plane_elems * (size_t)v;
    return reinterpret_cast<const char*>(pairs) + bytes;
}

// Per-view block state: the transfer function (staged in shared memory), the
// restricted variables in increasing order of how many bricks pass them alone
// (most selective first), and the brush bounds.
struct ViewShared {
    float4 tf[kTF];
    int order[kMaxVars];
    int nact;
    float lo[kMaxVars], hi[kMaxVars];
};

// Fill S for view A (all threads of the block call it; the caller syncs).
__device__ __forceinline__ void load_view_shared(const RenderArgs& A, ViewShared& S) {
    for (int i = threadIdx.x; i < kTF; i += blockDim.x) S.tf[i] = A.tf[i];
    if (threadIdx.x == 0) {
        int cnt = 0;
        unsigned pc[kMaxVars];
        for (int v = 0; v < A.nvars; ++v) {
            if (!((A.brush.mask >> v) & 1u)) continue;
            unsigned c = A.pass_count ? A.pass_count[v] : 0u;
            int j = cnt++;
            while (j > 0 && pc[j - 1] > c) { pc[j] = pc[j - 1]; S.order[j] = S.order[j - 1]; --j; }
            pc[j] = c;
            S.order[j] = v;
        }
        S.nact = cnt;
    }
    if (threadIdx.x < kMaxVars) {
        S.lo[threadIdx.x] = A.brush.lo[threadIdx.x];
        S.hi[threadIdx.x] = A.brush.hi[threadIdx.x];
    }
}

// March the ray of this thread's pixel in block tile (tile_x, tile_y) of view A
// and write its pixel, optional counts and (warp-aggregated) statistics. All
// 32 lanes of every warp must call it. DEPTH: the depth output may be requested
// (A.depth); without it the march keeps no trace of the first kept sample.
template <int DT, int VAR, bool DEPTH>
__device__ __forceinline__ void march_pixel(const RenderArgs& A, const ViewShared& S, int tile_x, int tile_y) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int WTW = warp_tile_w(VAR), WTH = 32 / WTW;
    const int px = tile_x * block_tile_w(VAR) + (warp & 1) * WTW + (lane % WTW);
    const int py = tile_y * block_tile_h(VAR) + (warp >> 1) * WTH + (lane / WTW);
    const bool inside = px < A.w && py < A.h;

    unsigned marched = 0, kept = 0, evald = 0, skipped = 0, hit = 0, ert_hit = 0;
    float Cr = 0.f, Cg = 0.f, Cb = 0.f, Aa = 0.f;
    float depth = __int_as_float(0x7f800000);       // t of the first kept sample; +inf if none

    if (inside) {
        // Camera basis and pixel direction (exactly rounded, fixed order; the same
        // arithmetic as camera_ray_rn, written out here for the register allocation).
        float Fx = __fsub_rn(A.target[0], A.eye[0]);
        float Fy = __fsub_rn(A.target[1], A.eye[1]);
        float Fz = __fsub_rn(A.target[2], A.eye[2]);
        normalize_rn(Fx, Fy, Fz);
        float Rx, Ry, Rz, Ux, Uy, Uz;
        cross_rn(Fx, Fy, Fz, A.up[0], A.up[1], A.up[2], Rx, Ry, Rz);
        normalize_rn(Rx, Ry, Rz);
        cross_rn(Rx, Ry, Rz, Fx, Fy, Fz, Ux, Uy, Uz);
        const float aspect = __fdiv_rn((float)A.w, (float)A.h);
        const float sxs = __fmul_rn(A.tan_half, aspect);
        const float qx = __fdiv_rn((float)(2 * px + 1), (float)A.w);
        const float qy = __fdiv_rn((float)(2 * py + 1), (float)A.h);
        const float sx = __fmul_rn(__fsub_rn(qx, 1.0f), sxs);
        const float sy = __fmul_rn(__fsub_rn(1.0f, qy), A.tan_half);
        float dx = __fmaf_rn(sy, Ux, __fmaf_rn(sx, Rx, Fx));
        float dy = __fmaf_rn(sy, Uy, __fmaf_rn(sx, Ry, Fy));
        float dz = __fmaf_rn(sy, Uz, __fmaf_rn(sx, Rz, Fz));
        normalize_rn(dx, dy, dz);
        const float ox = A.eye[0], oy = A.eye[1], oz = A.eye[2];
        // Outer-sphere interval through the point closest to the centre.
        const float b = dot3_rn(ox, oy, oz, dx, dy, dz);
        const float hx = __fmaf_rn(-b, dx, ox), hy = __fmaf_rn(-b, dy, oy), hz = __fmaf_rn(-b, dz, oz);
        const float disc = __fsub_rn(A.rout2, dot3_rn(hx, hy, hz, hx, hy, hz));
        if (disc > 0.0f) {
            hit = 1;
            const float sq = __fsqrt_rn(disc);
            const float t0 = fmaxf(__fsub_rn(-b, sq), 0.0f);
            const float t1 = __fadd_rn(-b, sq);
            const int n = A.lv.n, nsb = A.lv.nsb;
            const float hn = 0.5f * (float)n, off = hn - 0.5f;
            const float dt = A.dt;
            const size_t sy_ = (size_t)n, sz_ = (size_t)n * n, plane = sz_ * n;
            const int nact = S.nact;
            // Lattice end: the first k with t_k >= t1, found once per ray from an
            // estimate corrected with the exact predicate (t_k is non-decreasing in k).
            const float inv_dt = 1.0f / dt;
            // lattice offset of this pixel (1/2 unless this is a jittered progressive pass)
            const float jo = lattice_offset(A.jit_seed, A.jit_pass, (unsigned long long)py * A.w + px);
            int n_lat = max(0, (int)floorf((t1 - t0) * inv_dt - jo));
            while (n_lat > 0 && !(__fmaf_rn(__fadd_rn((float)(n_lat - 1), jo), dt, t0) < t1)) --n_lat;
            while (__fmaf_rn(__fadd_rn((float)n_lat, jo), dt, t0) < t1) ++n_lat;
            // samples that stay in a box of inactive sub-bricks extending 4 (D - 1) cells beyond
            // the current sub-brick (the lattice moves a cell index by at most dt n/2 cells per
            // sample on any axis)
            const int skip_near = (int)((4.0f - 0.0625f) / (dt * hn));                        // D >= 2
            const int skip_mid = (int)((12.0f - 0.0625f) / (dt * hn));                        // D >= 4
            const int skip_far = (int)((4.0f * (kDistCap - 1) - 0.0625f) / (dt * hn));         // D >= 8
            // Inner core: the samples core_a..core_b lie inside r_in and fail the shell
            // test, so the march jumps over them. The range comes from the core chord of
            // a slightly smaller sphere and is then verified with the per-sample FP32
            // arithmetic at both ends: t_k grows with k and the exact |o + t d|^2 is
            // convex in t, so no sample in between exceeds the larger end value, and the
            // FP32 |p|^2 of a sample differs from the exact value by at most ~5 * 2^-24
            // relative; ends below r_in^2 (1 - 2^-10) therefore prove every sample in
            // between fails the shell test.
            int core_a = n_lat, core_b = n_lat - 1;               // empty unless verified
            {
                const float hh = dot3_rn(hx, hy, hz, hx, hy, hz);
                const float shrink = __fmul_rn(A.keep_lo2, 1.0f - 0x1p-9f);
                if (hh < shrink) {
                    const float sc = __fsqrt_rn(__fsub_rn(shrink, hh));
                    const float tc0 = __fsub_rn(-b, sc), tc1 = __fadd_rn(-b, sc);
                    const int ka = max(0, (int)ceilf(fminf((tc0 - t0) * inv_dt - jo, 1.0e9f)));
                    const int kb = min(n_lat - 1, (int)floorf(fminf((tc1 - t0) * inv_dt - jo, 1.0e9f)));
                    if (ka < kb) {
                        const float lim = __fmul_rn(A.keep_lo2, 1.0f - 0x1p-10f);
                        const float ta = __fmaf_rn(__fadd_rn((float)ka, jo), dt, t0);
                        const float tb = __fmaf_rn(__fadd_rn((float)kb, jo), dt, t0);
                        const float ax = __fmaf_rn(ta, dx, ox), ay = __fmaf_rn(ta, dy, oy), az = __fmaf_rn(ta, dz, oz);
                        const float bx = __fmaf_rn(tb, dx, ox), by = __fmaf_rn(tb, dy, oy), bz = __fmaf_rn(tb, dz, oz);
                        if (dot3_rn(ax, ay, az, ax, ay, az) <= lim && dot3_rn(bx, by, bz, bx, by, bz) <= lim) {
                            core_a = ka;
                            core_b = kb;
                        }
                    }
                }
            }
            // Coordinate brushes: along the ray each coordinate fma(t_k, d, o) is
            // monotone in k, so the samples inside every restricted coordinate range
            // form one index range [k_first, k_last); the rest are marched but never kept.
            int k_first = 0, k_last = n_lat;
            if (A.brush.pmask & 7u) {
                const float dd[3] = {dx, dy, dz}, oo[3] = {ox, oy, oz};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (!((A.brush.pmask >> a) & 1u)) continue;
                    const float lo = A.brush.plo[a], hi = A.brush.phi[a];
                    const float d = dd[a], o = oo[a];
                    if (d == 0.0f) {                                   // constant coordinate o
                        if (!(o >= lo && o <= hi)) k_last = 0;
                        continue;
                    }
                    // smallest k in [0, n_lat] whose coordinate has entered (leave = false)
                    // or left (leave = true) the range
                    auto first = [&](bool leave) {
                        int l = 0, h = n_lat;
                        while (l < h) {
                            const int m = (l + h) >> 1;
                            const float c = __fmaf_rn(__fmaf_rn(__fadd_rn((float)m, jo), dt, t0), d, o);
                            const bool p = d > 0.0f ? (leave ? c > hi : c >= lo) : (leave ? c < lo : c <= hi);
                            if (p) h = m; else l = m + 1;
                        }
                        return l;
                    };
                    k_first = max(k_first, first(false));
                    k_last = min(k_last, first(true));
                }
            }
            // n_lat is needed again only for the count after the loop: park it in shared
            // memory rather than in a register across the loop
            __shared__ int s_lat[kThreads];
            reinterpret_cast<volatile int*>(s_lat)[threadIdx.x] = n_lat;
            int k = k_first;
            int kend = min(core_a, k_last);                       // first stretch ends at the core
            for (;;) {
                if (k >= kend) {
                    if (kend >= k_last) break;
                    k = max(k, core_b + 1);                      // the rest after the core
                    kend = k_last;
                    continue;
                }
                const float t = __fmaf_rn(__fadd_rn((float)k, jo), dt, t0);
                const float pxw = __fmaf_rn(t, dx, ox), pyw = __fmaf_rn(t, dy, oy), pzw = __fmaf_rn(t, dz, oz);
                int ix, iy, iz;
                float ux, uy, uz;
                ix = grid_index_rn(pxw, n, hn, off, ux);
                iy = grid_index_rn(pyw, n, hn, off, uy);
                iz = grid_index_rn(pzw, n, hn, off, uz);
                const uint32_t sid = ((uint32_t)(iz >> 2) * nsb + (iy >> 2)) * nsb + (ix >> 2);
                bool active;
                if (A.skip && A.lv.sdist) {
                    // the empty-space distance D (0: active): every sub-brick within D - 1 of
                    // this one is inactive, so the cell index stays in that box -- at least
                    // 4 (D - 1) cells beyond this sub-brick on every side -- while the lattice
                    // moves it by less than 4 (D - 1) cells per axis, i.e. for the next
                    // floor((4 (D - 1) - 1/16) / (dt n/2)) samples (dt n/2 bounds the cells
                    // per sample on any axis; 1/16 cell covers the FP32 rounding of t, the
                    // position and the grid coordinate). When all lanes running together
                    // are at D >= 2 (>= 4, >= 8) they skip those samples together, so they
                    // stay on neighbouring samples.
                    const int D = __ldg(A.lv.sdist + sid);
                    active = D == 0;
                    const unsigned grp = __activemask();
                    if (__all_sync(grp, D >= 2 && k + skip_far < 65536)) {
                        const int m = !__all_sync(grp, D >= 4) ? skip_near
                                    : (__all_sync(grp, D >= kDistCap) ? skip_far : skip_mid);
                        skipped += (unsigned)m;
                        k += m + 1;
                        continue;
                    }
                } else {
                    active = bit_of(A.lv.sactive, sid);
                }
                if (!active) {
                    ++k;
                    continue;
                }
                const float r2 = dot3_rn(pxw, pyw, pzw, pxw, pyw, pzw);
                if (!(r2 >= A.keep_lo2 && r2 <= A.keep_hi2)) { ++k; continue; }
                const size_t base = ((size_t)iz * n + iy) * n + ix;
                const float nm1 = (float)(n - 1);
                const float fx = grid_weight_rn(ux, ix, nm1), fy = grid_weight_rn(uy, iy, nm1), fz = grid_weight_rn(uz, iz, nm1);
                ++evald;
                // cell class: a variable whose 8 corners all pass needs no interpolation,
                // one whose corners all fail (or hold a NaN) rejects the sample outright
                unsigned need = 0xffu;
                if (A.cls) {
                    const unsigned c = __ldg(A.cls + base);
                    if (c & kCellFail) { ++k; continue; }
                    need = c;
                }
                bool pass = true;
                float vc = 0.0f;
                bool have_c = false;
                for (int j = 0; j < nact; ++j) {
                    const int v = S.order[j];
                    if (!((need >> v) & 1u)) continue;
                    const float s = interp_var<DT>(plane_ptr(A.lv.pairs, DT, v, plane), base, sy_, sz_, fx, fy, fz);
                    if (!(s >= S.lo[v] && s <= S.hi[v])) { pass = false; break; }
                    if (v == A.color_var) { vc = s; have_c = true; }
                }
                if (!pass) { ++k; continue; }
                if (!have_c)
                    vc = interp_var<DT>(plane_ptr(A.lv.pairs, DT, A.color_var, plane), base, sy_, sz_, fx, fy, fz);
                // index of the first kept sample, parked in the depth output until the end
                if (DEPTH && kept == 0u && A.depth) A.depth[(size_t)py * A.w + px] = __int_as_float(k);
                ++kept;
                // transfer function (continuous; no rounding contract needed)
                float sp = (vc - A.tf_lo) * A.tf_scale;
                sp = fminf(fmaxf(sp, 0.0f), 255.0f);
                const int jj = min((int)sp, kTF - 2);
                const float w = sp - (float)jj;
                const float4 e0 = S.tf[jj], e1 = S.tf[jj + 1];
                const float er = fmaf(w, e1.x - e0.x, e0.x);
                const float eg = fmaf(w, e1.y - e0.y, e0.y);
                const float eb = fmaf(w, e1.z - e0.z, e0.z);
                const float es = fmaf(w, e1.w - e0.w, e0.w);
                const float alpha = 1.0f - __expf(-es * dt);
                const float ta = (1.0f - Aa) * alpha;
                Cr = fmaf(ta, er, Cr);
                Cg = fmaf(ta, eg, Cg);
                Cb = fmaf(ta, eb, Cb);
                Aa += ta;
                if (A.ert && Aa >= kErtThreshold) { ert_hit = 1; ++k; break; }
                ++k;
            }
            // every lattice sample up to termination
            marched = ert_hit ? (unsigned)k : (unsigned)reinterpret_cast<volatile int*>(s_lat)[threadIdx.x];
            if (DEPTH && kept && A.depth)                         // t of the first kept sample
                depth = __fmaf_rn(__fadd_rn((float)__float_as_int(A.depth[(size_t)py * A.w + px]), jo), dt, t0);
        }
        const float tr = 1.0f - Aa;
        float4 o;
        o.x = fmaf(tr, A.bg[0], Cr);
        o.y = fmaf(tr, A.bg[1], Cg);
        o.z = fmaf(tr, A.bg[2], Cb);
        o.w = fmaf(tr, A.bg[3], Aa);
        const size_t pix = (size_t)py * A.w + px;
        A.out[pix] = o;
        if (A.accum) {
            // running mean of the passes 0..jit_pass
            float4 m = o;
            if (A.jit_pass != 0u) {
                const float4 prev = A.accum[pix];
                m.x = fmaf(A.accum_w, o.x - prev.x, prev.x);
                m.y = fmaf(A.accum_w, o.y - prev.y, prev.y);
                m.z = fmaf(A.accum_w, o.z - prev.z, prev.z);
                m.w = fmaf(A.accum_w, o.w - prev.w, prev.w);
            }
            A.accum[pix] = m;
        }
        if (A.counts) {
            A.counts[2 * pix] = marched;
            A.counts[2 * pix + 1] = kept;
        }
        if (DEPTH && A.depth) A.depth[pix] = depth;
    }
    if (A.stats) {
        unsigned vals[6] = {marched, evald, kept, skipped, hit, ert_hit};
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            unsigned r = __reduce_add_sync(0xffffffffu, vals[s]);
            if (lane == 0 && r) atomicAdd(A.stats + s, (unsigned long long)r);
        }
    }
}

template <int DT, int VAR, bool DEPTH>
__global__ void __launch_bounds__(kThreads) k_render(RenderArgs A) {
    __shared__ ViewShared S;
    load_view_shared(A, S);
    __syncthreads();
    march_pixel<DT, VAR, DEPTH>(A, S, blockIdx.x, blockIdx.y);
}

// Per-view classification of a batch: one thread per (view, brick); a warp's
// 32 consecutive flat indices always belong to one view.
__device__ __forceinline__ int view_of_brick(const BatchHeader& H, const BatchView* V, unsigned long long g) {
    int lo = 0, hi = H.nviews - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (V[mid].cls_begin <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_classify_views(const BatchHeader* __restrict__ hdr, const BatchView* __restrict__ views) {
    const BatchHeader H = *hdr;
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < H.cls_total; g += stride) {
        const int vi = view_of_brick(H, views, g - lane);
        const BatchView& V = views[vi];
        size_t b = g - V.cls_begin;
        const bool sub = b >= V.cls_sub;             // uniform per warp: cls_sub is a multiple of 32
        if (sub) b -= V.cls_sub;
        const int nb = sub ? V.a.lv.nsb : V.a.lv.nb;
        const size_t nbricks = (size_t)nb * nb * nb;
        unsigned pass_bits = 0;
        bool act = b < nbricks &&
            classify_brick(b, nb, sub ? kSub : kBrick, 2.0f / (float)V.a.lv.n, V.a.rin2, V.a.rout2, V.a.brush,
                           V.a.nvars, sub ? V.sbmin : V.bmin, sub ? V.sbmax : V.bmax, pass_bits);
        if (act && V.a.tf_skip) {                    // TF-aware skipping of this view
            const size_t o = b * V.a.nvars + V.a.color_var;
            act = tf_range_visible((sub ? V.sbmin : V.bmin)[o], (sub ? V.sbmax : V.bmax)[o], V.a.tf_prefix,
                                   V.a.tf_lo, V.a.tf_scale);
        }
        const unsigned word = __ballot_sync(0xffffffffu, act);
        uint32_t* active = const_cast<uint32_t*>(sub ? V.a.lv.sactive : V.a.lv.active);
        if (lane == 0) active[b >> 5] = word;
        if (sub) {
            // list the active sub-bricks for the view's cell classes
            if (V.slist && word) {
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(V.scount, (unsigned)__popc(word));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (act) V.slist[base + __popc(word & ((1u << lane) - 1u))] = (uint32_t)b;
            }
            continue;
        }
        for (int v = 0; v < V.a.nvars; ++v) {
            const unsigned cnt = __popc(__ballot_sync(0xffffffffu, (pass_bits >> v) & 1u));
            if (lane == 0 && cnt) atomicAdd(const_cast<unsigned*>(V.a.pass_count) + v, cnt);
        }
    }
}

// Cell classes of every view of a batch (see cell_classes_of_subbrick): the
// blocks walk the views in order, each warp taking listed sub-bricks of the
// current view; a view's restricted-variable list is built once per block.
template <int DT>
__global__ void __launch_bounds__(32 * kCellWarps) k_cell_classes_views(const BatchHeader* __restrict__ hdr,
                                                                       const BatchView* __restrict__ views) {
    __shared__ CellVars s_vars;
    const int nviews = hdr->nviews;
    const int lane = threadIdx.x & 31;
    for (int vi = 0; vi < nviews; ++vi) {
        const BatchView& V = views[vi];
        if (!V.slist || !V.a.cls) continue;                 // uniform: the view's table entry
        __syncthreads();                                    // previous view's s_vars no longer read
        if (threadIdx.x == 0) cell_vars_of(V.a.brush, V.a.nvars, s_vars);
        __syncthreads();
        const unsigned count = *V.scount;
        const int n = V.a.lv.n, nsb = V.a.lv.nsb;
        uint16_t* out = const_cast<uint16_t*>(V.a.cls);
        for (unsigned i = blockIdx.x * kCellWarps + (threadIdx.x >> 5); i < count; i += gridDim.x * kCellWarps)
            cell_classes_of_subbrick<DT>(V.a.lv.pairs, n, nsb, __ldg(V.slist + i), lane, s_vars, out);
    }
}

// Persistent batched render: every block repeatedly takes the next block tile
// of the whole batch from an atomic counter (tiles of one view are
// contiguous, views in submission order), reloads its per-view shared state
// when the view changes, and marches the tile. Blocks exit when the tiles run
// out, so the kernel's lifetime is bounded by the batch.
template <int DT, int VAR, bool DEPTH>
__global__ void __launch_bounds__(kThreads, 9) k_render_batch(const BatchHeader* __restrict__ hdr,
                                                           const BatchView* __restrict__ views,
                                                           unsigned* __restrict__ tile_counter) {
    __shared__ ViewShared S;
    __shared__ RenderArgs s_args;
    __shared__ int s_tile, s_view, s_tx, s_ty;
    const BatchHeader H = *hdr;
    int cur_view = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = (int)atomicAdd(tile_counter, 1u);
            int vi = -1;
            if (t < H.total_tiles) {
                int lo = 0, hi = H.nviews - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (views[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
                }
                vi = lo;
                const int local = t - views[vi].tile_begin;
                s_tx = local % views[vi].tiles_x;
                s_ty = local / views[vi].tiles_x;
            }
            s_tile = t;
            s_view = vi;
        }
        __syncthreads();
        if (s_tile >= H.total_tiles) break;
        const int vi = s_view;
        if (vi != cur_view) {
            if (threadIdx.x == 0) s_args = views[vi].a;
            __syncthreads();
            load_view_shared(s_args, S);
            cur_view = vi;
            __syncthreads();
        }
        march_pixel<DT, VAR, DEPTH>(s_args, S, s_tx, s_ty);
        __syncthreads();   // the tile's pixels and statistics are issued; s_* are rewritten next
        if (threadIdx.x == 0) {
            const BatchView& V = views[vi];
            __threadfence();                                  // this block's writes before the count
            const unsigned prev = atomicAdd(V.tile_done, 1u);
            if (prev + 1 == (unsigned)V.ntiles && V.done) {
                // last tile of the view: every other tile's writes precede their counts
                __threadfence();
                ViewDone* rec = V.done;
                for (int k = 0; k < kNStats; ++k)
                    rec->stats[k] = V.a.stats ? __ldcg(V.a.stats + k) : 0ull;
                __threadfence_system();                       // record before the flag, as the host sees it
                rec->seq = V.seq;
            }
        }
    }
}

template <int DT, int VAR, bool DEPTH>
cudaError_t launch_t(const RenderArgs& a, cudaStream_t stream) {
    dim3 grid((a.w + block_tile_w(VAR) - 1) / block_tile_w(VAR), (a.h + block_tile_h(VAR) - 1) / block_tile_h(VAR));
    k_render<DT, VAR, DEPTH><<<grid, kThreads, 0, stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_dt(const RenderArgs& a, cudaStream_t stream) {
    if (a.depth) return launch_t<DT, 1, true>(a, stream);   // depth renders use the 8x4 tiles
    switch (a.variant) {
        case 2: return launch_t<DT, 2, false>(a, stream);
        case 3: return launch_t<DT, 3, false>(a, stream);
        default: return launch_t<DT, 1, false>(a, stream);
    }
}

template <int DT, int VAR, bool DEPTH>
void batch_kernels(const BatchHeader* hdr, const BatchView* views, unsigned* counter, int blocks, cudaStream_t s) {
    k_render_batch<DT, VAR, DEPTH><<<blocks, kThreads, 0, s>>>(hdr, views, counter);
}

template <int DT, int VAR, bool DEPTH>
int batch_occupancy() {
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_render_batch<DT, VAR, DEPTH>, kThreads, 0);
    return blocks > 0 ? blocks : 1;
}

}  // namespace

cudaError_t launch_render(const RenderArgs& a, int dtype, cudaStream_t stream) {
    if (dtype == kF16) return launch_dt<kF16>(a, stream);
    return launch_dt<kF32>(a, stream);
}

// A batch with a depth output in any view runs the depth instance with 8x4 tiles.
int render_batch_blocks_per_sm(int dtype, int variant, bool depth) {
    if (depth) return dtype == kF16 ? batch_occupancy<kF16, 1, true>() : batch_occupancy<kF32, 1, true>();
    if (dtype == kF16)
        return variant == 2 ? batch_occupancy<kF16, 2, false>() : variant == 3 ? batch_occupancy<kF16, 3, false>()
                                                                : batch_occupancy<kF16, 1, false>();
    return variant == 2 ? batch_occupancy<kF32, 2, false>() : variant == 3 ? batch_occupancy<kF32, 3, false>()
                                                            : batch_occupancy<kF32, 1, false>();
}

cudaError_t launch_render_batch(const BatchHeader* hdr, const BatchView* views, unsigned* tile_counter, bool depth,
                                int dtype, int variant, unsigned cls_blocks, int blocks, cudaStream_t stream) {
    k_classify_views<<<cls_blocks, 256, 0, stream>>>(hdr, views);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (dtype == kF16) k_cell_classes_views<kF16><<<cls_blocks, 32 * kCellWarps, 0, stream>>>(hdr, views);
    else k_cell_classes_views<kF32><<<cls_blocks, 32 * kCellWarps, 0, stream>>>(hdr, views);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_subbrick_distance_views(hdr, views, cls_blocks, stream);
    if (e != cudaSuccess) return e;
    if (depth) {
        if (dtype == kF16) batch_kernels<kF16, 1, true>(hdr, views, tile_counter, blocks, stream);
        else batch_kernels<kF32, 1, true>(hdr, views, tile_counter, blocks, stream);
    } else if (dtype == kF16) {
        if (variant == 2) batch_kernels<kF16, 2, false>(hdr, views, tile_counter, blocks, stream);
        else if (variant == 3) batch_kernels<kF16, 3, false>(hdr, views, tile_counter, blocks, stream);
        else batch_kernels<kF16, 1, false>(hdr, views, tile_counter, blocks, stream);
    } else {
        if (variant == 2) batch_kernels<kF32, 2, false>(hdr, views, tile_counter, blocks, stream);
        else if (variant == 3) batch_kernels<kF32, 3, false>(hdr, views, tile_counter, blocks, stream);
        else batch_kernels<kF32, 1, false>(hdr, views, tile_counter, blocks, stream);
    }
    return cudaGetLastError();
}

}  // namespace raypc

// Image warping (Section 2.2): forward reprojection of a rendered frame with
// its depth to a new camera.
#include "common.cuh"

namespace raypc {

namespace {

// Image warping (Section 2.2: frames the renderer has not finished are
// interpolated by warping the last image). Source pixel s with a finite depth
// D becomes P = eye + D d (d its ray direction as in the march); P is projected
// into the new camera with exactly rounded FP32 operations in a fixed order,
// and every target pixel keeps the source of smallest camera-space z, ties to
// the smallest s: one 64-bit atomicMin per source on the key (z bits << 32) | s
// (z > 0, so the float bits order like the values).
__global__ void __launch_bounds__(256) k_warp_clear(unsigned long long* keys, long long npix) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x)
        keys[i] = ~0ull;
}

__global__ void __launch_bounds__(256) k_warp_scatter(WarpArgs A) {
    const long long npix = (long long)A.w * A.h;
    float Fx, Fy, Fz, Rx, Ry, Rz, Ux, Uy, Uz;
    camera_basis_rn(A.to_eye, A.to_target, A.to_up, Fx, Fy, Fz, Rx, Ry, Rz, Ux, Uy, Uz);
    const float aspect = __fdiv_rn((float)A.w, (float)A.h);
    const float sxs = __fmul_rn(A.to_tan_half, aspect), th = A.to_tan_half;
    const float hw = __fmul_rn((float)A.w, 0.5f), hh = __fmul_rn((float)A.h, 0.5f);
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < npix; s += (long long)gridDim.x * blockDim.x) {
        const float D = A.src_depth[s];
        if (!(D < __int_as_float(0x7f800000))) continue;    // no depth (also NaN)
        const int x = (int)(s % A.w), y = (int)(s / A.w);
        float dx, dy, dz;
        camera_ray_rn(A.from_eye, A.from_target, A.from_up, A.from_tan_half, A.w, A.h, x, y, dx, dy, dz);
        const float vx = __fsub_rn(__fmaf_rn(D, dx, A.from_eye[0]), A.to_eye[0]);
        const float vy = __fsub_rn(__fmaf_rn(D, dy, A.from_eye[1]), A.to_eye[1]);
        const float vz = __fsub_rn(__fmaf_rn(D, dz, A.from_eye[2]), A.to_eye[2]);
        const float z = dot3_rn(vx, vy, vz, Fx, Fy, Fz);
        if (!(z > 0.0f)) continue;
        const float X = dot3_rn(vx, vy, vz, Rx, Ry, Rz), Y = dot3_rn(vx, vy, vz, Ux, Uy, Uz);
        const float qx = __fdiv_rn(X, __fmul_rn(z, sxs)), qy = __fdiv_rn(Y, __fmul_rn(z, th));
        const float fi = floorf(__fmul_rn(__fadd_rn(qx, 1.0f), hw)), fj = floorf(__fmul_rn(__fsub_rn(1.0f, qy), hh));
        if (!(fi >= 0.0f && fi < (float)A.w && fj >= 0.0f && fj < (float)A.h)) continue;
        const long long t = (long long)fj * A.w + (long long)fi;
        atomicMin(A.keys + t, ((unsigned long long)__float_as_uint(z) << 32) | (unsigned long long)s);
    }
}

__global__ void __launch_bounds__(256) k_warp_gather(WarpArgs A) {
    const long long npix = (long long)A.w * A.h;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < npix; t += (long long)gridDim.x * blockDim.x) {
        unsigned long long key = A.keys[t];
        if (key == ~0ull && A.fill_holes) {
            // a hole takes its reached neighbour of smallest key: smallest z, then smallest source
            const int x = (int)(t % A.w), y = (int)(t / A.w);
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = x + dx, yy = y + dy;
                    if ((dx == 0 && dy == 0) || xx < 0 || yy < 0 || xx >= A.w || yy >= A.h) continue;
                    const unsigned long long k2 = A.keys[(long long)yy * A.w + xx];
                    key = k2 < key ? k2 : key;
                }
        }
        const bool hit = key != ~0ull;
        const long long s = hit ? (long long)(key & 0xffffffffull) : -1;
        A.out[t] = hit ? A.src_rgba[s] : make_float4(A.bg[0], A.bg[1], A.bg[2], A.bg[3]);
        if (A.out_src) A.out_src[t] = (int)s;
    }
}

}  // namespace

cudaError_t launch_warp(const WarpArgs& a, cudaStream_t stream) {
    const long long npix = (long long)a.w * a.h;
    const long long want = (npix + 255) / 256;
    const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
    k_warp_clear<<<blocks, 256, 0, stream>>>(a.keys, npix);
    k_warp_scatter<<<blocks, 256, 0, stream>>>(a);
    k_warp_gather<<<blocks, 256, 0, stream>>>(a);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace raypc

// normals.cu -- fused back-projection and normal image (Sec. III-C, Eq. 2,
// Alg. 1 second loop; the back-projection of Alg. 2) for sm_103a.
//
// Eq. 2 as printed mixes depth gradients with a pixel back-projection; the
// normal computed here is the exact surface normal of the back-projected depth
// map: n = normalize(t_u x t_v), t_u / t_v the horizontal / vertical
// differences of back-projected points (central, or Sobel-weighted (1,2,1)),
// oriented towards the camera.  One thread per pixel; neighbours come through
// L1.  Outputs SoA points and normals and a validity byte (bit 0 point,
// bit 1 normal).  Back-projection multiplies by 1/fx and 1/fy (rounded once
// from FP64) instead of dividing: a few FP32 ulps on the points, no division
// in the per-pixel work.  The same constant factor on every pixel changes
// normal directions by about 1e-7 rad.
#define PM_FILE_ID 2
#include "pm_internal.cuh"

namespace pm {

struct Cam {
    float ifx, ify, cx, cy;
};

__device__ __forceinline__ bool depth_ok(float z)
{
    return z > 0.0f && z < __int_as_float(0x7f800000);
}

__device__ __forceinline__ float3 backproject(float z, int u, int v, const Cam &k)
{
    float xt = __fmul_rn(__fsub_rn((float)u, k.cx), k.ifx);
    float yt = __fmul_rn(__fsub_rn((float)v, k.cy), k.ify);
    return make_float3(__fmul_rn(z, xt), __fmul_rn(z, yt), z);
}

// depth[i] of a frame of n pixels (bounds-checked in the PM_DEBUG_BOUNDS build)
__device__ __forceinline__ float ld_depth(const float *__restrict__ depth, long long i, long long n)
{
    return PM_INB(i, n) ? __ldg(depth + i) : 0.0f;
}

template <int STENCIL>
__device__ __forceinline__ void normal_at(const float *__restrict__ depth, int w, int h, int u,
                                          int v, const Cam &k, float *P, float *N,
                                          unsigned char *valid)
{
    const long long npx = (long long)w * h;
    const long long p = (long long)v * w + u;
    const float z = ld_depth(depth, p, npx);
    const bool ok = depth_ok(z);
    float3 Pp = ok ? backproject(z, u, v, k) : make_float3(0.f, 0.f, 0.f);
    if (PM_INB(2 * npx + p, 3 * npx)) {
        P[p] = Pp.x;
        P[npx + p] = Pp.y;
        P[2 * npx + p] = Pp.z;
    }
    unsigned char vb = ok ? 1 : 0;
    float3 n = make_float3(0.f, 0.f, 0.f);
    if (ok && u > 0 && v > 0 && u < w - 1 && v < h - 1) {
        float3 tu = make_float3(0.f, 0.f, 0.f), tv = make_float3(0.f, 0.f, 0.f);
        bool all = true;
        if (STENCIL == 0) {
            float ze = ld_depth(depth, p + 1, npx), zw = ld_depth(depth, p - 1, npx);
            float zs = ld_depth(depth, p + w, npx), zn = ld_depth(depth, p - w, npx);
            all = depth_ok(ze) && depth_ok(zw) && depth_ok(zs) && depth_ok(zn);
            float3 a = backproject(ze, u + 1, v, k), b = backproject(zw, u - 1, v, k);
            float3 c = backproject(zs, u, v + 1, k), d = backproject(zn, u, v - 1, k);
            tu = make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
            tv = make_float3(c.x - d.x, c.y - d.y, c.z - d.z);
        } else {
#pragma unroll
            for (int j = -1; j <= 1; ++j) {
                const float wt = j == 0 ? 2.0f : 1.0f;
                float zr1 = ld_depth(depth, p + (long long)j * w + 1, npx);
                float zr0 = ld_depth(depth, p + (long long)j * w - 1, npx);
                float zc1 = ld_depth(depth, p + w + j, npx);
                float zc0 = ld_depth(depth, p - w + j, npx);
                all = all && depth_ok(zr1) && depth_ok(zr0) && depth_ok(zc1) && depth_ok(zc0);
                float3 a = backproject(zr1, u + 1, v + j, k), b = backproject(zr0, u - 1, v + j, k);
                float3 c = backproject(zc1, u + j, v + 1, k), d = backproject(zc0, u + j, v - 1, k);
                tu.x += wt * (a.x - b.x); tu.y += wt * (a.y - b.y); tu.z += wt * (a.z - b.z);
                tv.x += wt * (c.x - d.x); tv.y += wt * (c.y - d.y); tv.z += wt * (c.z - d.z);
            }
        }
        if (all) {
            float cx = tu.y * tv.z - tu.z * tv.y;
            float cy = tu.z * tv.x - tu.x * tv.z;
            float cz = tu.x * tv.y - tu.y * tv.x;
            float l2 = cx * cx + cy * cy + cz * cz;
            if (l2 > 0.0f && l2 < __int_as_float(0x7f800000)) {
                float inv = 1.0f / sqrtf(l2);
                n = make_float3(cx * inv, cy * inv, cz * inv);
                if (n.x * Pp.x + n.y * Pp.y + n.z * Pp.z > 0.0f)
                    n = make_float3(-n.x, -n.y, -n.z);
                vb |= 2;
            }
        }
    }
    if (PM_INB(2 * npx + p, 3 * npx) && PM_INB(p, npx)) {
        N[p] = n.x;
        N[npx + p] = n.y;
        N[2 * npx + p] = n.z;
        valid[p] = vb;
    }
}

template <int STENCIL>
__global__ void __launch_bounds__(256) k_normals(const float *__restrict__ depth, int w, int h,
                                                 Cam k, float *P, float *N, unsigned char *valid)
{
    const int u = blockIdx.x * 32 + threadIdx.x;
    const int v = blockIdx.y * 8 + threadIdx.y;
    if (u < w && v < h)
        normal_at<STENCIL>(depth, w, h, u, v, k, P, N, valid);
}

// Batched form: blockIdx.z selects the frame; blocks past a frame's extent exit.
template <int STENCIL>
__global__ void __launch_bounds__(256) k_normals_batch(const NormFrame *__restrict__ frames)
{
    const NormFrame f = frames[blockIdx.z];
    const int u = blockIdx.x * 32 + threadIdx.x;
    const int v = blockIdx.y * 8 + threadIdx.y;
    if (u < f.w && v < f.h)
        normal_at<STENCIL>(f.depth, f.w, f.h, u, v, Cam{f.ifx, f.ify, f.cx, f.cy}, f.P, f.N,
                           f.valid);
}

cudaError_t launch_normals(const float *depth, int w, int h, float fx, float fy, float cx,
                           float cy, int stencil, float *P, float *N, unsigned char *valid,
                           cudaStream_t s)
{
    dim3 grid((w + 31) / 32, (h + 7) / 8);
    Cam k{(float)(1.0 / (double)fx), (float)(1.0 / (double)fy), cx, cy};
    if (stencil == 0)
        k_normals<0><<<grid, dim3(32, 8), 0, s>>>(depth, w, h, k, P, N, valid);
    else
        k_normals<1><<<grid, dim3(32, 8), 0, s>>>(depth, w, h, k, P, N, valid);
    return cudaGetLastError();
}

cudaError_t launch_normals_batch(const void *d_desc, int n_frames, int max_w, int max_h,
                                 int stencil, cudaStream_t s)
{
    dim3 grid((max_w + 31) / 32, (max_h + 7) / 8, n_frames);
    const NormFrame *f = (const NormFrame *)d_desc;
    if (stencil == 0)
        k_normals_batch<0><<<grid, dim3(32, 8), 0, s>>>(f);
    else
        k_normals_batch<1><<<grid, dim3(32, 8), 0, s>>>(f);
    return cudaGetLastError();
}

PM_BOUNDS_QUERY(bounds_normals)

}  // namespace pm

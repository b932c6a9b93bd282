// normals.cu -- fused back-projection and normal image (Sec. III-C, Eq. 2,
// Alg. 1 second loop; the back-projection of Alg. 2) for sm_103a.
//
// Eq. 2 as printed mixes depth gradients with a pixel back-projection; the
// normal computed here is the exact surface normal of the back-projected depth
// map: n = normalize(t_u x t_v), t_u / t_v the horizontal / vertical
// differences of back-projected points (central, or Sobel-weighted (1,2,1)),
// oriented towards the camera.  One thread per 4 pixels of a row (16-byte
// loads of the depth rows, 16-byte stores of the outputs).  Outputs SoA
// points and normals and a validity byte (bit 0 point, bit 1 normal).
// Back-projection multiplies by 1/fx and 1/fy (rounded once from FP64)
// instead of dividing: a few FP32 ulps on the points, no division in the
// per-pixel work; the factors (u - cx) / fx and (v - cy) / fy are formed once
// per column and row of a thread's window.  The same constant factor on every
// pixel changes normal directions by about 1e-7 rad; so does normalising with
// the hardware reciprocal square root (rsqrtf) instead of 1 / sqrt.
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

// The normal of pixel (u, v) from its 3x3 depth neighbourhood z[dv + 1][du + 1]
// (central differences read the four edge neighbours, Sobel all eight; the
// others are ignored): point Pp, unit normal n (0 if invalid), validity byte.
// xt[c] / yt[r]: the back-projection factors (u - cx) / fx of columns u - 1 ..
// u + 1 and (v - cy) / fy of rows v - 1 .. v + 1 (bp() multiplies by them).
__device__ __forceinline__ float3 bp(float z, float xt, float yt)
{
    return make_float3(__fmul_rn(z, xt), __fmul_rn(z, yt), z);
}

template <int STENCIL>
__device__ __forceinline__ void normal_core(const float (&z)[3][3], const float *xt,
                                            const float *yt, int u, int v, int w, int h,
                                            float3 &Pp, float3 &n, unsigned char &vb)
{
    const bool ok = depth_ok(z[1][1]);
    Pp = ok ? bp(z[1][1], xt[1], yt[1]) : make_float3(0.f, 0.f, 0.f);
    vb = ok ? 1 : 0;
    n = make_float3(0.f, 0.f, 0.f);
    if (!(ok && u > 0 && v > 0 && u < w - 1 && v < h - 1))
        return;
    float3 tu = make_float3(0.f, 0.f, 0.f), tv = make_float3(0.f, 0.f, 0.f);
    bool all = true;
    if (STENCIL == 0) {
        const float ze = z[1][2], zw = z[1][0], zs = z[2][1], zn = z[0][1];
        all = depth_ok(ze) && depth_ok(zw) && depth_ok(zs) && depth_ok(zn);
        float3 a = bp(ze, xt[2], yt[1]), b = bp(zw, xt[0], yt[1]);
        float3 c = bp(zs, xt[1], yt[2]), d = bp(zn, xt[1], yt[0]);
        tu = make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
        tv = make_float3(c.x - d.x, c.y - d.y, c.z - d.z);
    } else {
#pragma unroll
        for (int j = -1; j <= 1; ++j) {
            const float wt = j == 0 ? 2.0f : 1.0f;
            const float zr1 = z[1 + j][2], zr0 = z[1 + j][0];
            const float zc1 = z[2][1 + j], zc0 = z[0][1 + j];
            all = all && depth_ok(zr1) && depth_ok(zr0) && depth_ok(zc1) && depth_ok(zc0);
            float3 a = bp(zr1, xt[2], yt[1 + j]), b = bp(zr0, xt[0], yt[1 + j]);
            float3 c = bp(zc1, xt[1 + j], yt[2]), d = bp(zc0, xt[1 + j], yt[0]);
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
            const float inv = rsqrtf(l2);
            n = make_float3(cx * inv, cy * inv, cz * inv);
            if (n.x * Pp.x + n.y * Pp.y + n.z * Pp.z > 0.0f)
                n = make_float3(-n.x, -n.y, -n.z);
            vb |= 2;
        }
    }
}

// One thread computes 4 consecutive pixels of a row: the three depth rows it
// needs (columns u0 - 1 .. u0 + 4) come as one 16-byte load each plus the two
// edge columns, and the 4 points, normals and validity bytes leave as 16-byte
// (4-byte) stores.  `vec`: the frame's width is a multiple of 4 and every
// array 16-byte aligned (4 for the validity bytes); otherwise element loads
// and stores.  Out-of-image neighbours read as 0 (a pixel on the border is
// not given a normal, so they are never used).
template <int STENCIL>
__device__ __forceinline__ void normals4(const float *__restrict__ depth, int w, int h, int u0,
                                         int v, const Cam &k, float *P, float *N,
                                         unsigned char *valid, bool vec)
{
    if (u0 >= w || v >= h)
        return;
    const long long npx = (long long)w * h;
    float r[3][6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int vv = v + i - 1;
#pragma unroll
        for (int c = 0; c < 6; ++c)
            r[i][c] = 0.0f;
        if (vv < 0 || vv >= h)
            continue;
        const long long row = (long long)vv * w;
        // central differences need the outer columns of the middle row only
        const bool corners = STENCIL == 1 || i == 1;
        if (vec) {
            if (PM_INB(row + u0 + 3, npx)) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(depth + row + u0));
                r[i][1] = q.x; r[i][2] = q.y; r[i][3] = q.z; r[i][4] = q.w;
            }
            if (corners && u0 > 0 && PM_INB(row + u0 - 1, npx))
                r[i][0] = __ldg(depth + row + u0 - 1);
            if (corners && u0 + 4 < w && PM_INB(row + u0 + 4, npx))
                r[i][5] = __ldg(depth + row + u0 + 4);
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int uu = u0 - 1 + c;
                if ((corners || (c >= 1 && c <= 4)) && uu >= 0 && uu < w && PM_INB(row + uu, npx))
                    r[i][c] = __ldg(depth + row + uu);
            }
        }
    }
    // the back-projection factors of the 6 columns and 3 rows, once
    float xt6[6], yt3[3];
#pragma unroll
    for (int c = 0; c < 6; ++c)
        xt6[c] = __fmul_rn(__fsub_rn((float)(u0 - 1 + c), k.cx), k.ifx);
#pragma unroll
    for (int i = 0; i < 3; ++i)
        yt3[i] = __fmul_rn(__fsub_rn((float)(v - 1 + i), k.cy), k.ify);
    float3 Pp[4], n[4];
    unsigned char vb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float z[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                z[i][j] = r[i][q + j];
        normal_core<STENCIL>(z, xt6 + q, yt3, u0 + q, v, w, h, Pp[q], n[q], vb[q]);
    }
    const long long p = (long long)v * w + u0;
    if (vec) {
        if (PM_INB(2 * npx + p + 3, 3 * npx)) {
            *reinterpret_cast<float4 *>(P + p) = make_float4(Pp[0].x, Pp[1].x, Pp[2].x, Pp[3].x);
            *reinterpret_cast<float4 *>(P + npx + p) = make_float4(Pp[0].y, Pp[1].y, Pp[2].y, Pp[3].y);
            *reinterpret_cast<float4 *>(P + 2 * npx + p) =
                make_float4(Pp[0].z, Pp[1].z, Pp[2].z, Pp[3].z);
            *reinterpret_cast<float4 *>(N + p) = make_float4(n[0].x, n[1].x, n[2].x, n[3].x);
            *reinterpret_cast<float4 *>(N + npx + p) = make_float4(n[0].y, n[1].y, n[2].y, n[3].y);
            *reinterpret_cast<float4 *>(N + 2 * npx + p) = make_float4(n[0].z, n[1].z, n[2].z, n[3].z);
        }
        if (PM_INB(p + 3, npx))
            *reinterpret_cast<uchar4 *>(valid + p) = make_uchar4(vb[0], vb[1], vb[2], vb[3]);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (u0 + q >= w || !PM_INB(2 * npx + p + q, 3 * npx))
                continue;
            P[p + q] = Pp[q].x;
            P[npx + p + q] = Pp[q].y;
            P[2 * npx + p + q] = Pp[q].z;
            N[p + q] = n[q].x;
            N[npx + p + q] = n[q].y;
            N[2 * npx + p + q] = n[q].z;
            valid[p + q] = vb[q];
        }
    }
}

__host__ __device__ inline bool normals_vec(const float *depth, const float *P, const float *N,
                                            const unsigned char *valid, int w)
{
    return w % 4 == 0 && (uintptr_t)depth % 16 == 0 && (uintptr_t)P % 16 == 0 &&
           (uintptr_t)N % 16 == 0 && (uintptr_t)valid % 4 == 0;
}

// Block 32 x 8 threads = 128 columns x 8 rows.
template <int STENCIL>
__global__ void __launch_bounds__(256) k_normals(const float *__restrict__ depth, int w, int h,
                                                 Cam k, float *P, float *N, unsigned char *valid,
                                                 bool vec)
{
    normals4<STENCIL>(depth, w, h, (blockIdx.x * 32 + threadIdx.x) * 4, blockIdx.y * 8 + threadIdx.y,
                      k, P, N, valid, vec);
}

// Batched form: blockIdx.z selects the frame; blocks past a frame's extent exit.
template <int STENCIL>
__global__ void __launch_bounds__(256) k_normals_batch(const NormFrame *__restrict__ frames)
{
    const NormFrame f = frames[blockIdx.z];
    normals4<STENCIL>(f.depth, f.w, f.h, (blockIdx.x * 32 + threadIdx.x) * 4,
                      blockIdx.y * 8 + threadIdx.y, Cam{f.ifx, f.ify, f.cx, f.cy}, f.P, f.N,
                      f.valid, normals_vec(f.depth, f.P, f.N, f.valid, f.w));
}

cudaError_t launch_normals(const float *depth, int w, int h, float fx, float fy, float cx,
                           float cy, int stencil, float *P, float *N, unsigned char *valid,
                           cudaStream_t s)
{
    dim3 grid((w + 127) / 128, (h + 7) / 8);
    Cam k{(float)(1.0 / (double)fx), (float)(1.0 / (double)fy), cx, cy};
    const bool vec = normals_vec(depth, P, N, valid, w);
    if (stencil == 0)
        k_normals<0><<<grid, dim3(32, 8), 0, s>>>(depth, w, h, k, P, N, valid, vec);
    else
        k_normals<1><<<grid, dim3(32, 8), 0, s>>>(depth, w, h, k, P, N, valid, vec);
    return cudaGetLastError();
}

cudaError_t launch_normals_batch(const void *d_desc, int n_frames, int max_w, int max_h,
                                 int stencil, cudaStream_t s)
{
    dim3 grid((max_w + 127) / 128, (max_h + 7) / 8, n_frames);
    const NormFrame *f = (const NormFrame *)d_desc;
    if (stencil == 0)
        k_normals_batch<0><<<grid, dim3(32, 8), 0, s>>>(f);
    else
        k_normals_batch<1><<<grid, dim3(32, 8), 0, s>>>(f);
    return cudaGetLastError();
}

PM_BOUNDS_QUERY(bounds_normals)

}  // namespace pm

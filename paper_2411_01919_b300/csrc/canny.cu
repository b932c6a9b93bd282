// canny.cu -- edges of the normal image and the planar regions they bound
// (Sec. III-D: edge detection on the normal vector image, then one region per
// plane), for sm_103a.
//
//   k_canny_nms   : 8-bit code of each normal component (one FP32 FMA), 3x3
//                   Sobel per channel (borders replicated), the strongest
//                   channel's L1 magnitude, the exact 22.5-degree sector test,
//                   non-maximum suppression and the two thresholds, all in one
//                   shared-memory tile (halo 2); writes the state 0/1/2 and the
//                   union-find parent of every weak or strong pixel
//   hysteresis    : the 8-connected components of weak and strong pixels by
//                   union-find (k_uf_union<true>, k_uf_flatten); a component
//                   is an edge when it holds a strong pixel (k_hyst_mark,
//                   k_hyst_out).  No iteration and no host round trip.
//   regions       : eligible pixels (valid, no edge within `gap`) -> 4-connected
//                   components by the same union-find -> component sizes ->
//                   components of at least min_pixels numbered in the raster
//                   order of their first pixel (a prefix scan over the roots).
//
// Union-find: the parent of a pixel is never above the pixel (roots are the
// components' smallest pixel index), so every find follows a strictly
// decreasing chain; a union links the larger root below the smaller one with
// atomicMin and, when it finds that the larger one was no longer a root,
// retries with the parent it met.  The final partition and its roots do not
// depend on the order of the atomics, so the output is deterministic.
#include <climits>

#include "pm_internal.cuh"

namespace pm {

constexpr int CT_W = 32, CT_H = 8;       // output tile of k_canny_nms (one thread per pixel)
constexpr int SCAN_BLOCK = 1024;         // pixels per block of the region numbering scan

__device__ __forceinline__ int normal_code(float n)
{
    const int q = (int)floorf(__fmaf_rn(n, 127.5f, 128.0f));
    return q < 0 ? 0 : q > 255 ? 255 : q;
}

__device__ __forceinline__ int sector_of(int gx, int gy)
{
    const long long a = gx < 0 ? -gx : gx, b = gy < 0 ? -gy : gy, s2 = (a + b) * (a + b);
    if (s2 < 2 * a * a)
        return 0;
    if (s2 < 2 * b * b)
        return 2;
    return (long long)gx * gy > 0 ? 1 : 3;
}

__global__ void __launch_bounds__(CT_W *CT_H) k_canny_nms(const float *__restrict__ N,
                                                         const unsigned char *__restrict__ valid,
                                                         int w, int h, int low, int high,
                                                         unsigned char *state, int *L)
{
    __shared__ short q[3][CT_H + 4][CT_W + 4];
    __shared__ int m[CT_H + 2][CT_W + 2];
    __shared__ unsigned char sec[CT_H + 2][CT_W + 2];
    const int u0 = blockIdx.x * CT_W, v0 = blockIdx.y * CT_H;
    const int tid = threadIdx.y * CT_W + threadIdx.x;
    const long long npx = (long long)w * h;
    for (int i = tid; i < (CT_H + 4) * (CT_W + 4); i += CT_W * CT_H) {
        const int ly = i / (CT_W + 4), lx = i - ly * (CT_W + 4);
        const int u = min(max(u0 + lx - 2, 0), w - 1), v = min(max(v0 + ly - 2, 0), h - 1);
        const long long p = (long long)v * w + u;
        const bool ok = valid[p] & 1;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            q[c][ly][lx] = (short)(ok ? normal_code(N[c * npx + p]) : 128);
    }
    __syncthreads();
    for (int i = tid; i < (CT_H + 2) * (CT_W + 2); i += CT_W * CT_H) {
        const int ly = i / (CT_W + 2), lx = i - ly * (CT_W + 2);
        const int u = u0 + lx - 1, v = v0 + ly - 1;
        int best = 0, sct = 3;
        if (u >= 0 && u < w && v >= 0 && v < h) {
            int bgx = 0, bgy = 0;
            best = -1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // q index of pixel (u, v) is [ly + 1][lx + 1]
                const int gx = (q[c][ly][lx + 2] + 2 * q[c][ly + 1][lx + 2] + q[c][ly + 2][lx + 2]) -
                               (q[c][ly][lx] + 2 * q[c][ly + 1][lx] + q[c][ly + 2][lx]);
                const int gy = (q[c][ly + 2][lx] + 2 * q[c][ly + 2][lx + 1] + q[c][ly + 2][lx + 2]) -
                               (q[c][ly][lx] + 2 * q[c][ly][lx + 1] + q[c][ly][lx + 2]);
                const int mag = abs(gx) + abs(gy);
                if (mag > best) {
                    best = mag;
                    bgx = gx;
                    bgy = gy;
                }
            }
            sct = sector_of(bgx, bgy);
        }
        m[ly][lx] = best;
        sec[ly][lx] = (unsigned char)sct;
    }
    __syncthreads();
    const int u = u0 + threadIdx.x, v = v0 + threadIdx.y;
    if (u >= w || v >= h)
        return;
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
    const int mm = m[ly][lx];
    int behind, ahead;
    switch (sec[ly][lx]) {
    case 0: behind = m[ly][lx - 1]; ahead = m[ly][lx + 1]; break;
    case 1: behind = m[ly - 1][lx - 1]; ahead = m[ly + 1][lx + 1]; break;
    case 2: behind = m[ly - 1][lx]; ahead = m[ly + 1][lx]; break;
    default: behind = m[ly + 1][lx - 1]; ahead = m[ly - 1][lx + 1]; break;
    }
    const bool keep = mm > behind && mm >= ahead;
    const int st = !keep ? 0 : mm > high ? 2 : mm > low ? 1 : 0;
    const long long p = (long long)v * w + u;
    state[p] = (unsigned char)st;
    L[p] = st ? (int)p : -1;
}

// ---------------------------------------------------------------------------
// union-find over pixels (parents in L; -1: not a member)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int uf_find(const int *L, int x, int limit, int *err)
{
    for (int it = 0; it < limit; ++it) {
        const int y = __ldcg(L + x);
        if (y == x)
            return x;
        x = y;
    }
    atomicExch(err, 1);   // unreachable: parents strictly decrease
    return x;
}

__device__ __forceinline__ void uf_unite(int *L, int a, int b, int limit, int *err)
{
    for (int it = 0; it < limit; ++it) {
        a = uf_find(L, a, limit, err);
        b = uf_find(L, b, limit, err);
        if (a == b)
            return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(L + b, a);
        if (old == b)
            return;
        b = old;   // b had been linked meanwhile: join a with its parent instead
    }
    atomicExch(err, 1);
}

// Members p with L[p] >= 0 are joined with their member neighbours: right and
// down (4-connectivity), plus down-right and down-left (8-connectivity).
template <bool CONN8>
__global__ void __launch_bounds__(256) k_uf_union(int *L, int w, int h, int *err)
{
    const long long npx = (long long)w * h;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npx || __ldcg(L + p) < 0)
        return;
    const int limit = (int)npx + 1;
    const int u = (int)(p % w), v = (int)(p / w);
    if (u + 1 < w && __ldcg(L + p + 1) >= 0)
        uf_unite(L, (int)p, (int)p + 1, limit, err);
    if (v + 1 < h) {
        const long long d = p + w;
        if (__ldcg(L + d) >= 0)
            uf_unite(L, (int)p, (int)d, limit, err);
        if (CONN8) {
            if (u + 1 < w && __ldcg(L + d + 1) >= 0)
                uf_unite(L, (int)p, (int)d + 1, limit, err);
            if (u > 0 && __ldcg(L + d - 1) >= 0)
                uf_unite(L, (int)p, (int)d - 1, limit, err);
        }
    }
}

// Every member points at its root; with `size`, the roots count their members.
__global__ void __launch_bounds__(256) k_uf_flatten(int *L, int w, int h, int *size, int *err)
{
    const long long npx = (long long)w * h;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npx || __ldcg(L + p) < 0)
        return;
    const int r = uf_find(L, (int)p, (int)npx + 1, err);
    L[p] = r;
    if (size)
        atomicAdd(size + r, 1);
}

__global__ void __launch_bounds__(256) k_hyst_mark(const unsigned char *state, const int *L,
                                                   long long npx, unsigned char *strong)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < npx && state[p] == 2)
        strong[L[p]] = 1;
}

__global__ void __launch_bounds__(256) k_hyst_out(const unsigned char *state, const int *L,
                                                  long long npx, const unsigned char *strong,
                                                  unsigned char *edges)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < npx)
        edges[p] = (state[p] != 0 && strong[L[p]]) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// regions
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_seg_init(const unsigned char *__restrict__ edges,
                                                  const unsigned char *__restrict__ valid, int w,
                                                  int h, int gap, int *L)
{
    const long long npx = (long long)w * h;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npx)
        return;
    const int u = (int)(p % w), v = (int)(p / w);
    bool ok = valid[p] & 1;
    for (int dy = -gap; dy <= gap && ok; ++dy)
        for (int dx = -gap; dx <= gap; ++dx) {
            const int uu = u + dx, vv = v + dy;
            if (uu >= 0 && uu < w && vv >= 0 && vv < h && edges[(long long)vv * w + uu])
                ok = false;
        }
    L[p] = ok ? (int)p : -1;
}

// flag = root of a component with at least min_pixels members; per block of
// SCAN_BLOCK pixels: exclusive prefix of the flags (pre) and their sum (bsum).
__global__ void __launch_bounds__(SCAN_BLOCK) k_seg_scan1(const int *L, const int *size,
                                                          long long npx, int min_pixels,
                                                          int *pre, int *bsum)
{
    __shared__ int ws[SCAN_BLOCK / 32];
    const long long p = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int f = 0;
    if (p < npx) {
        const int r = L[p];
        f = (r == (int)p && size[r] >= min_pixels) ? 1 : 0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    if (p < npx)
        pre[p] = x - f + (wid > 0 ? ws[wid - 1] : 0);
    if (threadIdx.x == SCAN_BLOCK - 1)
        bsum[blockIdx.x] = ws[SCAN_BLOCK / 32 - 1];
}

// One block: exclusive prefix of the block sums in place; bsum[nb] = total.
__global__ void __launch_bounds__(1024) k_seg_scan2(int *bsum, int nb)
{
    __shared__ int ws[32];
    __shared__ int carry;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const int f = i < nb ? bsum[i] : 0;
        int x = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += y;
        }
        if (lane == 31)
            ws[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int t = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o)
                    t += y;
            }
            ws[lane] = t;
        }
        __syncthreads();
        if (i < nb)
            bsum[i] = carry + x - f + (wid > 0 ? ws[wid - 1] : 0);
        __syncthreads();
        if (threadIdx.x == 0)
            carry += ws[31];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        bsum[nb] = carry;
}

__global__ void __launch_bounds__(256) k_seg_label(const int *L, const int *size, long long npx,
                                                   int min_pixels, const int *pre,
                                                   const int *bsum, int *labels)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npx)
        return;
    const int r = L[p];
    int lab = -1;
    if (r >= 0 && size[r] >= min_pixels)
        lab = bsum[r / SCAN_BLOCK] + pre[r];
    labels[p] = lab;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

cudaError_t canny_edges(const EdgeLaunch &E, cudaStream_t s)
{
    const long long npx = (long long)E.w * E.h;
    cudaError_t e = cudaMemsetAsync(E.strong, 0, (size_t)npx, s);
    if (e != cudaSuccess)
        return e;
    k_canny_nms<<<dim3((E.w + CT_W - 1) / CT_W, (E.h + CT_H - 1) / CT_H), dim3(CT_W, CT_H), 0,
                  s>>>(E.N, E.valid, E.w, E.h, E.low, E.high, E.state, E.L);
    k_uf_union<true><<<blocks_for(npx, 256), 256, 0, s>>>(E.L, E.w, E.h, E.err);
    k_uf_flatten<<<blocks_for(npx, 256), 256, 0, s>>>(E.L, E.w, E.h, nullptr, E.err);
    k_hyst_mark<<<blocks_for(npx, 256), 256, 0, s>>>(E.state, E.L, npx, E.strong);
    k_hyst_out<<<blocks_for(npx, 256), 256, 0, s>>>(E.state, E.L, npx, E.strong, E.edges);
    return cudaGetLastError();
}

cudaError_t segment_regions(const SegLaunch &S, cudaStream_t s)
{
    const long long npx = (long long)S.w * S.h;
    const int nb = blocks_for(npx, SCAN_BLOCK);
    cudaError_t e = cudaMemsetAsync(S.size, 0, (size_t)npx * sizeof(int), s);
    if (e != cudaSuccess)
        return e;
    k_seg_init<<<blocks_for(npx, 256), 256, 0, s>>>(S.edges, S.valid, S.w, S.h, S.gap, S.L);
    k_uf_union<false><<<blocks_for(npx, 256), 256, 0, s>>>(S.L, S.w, S.h, S.err);
    k_uf_flatten<<<blocks_for(npx, 256), 256, 0, s>>>(S.L, S.w, S.h, S.size, S.err);
    k_seg_scan1<<<nb, SCAN_BLOCK, 0, s>>>(S.L, S.size, npx, S.min_pixels, S.pre, S.bsum);
    k_seg_scan2<<<1, 1024, 0, s>>>(S.bsum, nb);
    k_seg_label<<<blocks_for(npx, 256), 256, 0, s>>>(S.L, S.size, npx, S.min_pixels, S.pre,
                                                     S.bsum, S.labels);
    return cudaGetLastError();
}

}  // namespace pm

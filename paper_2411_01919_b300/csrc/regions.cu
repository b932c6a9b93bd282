// regions.cu -- per-region RANSAC in the literal form of Alg. 2 (Sec. III-D):
// one plane model per region (a polygon of the paper's contour step), the
// hypothesis with the minimum total point-to-plane distance wins, and the
// model is kept when more than 90% of the region's points are inliers.
//
//   k_reg_reset   : per-region counters, bounding boxes, error sums
//   k_reg_stats   : point count and bounding box of every region (atomics)
//   k_reg_scan    : prefix of point counts and of chunk counts over regions
//   k_reg_scatter : region-grouped point list (order within a region does not
//                   matter: sums are exact integers, samples come from pixels)
//   k_reg_hyp     : three samples per hypothesis, drawn uniformly over the
//                   region's points by rejection in its bounding box
//                   (Philox4x64-10, key (seed, 1), counter (h, r, frame, 64 j + a)),
//                   FP32 plane through them (hyp_plane)
//   k_reg_score   : every hypothesis of a region against every point of the
//                   region: distance |r| (FP32, the residual of is_inlier)
//                   truncated to a multiple of 2^-32 m and summed in 64-bit
//                   integers; inliers counted with the FP32 decision
//   k_reg_select  : minimum sum (ties: lowest index), 10 * inliers > 9 * points
#include <climits>

#include "pm_internal.cuh"

namespace pm {

constexpr int REG_TRIES = 64;
constexpr int REG_CH = 256;          // points per scoring work item
constexpr int REG_HB = 32;           // hypotheses per scoring work item

__device__ __forceinline__ void philox4x64_10_reg(unsigned long long c[4], unsigned long long k0,
                                                  unsigned long long k1)
{
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
        const unsigned long long lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
        const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0; k1 += W1;
    }
}

__global__ void k_reg_reset(RegionLaunch L)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L.R) {
        L.cnt[i] = 0;
        L.box[4 * i + 0] = INT_MAX;
        L.box[4 * i + 1] = INT_MAX;
        L.box[4 * i + 2] = -1;
        L.box[4 * i + 3] = -1;
    }
    if (i < (long long)L.R * L.H) {
        L.err[i] = 0ull;
        L.inl[i] = 0;
    }
}

// Pixel -> region of a valid member, or -1.
__device__ __forceinline__ int member_region(const RegionLaunch &L, int u, int v)
{
    if (u >= L.w || v >= L.h)
        return -1;
    const long long p = (long long)v * L.w + u;
    const int r = L.regions[p];
    return (r < 0 || r >= L.R || !(L.valid[p] & 1)) ? -1 : r;
}

// Point count and bounding box of every region.  The lanes of a warp that
// hold the same region are combined first (a warp covers 32 pixels of one
// row, mostly of one region), so a region gets one atomic per warp instead
// of one per pixel.
__global__ void k_reg_stats(RegionLaunch L)
{
    const int u = blockIdx.x * 32 + threadIdx.x, v = blockIdx.y * 8 + threadIdx.y;
    const int r = member_region(L, u, v);
    unsigned todo = __ballot_sync(0xffffffffu, r >= 0);
    while (todo) {
        const int lead = __ffs(todo) - 1;
        const int rr = __shfl_sync(0xffffffffu, r, lead);
        const bool in = r == rr;
        const unsigned grp = __ballot_sync(0xffffffffu, in);
        const unsigned u0 = __reduce_min_sync(0xffffffffu, in ? (unsigned)u : 0xffffffffu);
        const unsigned u1 = __reduce_max_sync(0xffffffffu, in ? (unsigned)u : 0u);
        if ((int)threadIdx.x == lead) {
            atomicAdd(L.cnt + rr, __popc(grp));
            atomicMin(L.box + 4 * rr + 0, (int)u0);
            atomicMin(L.box + 4 * rr + 1, v);
            atomicMax(L.box + 4 * rr + 2, (int)u1);
            atomicMax(L.box + 4 * rr + 3, v);
        }
        todo &= ~grp;
    }
}

// One block: exclusive prefix of the point counts (list offsets, scatter
// cursors) and of the chunk counts (scoring work items) over all regions.
__global__ void __launch_bounds__(1024) k_reg_scan(RegionLaunch L)
{
    __shared__ int warp_a[32], warp_b[32];
    __shared__ int carry_a, carry_b;
    if (threadIdx.x == 0) {
        carry_a = 0;
        carry_b = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < L.R; base += blockDim.x) {
        const int r = base + threadIdx.x;
        const int a = r < L.R ? L.cnt[r] : 0;
        const int b = r < L.R ? (a + REG_CH - 1) / REG_CH : 0;
        int xa = a, xb = b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(0xffffffffu, xa, o);
            const int yb = __shfl_up_sync(0xffffffffu, xb, o);
            if (lane >= o) {
                xa += ya;
                xb += yb;
            }
        }
        if (lane == 31) {
            warp_a[wid] = xa;
            warp_b[wid] = xb;
        }
        __syncthreads();
        if (wid == 0) {
            int ta = warp_a[lane], tb = warp_b[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int ya = __shfl_up_sync(0xffffffffu, ta, o);
                const int yb = __shfl_up_sync(0xffffffffu, tb, o);
                if (lane >= o) {
                    ta += ya;
                    tb += yb;
                }
            }
            warp_a[lane] = ta;
            warp_b[lane] = tb;
        }
        __syncthreads();
        const int off_a = carry_a + xa - a + (wid > 0 ? warp_a[wid - 1] : 0);
        const int off_b = carry_b + xb - b + (wid > 0 ? warp_b[wid - 1] : 0);
        if (r < L.R) {
            L.cursor[r] = off_a;
            L.offset[r] = off_a;
            L.chunk_base[r] = off_b;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_a += warp_a[31];
            carry_b += warp_b[31];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        L.chunk_base[L.R] = carry_b;
}

// Region-grouped point list: one cursor atomic per (warp, region).
__global__ void k_reg_scatter(RegionLaunch L)
{
    const int u = blockIdx.x * 32 + threadIdx.x, v = blockIdx.y * 8 + threadIdx.y;
    const int r = member_region(L, u, v);
    const unsigned lt = (1u << threadIdx.x) - 1u;
    unsigned todo = __ballot_sync(0xffffffffu, r >= 0);
    while (todo) {
        const int lead = __ffs(todo) - 1;
        const int rr = __shfl_sync(0xffffffffu, r, lead);
        const bool in = r == rr;
        const unsigned grp = __ballot_sync(0xffffffffu, in);
        int pos = 0;
        if ((int)threadIdx.x == lead)
            pos = atomicAdd(L.cursor + rr, __popc(grp));
        pos = __shfl_sync(0xffffffffu, pos, lead) + __popc(grp & lt);
        if (in) {
            const long long p = (long long)v * L.w + u;
            const long long npx = (long long)L.w * L.h;
            L.list[pos] = make_float4(L.P[p], L.P[npx + p], L.P[2 * npx + p], 0.0f);
        }
        todo &= ~grp;
    }
}

__global__ void __launch_bounds__(128) k_reg_hyp(RegionLaunch L)
{
    const int r = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= L.H)
        return;
    const long long slot = (long long)r * L.H + h;
    L.deg[slot] = 1;
    if (L.cnt[r] < 3)
        return;
    const int u0 = L.box[4 * r + 0], v0 = L.box[4 * r + 1];
    const unsigned long long bw = (unsigned long long)(L.box[4 * r + 2] - u0 + 1);
    const unsigned long long bh = (unsigned long long)(L.box[4 * r + 3] - v0 + 1);
    const long long npx = (long long)L.w * L.h;
    float3 q[3];
    for (int j = 0; j < 3; ++j) {
        long long pick = -1;
        for (int a = 0; a < REG_TRIES && pick < 0; ++a) {
            unsigned long long c[4] = {(unsigned long long)h, (unsigned long long)r, L.frame_idx,
                                       (unsigned long long)(REG_TRIES * j + a)};
            philox4x64_10_reg(c, L.seed, 1ull);
            const int u = u0 + (int)__umul64hi(c[0], bw);
            const int v = v0 + (int)__umul64hi(c[1], bh);
            const long long p = (long long)v * L.w + u;
            if ((L.valid[p] & 1) && L.regions[p] == r)
                pick = p;
        }
        if (pick < 0)
            return;
        q[j] = make_float3(L.P[pick], L.P[npx + pick], L.P[2 * npx + pick]);
    }
    float4 pl;
    if (!hyp_plane(q[0], q[1], q[2], pl))
        return;
    L.hyp[slot] = pl;
    L.deg[slot] = 0;
}

// Work item = (region chunk of REG_CH points, block of REG_HB hypotheses).
// Lane = hypothesis of the block, warp w = the points j = w (mod 4) of the
// chunk; the four warps' partial sums are added in a fixed order and then
// atomically (64-bit integers: exact, order-independent).
__global__ void __launch_bounds__(128) k_reg_score(RegionLaunch L)
{
    __shared__ float4 pts[REG_CH];
    __shared__ unsigned long long se[4][REG_HB];
    __shared__ int si[4][REG_HB];
    const int nhb = (L.H + REG_HB - 1) / REG_HB;
    const long long total = (long long)L.chunk_base[L.R] * nhb;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float nthr2 = -L.thr2;
    const float scale = 4294967296.0f;   // 2^32
    for (long long it = blockIdx.x; it < total; it += gridDim.x) {
        const int wi = (int)(it / nhb), hb = (int)(it - (long long)wi * nhb);
        int lo = 0, hi = L.R - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.chunk_base[mid] <= wi)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int r = lo;
        const int c = wi - L.chunk_base[r];
        const int base = L.offset[r] + c * REG_CH;
        const int cnt = min(REG_CH, L.cnt[r] - c * REG_CH);
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += blockDim.x)
            pts[j] = L.list[base + j];
        __syncthreads();
        const int h = hb * REG_HB + lane;
        const long long slot = (long long)r * L.H + h;
        const bool live = h < L.H && !L.deg[slot];
        unsigned long long e = 0ull;
        int in = 0;
        if (live) {
            const float4 pl = L.hyp[slot];
            for (int j = wid; j < cnt; j += 4) {
                const float4 p = pts[j];
                float res = __fmaf_rn(pl.x, p.x, pl.w);
                res = __fmaf_rn(pl.y, p.y, res);
                res = __fmaf_rn(pl.z, p.z, res);
                e += (unsigned long long)__fmul_rn(fabsf(res), scale);
                in += (int)(__float_as_uint(__fmaf_rn(res, res, nthr2)) >> 31);
            }
        }
        se[wid][lane] = e;
        si[wid][lane] = in;
        __syncthreads();
        if (wid == 0 && live) {
            const unsigned long long es = se[0][lane] + se[1][lane] + se[2][lane] + se[3][lane];
            const int is = si[0][lane] + si[1][lane] + si[2][lane] + si[3][lane];
            atomicAdd(L.err + slot, es);
            atomicAdd(L.inl + slot, is);
        }
    }
}

__global__ void __launch_bounds__(128) k_reg_select(RegionLaunch L)
{
    __shared__ unsigned long long best_e[4];
    __shared__ int best_h[4];
    const int r = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long e = ULLONG_MAX;
    int hbest = INT_MAX;
    if (L.cnt[r] >= 3) {
        for (int h = threadIdx.x; h < L.H; h += blockDim.x) {
            const long long slot = (long long)r * L.H + h;
            if (L.deg[slot])
                continue;
            const unsigned long long v = L.err[slot];
            if (v < e || (v == e && h < hbest)) {
                e = v;
                hbest = h;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long oe = __shfl_xor_sync(0xffffffffu, e, o);
        const int oh = __shfl_xor_sync(0xffffffffu, hbest, o);
        if (oe < e || (oe == e && oh < hbest)) {
            e = oe;
            hbest = oh;
        }
    }
    if (lane == 0) {
        best_e[wid] = e;
        best_h[wid] = hbest;
    }
    __syncthreads();
    if (threadIdx.x != 0)
        return;
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (best_e[w] < e || (best_e[w] == e && best_h[w] < hbest)) {
            e = best_e[w];
            hbest = best_h[w];
        }
    pm_region_plane o;
    o.n[0] = o.n[1] = o.n[2] = 0.0;
    o.d = 0.0;
    o.error = 0ull;
    o.inliers = 0;
    o.total = L.cnt[r];
    o.accepted = 0;
    o.hyp_index = -1;
    if (hbest != INT_MAX) {
        const long long slot = (long long)r * L.H + hbest;
        const float4 pl = L.hyp[slot];
        o.n[0] = pl.x;
        o.n[1] = pl.y;
        o.n[2] = pl.z;
        o.d = pl.w;
        o.error = L.err[slot];
        o.inliers = L.inl[slot];
        o.accepted = 10LL * o.inliers > 9LL * o.total ? 1 : 0;
        o.hyp_index = hbest;
    }
    L.out[r] = o;
}

cudaError_t ransac_regions(const RegionLaunch &L, int sms, cudaStream_t s)
{
    const long long nreset = (long long)L.R * L.H > L.R ? (long long)L.R * L.H : L.R;
    k_reg_reset<<<(int)((nreset + 255) / 256), 256, 0, s>>>(L);
    const dim3 pg((L.w + 31) / 32, (L.h + 7) / 8);
    k_reg_stats<<<pg, dim3(32, 8), 0, s>>>(L);
    k_reg_scan<<<1, 1024, 0, s>>>(L);
    k_reg_scatter<<<pg, dim3(32, 8), 0, s>>>(L);
    k_reg_hyp<<<dim3((L.H + 127) / 128, L.R), 128, 0, s>>>(L);
    k_reg_score<<<sms * 8, 128, 0, s>>>(L);
    k_reg_select<<<L.R, 128, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace pm

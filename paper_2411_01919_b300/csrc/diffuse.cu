// diffuse.cu -- anisotropic diffusion of the depth image (Sec. III-C, Eq. 1,
// Alg. 1 first loop) for sm_103a.
//
// Numerics.  Where neighbouring depths differ by more than K/sqrt(2) the
// Perona-Malik flux g(x) x decreases with |x| (backward diffusion), and a
// rounding error of the iterate grows from one iteration to the next: a plain
// FP32 iterate drifts 2e-5 m (640x480 staircase, 30 iterations) to 1.5e-4 m
// (far spiral floor, 40 iterations) away from exact arithmetic.  The iterate
// is therefore carried as a pair of FP32 numbers (hi, lo) with I = hi + lo:
// hi is the decoded depth, split exactly from the u16 encoding (two-product)
// and never changed; lo starts at the decode's tail and accumulates every
// update.  lo stays within a few centimetres, so its rounding is near 1e-9 m;
// neighbour differences take the hi parts exactly (neighbouring depths differ
// by less than a factor of two) and add the lo parts.  The output is hi + lo
// rounded once.  All arithmetic stays on the FP32 pipes.
//
// Two kernels share one per-pixel update (so their results are bit-identical):
//  * k_diffuse_tiles: temporal blocking.  A CTA loads a (dx+2T) x (dy+2T) tile
//    with a T-pixel halo into shared memory, runs T Jacobi iterations there on
//    a shrinking region, and writes the dx x dy interior.  Tiles of every
//    frame of a batch form one grid (a frame table maps tile -> frame).
//  * k_diffuse_stream: one iteration per launch over one frame, one pass over
//    HBM.
// Holes and pixels outside the image hold the sentinel HOLE = 1e30 in the
// iterate: across a link to it the difference x is about 1e30, x*x overflows
// to +inf, 2^(x*x*c) is exactly +0 and so is the flux g(x) x -- the ghost rule
// J_q = I_p of the oracle (no flux across a hole or the border) without a
// branch; a hole receives only zero fluxes and keeps its value.  The first
// launch decodes the sensor encoding on the fly (holes -> HOLE); the last
// writes FP32 depth (hi + lo rounded to nearest; HOLE -> 0).
#include "pm_internal.cuh"

namespace pm {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// q - p for two compensated values (exactly antisymmetric in p, q).
__device__ __forceinline__ float pair_diff(float2 q, float2 p)
{
    return __fadd_rn(__fsub_rn(q.x, p.x), __fsub_rn(q.y, p.y));
}

// (hi, lo) + a: the update goes to lo (hi is the fixed decoded depth).
__device__ __forceinline__ float2 pair_add(float2 p, float a)
{
    return make_float2(p.x, __fadd_rn(p.y, a));
}

constexpr float HOLE = 1e30f;

// Flux into p from neighbour q across one link: g(x) x with x = I_q - I_p and
// g(x) = exp(-(x/K)^2) = 2^(x^2 * c), c = -log2(e)/K^2.  Exactly antisymmetric
// in (p, q) (the negation of x is exact, and so are x*x and g), and exactly
// zero when either end is HOLE.
__device__ __forceinline__ float link_flux(float2 Ip, float2 Iq, float c)
{
    const float x = pair_diff(Iq, Ip);
    const float g = ex2_approx(__fmul_rn(__fmul_rn(x, x), c));
    return __fmul_rn(g, x);
}

// mode 0 (PM4): I' = I + lambda * (((f_N + f_S) + f_W) + f_E)
__device__ __forceinline__ float2 update_pm4(float2 Ip, float2 In, float2 Is, float2 Iw,
                                             float2 Ie, float lam, float c)
{
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(link_flux(Ip, In, c), link_flux(Ip, Is, c)),
                                        link_flux(Ip, Iw, c)), link_flux(Ip, Ie, c));
    return pair_add(Ip, __fmul_rn(lam, s));
}

// mode 1 (ALG1): c_p from the central-difference gradient of the ghosted
// values, times the 4-neighbour Laplacian.
__device__ __forceinline__ float2 update_alg1(float2 Ip, float2 In, float2 Is, float2 Iw,
                                              float2 Ie, float lam, float c)
{
    if (Ip.x == HOLE)
        return Ip;
    const float2 Jn = In.x == HOLE ? Ip : In, Js = Is.x == HOLE ? Ip : Is;
    const float2 Jw = Iw.x == HOLE ? Ip : Iw, Je = Ie.x == HOLE ? Ip : Ie;
    const float gx = __fmul_rn(pair_diff(Je, Jw), 0.5f);
    const float gy = __fmul_rn(pair_diff(Js, Jn), 0.5f);
    const float g2 = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
    const float cp = ex2_approx(__fmul_rn(g2, c));
    const float lap = __fadd_rn(__fadd_rn(__fadd_rn(pair_diff(Jn, Ip), pair_diff(Js, Ip)),
                                          pair_diff(Jw, Ip)), pair_diff(Je, Ip));
    return pair_add(Ip, __fmul_rn(__fmul_rn(lam, cp), lap));
}

template <int MODE>
__device__ __forceinline__ float2 update(float2 Ip, float2 In, float2 Is, float2 Iw, float2 Ie,
                                         float lam, float c)
{
    return MODE == 0 ? update_pm4(Ip, In, Is, Iw, Ie, lam, c)
                     : update_alg1(Ip, In, Is, Iw, Ie, lam, c);
}

// Source pixel -> compensated metres; holes (0, negative, non-finite) -> HOLE.
// u16: q * scale split exactly (q has at most 16 significant bits, so the
// product fits in 40 bits and the fused multiply-add returns its exact tail).
__device__ __forceinline__ float2 load_px(const void *src, int dtype, long long pitch, int x,
                                          int y, float scale)
{
    const char *row = (const char *)src + (long long)y * pitch;
    float v;
    if (dtype == SRC_PAIR) {
        return __ldg((const float2 *)row + x);
    } else if (dtype == PM_U16_MM) {
        const unsigned short q = __ldg((const unsigned short *)row + x);
        if (!q)
            return make_float2(HOLE, 0.0f);
        const float qf = (float)q;
        const float hi = __fmul_rn(qf, scale);
        return make_float2(hi, __fmaf_rn(qf, scale, -hi));
    } else if (dtype == PM_F16_M) {
        v = __half2float(__ldg((const __half *)row + x));
    } else {
        v = __ldg((const float *)row + x);
    }
    return make_float2((v > 0.0f && v < __int_as_float(0x7f800000)) ? v : HOLE, 0.0f);
}

__device__ __forceinline__ float depth_out(float2 v)
{
    return v.x == HOLE ? 0.0f : __fadd_rn(v.x, v.y);
}

__device__ __forceinline__ void store_px(const DiffFrame &f, long long i, float2 v)
{
    if (f.dst_pair)
        reinterpret_cast<float2 *>(f.dst)[i] = v;
    else
        reinterpret_cast<float *>(f.dst)[i] = depth_out(v);
}

// PM4 update from the four link fluxes, in the order of update_pm4 (a HOLE
// pixel receives only zero fluxes and keeps its value).
__device__ __forceinline__ float2 pm4_combine(float2 Ip, float fN, float fS, float fW, float fE,
                                              float lam)
{
    return pair_add(Ip, __fmul_rn(lam, __fadd_rn(__fadd_rn(__fadd_rn(fN, fS), fW), fE)));
}

// Temporal blocking.  Block = 32 x 8 threads; tile = dx x dy output pixels
// with a T-pixel halo, (dx + 2T) x (dy + 2T) cells in shared memory: the hi
// parts once (they never change), the lo parts in two buffers (12 bytes per
// cell).  Iteration it updates the region shrunk by it + 1 on every side.  Each warp (one threadIdx.y) walks a band of rows top to bottom for
// its columns (lane, lane + 32, ...): the south link flux of a row is the
// negated north link flux of the next row (exactly, see link_flux), so each
// pixel evaluates three links (N reused) instead of four.
template <int MODE>
__global__ void __launch_bounds__(256) k_diffuse_tiles(const DiffFrame *__restrict__ frames,
                                                       int n_frames, int T, int dx, int dy,
                                                       float lam, float c)
{
    extern __shared__ float sm1[];
    const int tile = blockIdx.x;
    int lo = 0, hi = n_frames - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (frames[mid].tile_begin <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    const DiffFrame f = frames[lo];
    const int tl = tile - f.tile_begin;
    const int tx0 = (tl % f.tiles_x) * dx;
    const int ty0 = (tl / f.tiles_x) * dy;
    const int SX = dx + 2 * T, SY = dy + 2 * T, NC = SX * SY;
    float *Hs = sm1;             // hi parts
    float *A = sm1 + NC;         // lo parts read by this iteration
    float *B = sm1 + 2 * NC;     // lo parts it writes
    const int lane = threadIdx.x, wy = threadIdx.y;

    if (f.src_dtype == SRC_PAIR || f.src_dtype == PM_U16_MM) {
        // the iterate of the previous launch, or the u16 encoding (decoded on
        // the store): per warp two rows of 96 cells in flight before any
        // shared-memory store
        constexpr int G = 3;
        const bool pair = f.src_dtype == SRC_PAIR;
        const float2 hole = make_float2(HOLE, 0.0f);
        for (int y0 = wy; y0 < SY; y0 += 16) {
            for (int x0 = 0; x0 < SX; x0 += 32 * G) {
                float2 v[2][G];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int y = y0 + 8 * r, gy = ty0 - T + y;
                    const bool row_ok = y < SY && gy >= 0 && gy < f.h;
                    const char *row = (const char *)f.src + (long long)(row_ok ? gy : 0) * f.src_pitch;
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int x = x0 + lane + 32 * g, gx = tx0 - T + x;
                        const bool ok = row_ok && x < SX && gx >= 0 && gx < f.w;
                        if (pair) {
                            v[r][g] = ok ? __ldg(reinterpret_cast<const float2 *>(row) + gx) : hole;
                        } else {
                            const unsigned short q =
                                ok ? __ldg(reinterpret_cast<const unsigned short *>(row) + gx) : 0;
                            v[r][g].x = __int_as_float((int)q);   // the raw code, decoded below
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int y = y0 + 8 * r;
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int x = x0 + lane + 32 * g;
                        if (y < SY && x < SX) {
                            float2 w = v[r][g];
                            if (!pair) {
                                const int q = __float_as_int(w.x);
                                const float qf = (float)q;
                                const float h = __fmul_rn(qf, f.scale);
                                w = q ? make_float2(h, __fmaf_rn(qf, f.scale, -h)) : hole;
                            }
                            Hs[y * SX + x] = w.x;
                            A[y * SX + x] = w.y;
                        }
                    }
                }
            }
        }
    } else {
        for (int y = wy; y < SY; y += 8) {
            const int gy = ty0 - T + y;
            for (int x = lane; x < SX; x += 32) {
                const int gx = tx0 - T + x;
                float2 v = make_float2(HOLE, 0.0f);
                if (gx >= 0 && gx < f.w && gy >= 0 && gy < f.h)
                    v = load_px(f.src, f.src_dtype, f.src_pitch, gx, gy, f.scale);
                Hs[y * SX + x] = v.x;
                A[y * SX + x] = v.y;
            }
        }
    }
    __syncthreads();
    for (int it = 0; it < f.n_iters; ++it) {
        const int r0 = it + 1;
        const int RH = SY - 2 * r0;
        const int band = (RH + 7) >> 3;
        const int y0 = r0 + wy * band;
        const int y1 = min(y0 + band, SY - r0);
        if (y0 < y1) {
            if (MODE == 0) {
                // the lane's columns x = r0 + lane + 32 g, one group at a time,
                // each walked down the band with running pointers; lanes past
                // the region's right edge compute on a clamped column and do
                // not store
                const int xe = SX - r0;
                for (int g = 0; r0 + 32 * g < xe; ++g) {
                    const int x = r0 + lane + 32 * g;
                    const bool act = x < xe;
                    const int k0 = y0 * SX + (act ? x : xe - 1);
                    const float *ph = Hs + k0;
                    const float *pa = A + k0;
                    float *pb = B + k0;
                    float2 cen = make_float2(ph[0], pa[0]);
                    float fN = link_flux(cen, make_float2(ph[-SX], pa[-SX]), c);
                    for (int y = y0; y < y1; ++y, ph += SX, pa += SX, pb += SX) {
                        const float2 dn = make_float2(ph[SX], pa[SX]);
                        const float fS = link_flux(cen, dn, c);
                        const float fW = link_flux(cen, make_float2(ph[-1], pa[-1]), c);
                        const float fE = link_flux(cen, make_float2(ph[1], pa[1]), c);
                        const float2 v = pm4_combine(cen, fN, fS, fW, fE, lam);
                        if (act)
                            *pb = v.y;
                        fN = -fS;
                        cen = dn;
                    }
                }
            } else {
                for (int x = r0 + lane; x < SX - r0; x += 32)
                    for (int y = y0; y < y1; ++y) {
                        const int k = y * SX + x;
                        const float2 v = update_alg1(
                            make_float2(Hs[k], A[k]), make_float2(Hs[k - SX], A[k - SX]),
                            make_float2(Hs[k + SX], A[k + SX]), make_float2(Hs[k - 1], A[k - 1]),
                            make_float2(Hs[k + 1], A[k + 1]), lam, c);
                        B[k] = v.y;
                    }
            }
        }
        __syncthreads();
        float *t = A; A = B; B = t;
    }
    for (int y = wy; y < dy; y += 8) {
        const int gy = ty0 + y;
        if (gy >= f.h)
            break;
        for (int x = lane; x < dx; x += 32) {
            const int gx = tx0 + x;
            const int k = (y + T) * SX + x + T;
            if (gx < f.w)
                store_px(f, (long long)gy * f.w + gx, make_float2(Hs[k], A[k]));
        }
    }
}

// Source pixel of a launch whose encoding SRC is known at compile time.
template <int SRC>
__device__ __forceinline__ float2 load_src(const DiffFrame &f, int x, int y)
{
    const char *row = (const char *)f.src + (long long)y * f.src_pitch;
    if (SRC == SRC_PAIR)
        return __ldg((const float2 *)row + x);
    return load_px(f.src, SRC, f.src_pitch, x, y, f.scale);
}

// Two horizontally adjacent pixels (x even) in one access where the row
// pitch and the base pointer allow it: 16 bytes for the float2 iterate, 8 for
// FP32.
template <int SRC>
__device__ __forceinline__ void load_src2(const DiffFrame &f, int x, int y, bool vec, float2 &a,
                                          float2 &b)
{
    const char *row = (const char *)f.src + (long long)y * f.src_pitch;
    if (SRC == SRC_PAIR && vec) {
        const float4 v = __ldg((const float4 *)row + (x >> 1));
        a = make_float2(v.x, v.y);
        b = make_float2(v.z, v.w);
        return;
    }
    if (SRC == PM_F32_M && vec) {
        const float2 v = __ldg((const float2 *)row + (x >> 1));
        const float inf = __int_as_float(0x7f800000);
        a = make_float2((v.x > 0.0f && v.x < inf) ? v.x : HOLE, 0.0f);
        b = make_float2((v.y > 0.0f && v.y < inf) ? v.y : HOLE, 0.0f);
        return;
    }
    a = load_src<SRC>(f, x, y);
    b = load_src<SRC>(f, x + 1, y);
}

// One iteration over one frame, one pass over HBM.  Block = 32 x 8 threads;
// lane l of warp w covers the two columns x0 = 64*blockIdx.x + 2l, x0 + 1 and
// walks STREAM_ROWS rows down: the north link flux of a row is the negated
// south link flux of the row before (exactly, see link_flux) and the link
// between the two columns is evaluated once; the horizontal neighbours come
// from the adjacent lanes by shuffle, and lanes 0 and 31 fetch the column
// just outside the warp.  Every link enters the sum of update_pm4 with the
// same value and in the same order, so the result is bit-identical to the
// tiled kernel.
constexpr int STREAM_ROWS = 8;

template <int MODE, int SRC>
__global__ void __launch_bounds__(256) k_diffuse_stream(DiffFrame f, float lam, float c)
{
    const int lane = threadIdx.x;
    const int x0 = blockIdx.x * 64 + 2 * lane;
    const int y0 = (blockIdx.y * 8 + threadIdx.y) * STREAM_ROWS;
    if (y0 >= f.h)
        return;
    const int y1 = min(y0 + STREAM_ROWS, f.h);
    const float2 Z = make_float2(HOLE, 0.0f);
    const int vb = SRC == SRC_PAIR ? 16 : 8;
    const bool vec_ld = (SRC == SRC_PAIR || SRC == PM_F32_M) && f.src_pitch % vb == 0 &&
                        ((uintptr_t)f.src % vb) == 0;
    const int ob = f.dst_pair ? 16 : 8;
    const bool vec_st = ((long long)f.w * (f.dst_pair ? 8 : 4)) % ob == 0 &&
                        ((uintptr_t)f.dst % ob) == 0;
    auto ld2 = [&](int y, float2 &a, float2 &b) {
        a = Z;
        b = Z;
        if (y < 0 || y >= f.h)
            return;
        if (x0 + 1 < f.w)
            load_src2<SRC>(f, x0, y, vec_ld, a, b);
        else if (x0 < f.w)
            a = load_src<SRC>(f, x0, y);
    };
    // the column just outside the warp: x0 - 1 for lane 0, x0 + 2 for lane 31
    const int xe = lane == 0 ? x0 - 1 : x0 + 2;
    const bool edge = (lane == 0 || lane == 31) && xe >= 0 && xe < f.w;

    float2 a0, a1, u0, u1;
    ld2(y0, a0, a1);
    ld2(y0 - 1, u0, u1);
    float fN0 = 0.0f, fN1 = 0.0f;
    if (MODE == 0) {
        fN0 = link_flux(a0, u0, c);
        fN1 = link_flux(a1, u1, c);
    }
    for (int y = y0; y < y1; ++y) {
        float2 d0, d1;
        ld2(y + 1, d0, d1);
        float2 E = Z;
        if (edge)
            E = load_src<SRC>(f, xe, y);
        float2 L = make_float2(__shfl_up_sync(0xffffffffu, a1.x, 1),
                               __shfl_up_sync(0xffffffffu, a1.y, 1));
        float2 R = make_float2(__shfl_down_sync(0xffffffffu, a0.x, 1),
                               __shfl_down_sync(0xffffffffu, a0.y, 1));
        if (lane == 0)
            L = E;
        if (lane == 31)
            R = E;
        float2 n0, n1;
        if (MODE == 0) {
            const float f01 = link_flux(a0, a1, c);              // into x0 from x0+1
            const float fE1 = link_flux(a1, R, c);               // into x0+1 from x0+2
            const float fW0 = link_flux(a0, L, c);               // into x0 from x0-1
            const float fW1 = -f01;
            const float fS0 = link_flux(a0, d0, c), fS1 = link_flux(a1, d1, c);
            n0 = pm4_combine(a0, fN0, fS0, fW0, f01, lam);
            n1 = pm4_combine(a1, fN1, fS1, fW1, fE1, lam);
            fN0 = -fS0;
            fN1 = -fS1;
        } else {
            n0 = update_alg1(a0, u0, d0, L, a1, lam, c);
            n1 = update_alg1(a1, u1, d1, a0, R, lam, c);
        }
        if (f.n_iters == 0) {
            n0 = a0;
            n1 = a1;
        }
        const long long row = (long long)y * f.w;
        if (vec_st && x0 + 1 < f.w) {
            if (f.dst_pair)
                reinterpret_cast<float4 *>(f.dst)[(row + x0) >> 1] = make_float4(n0.x, n0.y, n1.x, n1.y);
            else
                reinterpret_cast<float2 *>(f.dst)[(row + x0) >> 1] =
                    make_float2(depth_out(n0), depth_out(n1));
        } else {
            if (x0 < f.w)
                store_px(f, row + x0, n0);
            if (x0 + 1 < f.w)
                store_px(f, row + x0 + 1, n1);
        }
        u0 = a0; u1 = a1;
        a0 = d0; a1 = d1;
    }
}

static inline float conductance_scale(float K)
{
    // exp(-(x/K)^2) = 2^(x^2 * c) with c = -log2(e) / K^2
    return (float)(-1.4426950408889634 / ((double)K * (double)K));
}

size_t diffuse_tiles_smem(int T, int dx, int dy)
{
    return 3ull * (dx + 2 * T) * (dy + 2 * T) * sizeof(float);
}

cudaError_t diffuse_init()
{
    const int mx = (int)diffuse_tiles_smem(DT_MAX, TILE_MAX_DX, TILE_MAX_DY);
    cudaError_t e = cudaFuncSetAttribute(k_diffuse_tiles<0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_diffuse_tiles<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 mx);
    return e;
}

cudaError_t launch_diffuse_tiles(const DiffFrame *d_frames, int n_frames, int total_tiles, int T,
                                 int dx, int dy, float lambda, float K, int mode, cudaStream_t s)
{
    if (T < 0 || T > DT_MAX || dx < 1 || dy < 1 || dx > TILE_MAX_DX || dy > TILE_MAX_DY)
        return cudaErrorInvalidValue;
    const size_t smem = diffuse_tiles_smem(T, dx, dy);
    const float c = conductance_scale(K);
    const dim3 block(32, 8);
    if (mode == 0)
        k_diffuse_tiles<0><<<total_tiles, block, smem, s>>>(d_frames, n_frames, T, dx, dy, lambda, c);
    else
        k_diffuse_tiles<1><<<total_tiles, block, smem, s>>>(d_frames, n_frames, T, dx, dy, lambda, c);
    return cudaGetLastError();
}

cudaError_t launch_diffuse_stream(const DiffFrame &f, float lambda, float K, int mode,
                                  cudaStream_t s)
{
    dim3 grid((f.w + 63) / 64, (f.h + 8 * STREAM_ROWS - 1) / (8 * STREAM_ROWS));
    const dim3 block(32, 8);
    const float c = conductance_scale(K);
#define PM_STREAM(M, S) k_diffuse_stream<M, S><<<grid, block, 0, s>>>(f, lambda, c)
    switch (f.src_dtype * 2 + (mode ? 1 : 0)) {
    case PM_U16_MM * 2: PM_STREAM(0, PM_U16_MM); break;
    case PM_U16_MM * 2 + 1: PM_STREAM(1, PM_U16_MM); break;
    case PM_F16_M * 2: PM_STREAM(0, PM_F16_M); break;
    case PM_F16_M * 2 + 1: PM_STREAM(1, PM_F16_M); break;
    case PM_F32_M * 2: PM_STREAM(0, PM_F32_M); break;
    case PM_F32_M * 2 + 1: PM_STREAM(1, PM_F32_M); break;
    case SRC_PAIR * 2: PM_STREAM(0, SRC_PAIR); break;
    case SRC_PAIR * 2 + 1: PM_STREAM(1, SRC_PAIR); break;
    default: return cudaErrorInvalidValue;
    }
#undef PM_STREAM
    return cudaGetLastError();
}

}  // namespace pm

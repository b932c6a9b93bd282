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
// Because hi is the decoded input, a launch decodes it again from the sensor
// encoding (2 bytes per pixel for u16 / f16, 4 for f32) and only the 4-byte lo
// parts pass from one launch to the next: a middle launch of a u16 frame
// moves 2 + 4 bytes in and 4 out per pixel.
//
// Two kernels share one per-pixel update (so their results are bit-identical):
//  * k_diffuse_tiles: temporal blocking.  A CTA loads a (dx+2T) x (dy+2T) tile
//    with a T-pixel halo into shared memory, runs T Jacobi iterations there on
//    a shrinking region, and writes the dx x dy interior.  Tiles of every
//    frame of a batch form one grid (a frame table maps tile -> frame).
//  * k_diffuse_stream: one iteration per launch over one frame, one pass over
//    HBM.
// Holes and pixels outside the image hold the sentinel HOLE = 1e30 as hi:
// across a link to it the difference x is about 1e30, x*x overflows to +inf,
// 2^(x*x*c) is exactly +0 and so is the flux g(x) x -- the ghost rule
// J_q = I_p of the oracle (no flux across a hole or the border) without a
// branch; a hole receives only zero fluxes and keeps its value.  The last
// launch writes FP32 depth (hi + lo rounded to nearest; HOLE -> 0).
#define PM_FILE_ID 1
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

// PM4 update from the four link fluxes: I' = I + lambda * (((f_N + f_S) + f_W)
// + f_E) (a HOLE pixel receives only zero fluxes and keeps its value).
__device__ __forceinline__ float2 pm4_combine(float2 Ip, float fN, float fS, float fW, float fE,
                                              float lam)
{
    return pair_add(Ip, __fmul_rn(lam, __fadd_rn(__fadd_rn(__fadd_rn(fN, fS), fW), fE)));
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

// ---------------------------------------------------------------------------
// the sensor encoding: each pixel read as a 32-bit container (the u16 code,
// the f16 bits or the f32 bits); a pixel outside the image reads as 0, which
// decodes to a hole in every encoding
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned load_raw(const DiffFrame &f, int x, int y)
{
    if (!(PM_INB(y, f.h) && PM_INB(x, f.w)))
        return 0u;
    const char *row = (const char *)f.src + (long long)y * f.src_pitch;
    if (f.src_dtype == PM_F32_M)
        return __float_as_uint(__ldg(reinterpret_cast<const float *>(row) + x));
    return __ldg(reinterpret_cast<const unsigned short *>(row) + x);
}

// Raw container -> (hi, decode tail); holes (0, negative, non-finite) ->
// (HOLE, 0).  u16: q * scale split exactly (q has at most 16 significant
// bits, so the product fits in 40 bits and the fused multiply-add returns its
// exact tail).
template <int DT>
__device__ __forceinline__ float2 decode(unsigned r, float scale)
{
    if (DT == PM_U16_MM) {
        if (!r)
            return make_float2(HOLE, 0.0f);
        // q exactly as a float: the bits of 2^23 + q (q < 2^16) minus 2^23
        const float qf = __fsub_rn(__uint_as_float(0x4B000000u | r), 8388608.0f);
        const float hi = __fmul_rn(qf, scale);
        return make_float2(hi, __fmaf_rn(qf, scale, -hi));
    }
    const float v = DT == PM_F16_M ? __half2float(__ushort_as_half((unsigned short)r))
                                   : __uint_as_float(r);
    return make_float2((v > 0.0f && v < __int_as_float(0x7f800000)) ? v : HOLE, 0.0f);
}

__device__ __forceinline__ float2 decode_rt(unsigned r, int dt, float scale)
{
    return dt == PM_U16_MM ? decode<PM_U16_MM>(r, scale)
         : dt == PM_F16_M ? decode<PM_F16_M>(r, scale) : decode<PM_F32_M>(r, scale);
}

__device__ __forceinline__ float depth_out(float2 v)
{
    return v.x == HOLE ? 0.0f : __fadd_rn(v.x, v.y);
}

// ---------------------------------------------------------------------------
// temporal blocking
// ---------------------------------------------------------------------------

// Block = 32 x 8 threads; tile = dx x dy output pixels with a T-pixel halo,
// (dx + 2T) x (dy + 2T) cells in shared memory: the hi parts once (they never
// change), the lo parts in two buffers (12 bytes per cell).  Iteration it
// updates the region shrunk by it + 1 on every side.  Each warp (one
// threadIdx.y) walks a band of rows top to bottom for its columns (lane,
// lane + 32, ...): the south link flux of a row is the negated north link flux
// of the next row (exactly, see link_flux), so each pixel evaluates three
// links (N reused) instead of four.
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

    // the tile with its halo: per warp two rows of 96 cells (encoding and lo
    // parts) in flight before any shared-memory store
    {
        constexpr int G = 3;
        const bool has_lo = f.lo_in != nullptr;
        for (int y0 = wy; y0 < SY; y0 += 16) {
            for (int x0 = 0; x0 < SX; x0 += 32 * G) {
                unsigned rv[2][G];
                float lv[2][G];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int y = y0 + 8 * r, gy = ty0 - T + y;
                    const bool row_ok = y < SY && gy >= 0 && gy < f.h;
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int x = x0 + lane + 32 * g, gx = tx0 - T + x;
                        const bool ok = row_ok && x < SX && gx >= 0 && gx < f.w;
                        rv[r][g] = ok ? load_raw(f, gx, gy) : 0u;
                        lv[r][g] = ok && has_lo && PM_INB((long long)gy * f.w + gx, (long long)f.w * f.h)
                                       ? __ldg(f.lo_in + (long long)gy * f.w + gx) : 0.0f;
                    }
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int y = y0 + 8 * r;
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int x = x0 + lane + 32 * g;
                        if (y < SY && x < SX && PM_INB(y * SX + x, NC)) {
                            const float2 v = decode_rt(rv[r][g], f.src_dtype, f.scale);
                            Hs[y * SX + x] = v.x;
                            A[y * SX + x] = has_lo ? lv[r][g] : v.y;
                        }
                    }
                }
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
            if (gx < f.w && PM_INB((long long)gy * f.w + gx, (long long)f.w * f.h) && PM_INB(k, NC))
                f.dst[(long long)gy * f.w + gx] =
                    f.dst_lo ? A[k] : depth_out(make_float2(Hs[k], A[k]));
        }
    }
}

// ---------------------------------------------------------------------------
// temporal blocking in registers (mode PM4)
// ---------------------------------------------------------------------------

// Packed pairs of FP32 values: one 64-bit register pair, low word first.  The
// sm_100-family f32x2 instructions round each half exactly as the scalar
// instruction does, so a packed update is bit-identical to two scalar ones.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 unpk(f2 v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ float lo_of(f2 v) { return unpk(v).x; }
__device__ __forceinline__ float hi_of(f2 v) { return unpk(v).y; }
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 neg2(f2 a) { return a ^ 0x8000000080000000ull; }
// a b rounded once, for a product that feeds an addition: two scalar
// multiplies.  The compiler may fuse a packed multiply into the packed
// addition that consumes it (one rounding instead of two), which would break
// the bit-identity with the scalar kernels; scalar multiplies followed by a
// packed addition are kept apart.
__device__ __forceinline__ f2 mulr2(f2 a, f2 b)
{
    const float2 x = unpk(a), y = unpk(b);
    return pk(__fmul_rn(x.x, y.x), __fmul_rn(x.y, y.y));
}

// Two link fluxes at once, each exactly link_flux(p, q) of its half:
// x = (hi_q - hi_p) + (lo_q - lo_p), g = 2^(x x c), flux g x.
__device__ __forceinline__ f2 link_flux2(f2 ph, f2 pl, f2 qh, f2 ql, f2 c2)
{
    const f2 x = add2(sub2(qh, ph), sub2(ql, pl));
    const f2 t = mul2(mul2(x, x), c2);
    return mulr2(pk(ex2_approx(lo_of(t)), ex2_approx(hi_of(t))), x);
}

// Block = 8 warps; tile = 128 columns (4 per lane) x 8R rows (R per warp),
// with a T-cell halo on every side, so the output is (128 - 2T) x (8R - 2T)
// pixels.  Every thread keeps its 4 x R cells (hi and lo, as packed pairs of
// columns 0-1 and 2-3) in registers for all T iterations of the launch: the
// horizontal neighbours come from the adjacent lanes by shuffle, the vertical
// ones from the thread's own rows,
// except across the boundary between two warps, whose rows pass through
// shared memory once per iteration (double-buffered: one barrier per
// iteration).  Each warp walks its rows top to bottom with the north flux of
// a row the negated south flux of the row above, and each lane evaluates the
// five horizontal links of its columns once (exactly antisymmetric, see
// link_flux), so the fluxes and their order of summation are those of the
// other kernels: the results are bit-identical.  Every cell of the tile is
// updated every iteration; those outside the region an iteration can update
// exactly (the ring of width it + 1) come out wrong, but only cells further
// out read them, and the output region lies inside every iteration's exact
// region.
template <int R>
__global__ void __launch_bounds__(256, 3) k_diffuse_regs(const DiffFrame *__restrict__ frames,
                                                          int n_frames, int T, float lam, float c)
{
    __shared__ float4 hs[8 * R][32];            // hi parts: [tile row][lane] (4 columns)
    __shared__ float4 bnd_lo[2][2][8][32];      // [buffer][first / last row][warp][lane]
    const int tile = blockIdx.x;
    int lo_f = 0, hi_f = n_frames - 1;
    while (lo_f < hi_f) {
        int mid = (lo_f + hi_f + 1) >> 1;
        if (frames[mid].tile_begin <= tile)
            lo_f = mid;
        else
            hi_f = mid - 1;
    }
    const DiffFrame f = frames[lo_f];
    const int DX = 128 - 2 * T, DY = 8 * R - 2 * T;
    const int tl = tile - f.tile_begin;
    const int tx0 = (tl % f.tiles_x) * DX - T;    // tile column of cell column 0
    const int ty0 = (tl / f.tiles_x) * DY - T;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int x0 = tx0 + 4 * lane;
    const bool has_lo = f.lo_in != nullptr;

    f2 l01[R], l23[R];                          // the thread's lo parts, row r
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gy = ty0 + w * R + r;
        float hv[4], lv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int gx = x0 + k;
            const bool ok = gy >= 0 && gy < f.h && gx >= 0 && gx < f.w;
            const float2 d = decode_rt(ok ? load_raw(f, gx, gy) : 0u, f.src_dtype, f.scale);
            hv[k] = d.x;
            lv[k] = has_lo ? (ok && PM_INB((long long)gy * f.w + gx, (long long)f.w * f.h)
                                  ? __ldg(f.lo_in + (long long)gy * f.w + gx) : 0.0f)
                           : d.y;
        }
        hs[w * R + r][lane] = make_float4(hv[0], hv[1], hv[2], hv[3]);
        l01[r] = pk(lv[0], lv[1]);
        l23[r] = pk(lv[2], lv[3]);
    }
    const float4 HOLE4 = make_float4(HOLE, HOLE, HOLE, HOLE);
    const f2 c2 = pk(c, c), lam2 = pk(lam, lam);
    constexpr int H2 = R / 2;
    for (int it = 0; it < f.n_iters; ++it) {
        const int buf = it & 1;
        bnd_lo[buf][0][w][lane] = make_float4(lo_of(l01[0]), hi_of(l01[0]), lo_of(l23[0]),
                                              hi_of(l23[0]));
        bnd_lo[buf][1][w][lane] = make_float4(lo_of(l01[R - 1]), hi_of(l01[R - 1]),
                                              lo_of(l23[R - 1]), hi_of(l23[R - 1]));
        __syncthreads();   // (the first one also publishes the hi tile)
        const float4 a = w > 0 ? bnd_lo[buf][1][w - 1][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = w < 7 ? bnd_lo[buf][0][w + 1][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hn = w > 0 ? hs[w * R - 1][lane] : HOLE4;
        const float4 hsb = w < 7 ? hs[w * R + R][lane] : HOLE4;
        // Two chains walk the warp's rows top to bottom, rows [0, H2) and
        // [H2, R), independent of each other (more instructions in flight).
        // The flux between rows H2 - 1 and H2 is taken before either is
        // updated: it is the second chain's first north flux and, negated,
        // the first chain's last south flux.
        float4 hc[2], hb = hs[w * R + H2 - 1][lane];
        hc[0] = hs[w * R][lane];
        hc[1] = hs[w * R + H2][lane];
        const f2 fB01 = link_flux2(pk(hc[1].x, hc[1].y), l01[H2], pk(hb.x, hb.y), l01[H2 - 1], c2);
        const f2 fB23 = link_flux2(pk(hc[1].z, hc[1].w), l23[H2], pk(hb.z, hb.w), l23[H2 - 1], c2);
        f2 fN01[2], fN23[2];
        fN01[0] = link_flux2(pk(hc[0].x, hc[0].y), l01[0], pk(hn.x, hn.y), pk(a.x, a.y), c2);
        fN23[0] = link_flux2(pk(hc[0].z, hc[0].w), l23[0], pk(hn.z, hn.w), pk(a.z, a.w), c2);
        fN01[1] = fB01;
        fN23[1] = fB23;
#pragma unroll
        for (int j = 0; j < H2; ++j) {
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                const int r = ch * H2 + j;
                const float4 h = hc[ch];
                const f2 h01 = pk(h.x, h.y), h23 = pk(h.z, h.w);
                float4 hnext = h;   // hi of row r + 1 (the next step's row)
                f2 fS01, fS23;
                if (j + 1 < H2) {
                    const int rs = j + 1 < H2 ? r + 1 : r;
                    hnext = hs[w * R + rs][lane];
                    fS01 = link_flux2(h01, l01[r], pk(hnext.x, hnext.y), l01[rs], c2);
                    fS23 = link_flux2(h23, l23[r], pk(hnext.z, hnext.w), l23[rs], c2);
                } else if (ch == 0) {
                    fS01 = neg2(fB01);
                    fS23 = neg2(fB23);
                } else {
                    fS01 = link_flux2(h01, l01[r], pk(hsb.x, hsb.y), pk(b.x, b.y), c2);
                    fS23 = link_flux2(h23, l23[r], pk(hsb.z, hsb.w), pk(b.z, b.w), c2);
                }
                // the column left of the lane's and right of it (lanes 0 and
                // 31: outside the tile, holes)
                float hW = __shfl_up_sync(0xffffffffu, h.w, 1);
                float hE = __shfl_down_sync(0xffffffffu, h.x, 1);
                float lW = __shfl_up_sync(0xffffffffu, hi_of(l23[r]), 1);
                float lE = __shfl_down_sync(0xffffffffu, lo_of(l01[r]), 1);
                if (lane == 0) {
                    hW = HOLE;
                    lW = 0.0f;
                }
                if (lane == 31) {
                    hE = HOLE;
                    lE = 0.0f;
                }
                const float v0 = lo_of(l01[r]), v1 = hi_of(l01[r]), v2 = lo_of(l23[r]),
                            v3 = hi_of(l23[r]);
                // horizontal: (W of column 0, E of column 3) and (0-1, 2-3)
                // packed, 1-2 alone
                const f2 fWE = link_flux2(pk(h.x, h.w), pk(v0, v3), pk(hW, hE), pk(lW, lE), c2);
                const f2 fIn = link_flux2(pk(h.x, h.z), pk(v0, v2), pk(h.y, h.w), pk(v1, v3), c2);
                const float f12 = link_flux(make_float2(h.y, v1), make_float2(h.z, v2), c);
                const float fW0 = lo_of(fWE), fE3 = hi_of(fWE);
                const float f01 = lo_of(fIn), f23 = hi_of(fIn);
                // column k: W flux, then E flux, as pm4_combine sums them
                const f2 fW01 = pk(fW0, -f01), fE01 = pk(f01, f12);
                const f2 fW23 = pk(-f12, -f23), fE23 = pk(f23, fE3);
                l01[r] = add2(l01[r], mulr2(lam2, add2(add2(add2(fN01[ch], fS01), fW01), fE01)));
                l23[r] = add2(l23[r], mulr2(lam2, add2(add2(add2(fN23[ch], fS23), fW23), fE23)));
                fN01[ch] = neg2(fS01);
                fN23[ch] = neg2(fS23);
                hc[ch] = hnext;
            }
        }
    }
    // the output region: rows [T, 8R - T), columns [T, 128 - T) of the tile
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ty = w * R + r;
        const int gy = ty0 + ty;
        if (ty < T || ty >= 8 * R - T || gy >= f.h)
            continue;
        const float4 h = hs[ty][lane];
        const float hv[4] = {h.x, h.y, h.z, h.w};
        const float lv[4] = {lo_of(l01[r]), hi_of(l01[r]), lo_of(l23[r]), hi_of(l23[r])};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int tx = 4 * lane + k, gx = x0 + k;
            if (tx >= T && tx < 128 - T && gx < f.w &&
                PM_INB((long long)gy * f.w + gx, (long long)f.w * f.h))
                f.dst[(long long)gy * f.w + gx] =
                    f.dst_lo ? lv[k] : depth_out(make_float2(hv[k], lv[k]));
        }
    }
}

// ---------------------------------------------------------------------------
// one iteration per launch, one pass over HBM
// ---------------------------------------------------------------------------

// Block = 32 x 8 threads, 8 independent warps.  The image is cut into strips
// of 32 SC columns (SC = 8 for the 2-byte encodings, 4 for FP32: 16-byte
// loads of the encoding either way) and bands of `rows` rows; block b takes
// strip b % strips and the 8 bands 8 (b / strips) .. + 7, one per warp (the
// blocks of a wave cover a contiguous slab of rows across the whole width).
// Lane l covers columns x0 = 32 SC strip + SC l .. x0 + SC - 1 and walks its
// band down.  The host picks the band height so that the blocks fill the
// resident CTAs in whole waves as nearly as it can.  The north link flux of
// a row is the negated south link flux of the row before and the links
// inside a lane's columns are evaluated once (exactly antisymmetric, see
// link_flux); the horizontal neighbours come from the adjacent lanes by
// shuffle, and lanes 0 and 31 read the column just outside the warp.  Every
// link enters the sum of pm4_combine with the same value and in the same
// order as in the tiled kernels, so the results are bit-identical.  Two rows
// below the current one are in flight while it is computed, and the row
// STREAM_PF further down is prefetched into L2.
constexpr int STREAM_PF = 2;

template <int DT>
__host__ __device__ constexpr int stream_cols() { return DT == PM_F32_M ? 4 : 8; }
// resident CTAs per SM the register budget is fitted to (8 columns per lane
// need about 128 registers, 4 fit in 80)
template <int DT>
__host__ __device__ constexpr int stream_min_ctas() { return DT == PM_F32_M ? 3 : 2; }

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// One row of a lane's columns as read from memory: encoding containers, lo
// parts, and the column outside the warp (lanes 0 and 31).
template <int SC>
struct RowRaw {
    unsigned r[SC];
    float l[SC];
    unsigned re;
    float le;
};

template <int DT, bool HAS_LO, int SC>
__device__ __forceinline__ void load_row(const DiffFrame &f, int y, int x0, int xe, bool edge,
                                         bool vsrc, bool vlo, RowRaw<SC> &o)
{
#pragma unroll
    for (int k = 0; k < SC; ++k) {
        o.r[k] = 0u;
        o.l[k] = 0.0f;
    }
    o.re = 0u;
    o.le = 0.0f;
    if (y < 0 || y >= f.h)
        return;
    const char *row = (const char *)f.src + (long long)y * f.src_pitch;
    const bool full = x0 + SC <= f.w;
    if (full && vsrc && PM_INB(x0 + SC - 1, f.w) && PM_INB(x0, f.w)) {
        // 16 bytes: 8 two-byte codes or 4 FP32 values
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(row) + x0 / SC);
        const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < SC; ++k)
            o.r[k] = SC == 8 ? ((k & 1) ? u[k >> 1] >> 16 : u[k >> 1] & 0xffffu) : u[k];
    } else {
#pragma unroll
        for (int k = 0; k < SC; ++k)
            if (x0 + k < f.w)
                o.r[k] = load_raw(f, x0 + k, y);
    }
    if (HAS_LO) {
        const float *lrow = f.lo_in + (long long)y * f.w;
        if (full && vlo && PM_INB(x0 + SC - 1, f.w) && PM_INB(x0, f.w)) {
#pragma unroll
            for (int q = 0; q < SC / 4; ++q) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(lrow + x0) + q);
                o.l[4 * q] = v.x;
                o.l[4 * q + 1] = v.y;
                o.l[4 * q + 2] = v.z;
                o.l[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < SC; ++k)
                if (x0 + k < f.w && PM_INB(x0 + k, f.w))
                    o.l[k] = __ldg(lrow + x0 + k);
        }
        if (edge && PM_INB(xe, f.w))
            o.le = __ldg(lrow + xe);
    }
    if (edge)
        o.re = load_raw(f, xe, y);
}

template <int DT, bool HAS_LO, int SC>
__device__ __forceinline__ void decode_row(const RowRaw<SC> &o, float scale, float2 (&a)[SC],
                                           float2 &e)
{
#pragma unroll
    for (int k = 0; k < SC; ++k) {
        a[k] = decode<DT>(o.r[k], scale);
        if (HAS_LO)
            a[k].y = o.l[k];
    }
    e = decode<DT>(o.re, scale);
    if (HAS_LO)
        e.y = o.le;
}

// State of a lane walking down its columns: the row being computed (a, with
// the column outside the warp ae), the row above (u, for the Alg. 1 form) and
// the north fluxes of the row in packed column pairs (PM4).
template <int SC>
struct StreamState {
    float2 u[SC], a[SC], ae;
    f2 fN[SC / 2];
};

// Row y of the lane's columns from the rows above (in S) and the decoded row
// below (d, with the column outside the warp de); written out, then S moves
// down one row.
template <int MODE, int DT, bool DST_LO, int SC>
__device__ __forceinline__ void stream_compute(const DiffFrame &f, int y, int x0, bool edge,
                                               bool vdst, int lane, float lam, float c,
                                               const float2 (&d)[SC], float2 de,
                                               StreamState<SC> &S)
{
    const float2 Z = make_float2(HOLE, 0.0f);
    float2 L = make_float2(__shfl_up_sync(0xffffffffu, S.a[SC - 1].x, 1),
                           __shfl_up_sync(0xffffffffu, S.a[SC - 1].y, 1));
    float2 R = make_float2(__shfl_down_sync(0xffffffffu, S.a[0].x, 1),
                           __shfl_down_sync(0xffffffffu, S.a[0].y, 1));
    if (lane == 0)
        L = edge ? S.ae : Z;
    if (lane == 31)
        R = edge ? S.ae : Z;
    float2 n[SC];
    if (MODE == 0) {
        // fH[k]: the flux into column k from column k - 1 (fH[0] from L;
        // fH[SC] into the last column from R), each exactly the link_flux of
        // the scalar kernels, evaluated in packed pairs
        const float2 *a = S.a;
        const f2 c2 = pk(c, c), lam2 = pk(lam, lam);
        float fH[SC + 1];
        {
            const f2 e = link_flux2(pk(a[0].x, a[SC - 1].x), pk(a[0].y, a[SC - 1].y),
                                    pk(L.x, R.x), pk(L.y, R.y), c2);
            fH[0] = lo_of(e);
            fH[SC] = hi_of(e);
        }
#pragma unroll
        for (int k = 1; k + 1 < SC; k += 2) {
            const f2 e = link_flux2(pk(a[k].x, a[k + 1].x), pk(a[k].y, a[k + 1].y),
                                    pk(a[k - 1].x, a[k].x), pk(a[k - 1].y, a[k].y), c2);
            fH[k] = lo_of(e);
            fH[k + 1] = hi_of(e);
        }
        fH[SC - 1] = link_flux(a[SC - 1], a[SC - 2], c);
#pragma unroll
        for (int q = 0; q < SC / 2; ++q) {
            const int k = 2 * q;
            const f2 fS = link_flux2(pk(a[k].x, a[k + 1].x), pk(a[k].y, a[k + 1].y),
                                     pk(d[k].x, d[k + 1].x), pk(d[k].y, d[k + 1].y), c2);
            // column k: W flux fH[k], E flux -fH[k + 1] (the last column: fH[SC])
            const f2 fW = pk(fH[k], fH[k + 1]);
            const f2 fE = pk(-fH[k + 1], k + 2 < SC ? -fH[k + 2] : fH[SC]);
            const f2 l = add2(pk(a[k].y, a[k + 1].y),
                              mulr2(lam2, add2(add2(add2(S.fN[q], fS), fW), fE)));
            n[k] = make_float2(a[k].x, lo_of(l));
            n[k + 1] = make_float2(a[k + 1].x, hi_of(l));
            S.fN[q] = neg2(fS);
        }
    } else {
#pragma unroll
        for (int k = 0; k < SC; ++k)
            n[k] = update_alg1(S.a[k], S.u[k], d[k], k ? S.a[k - 1] : L,
                               k + 1 < SC ? S.a[k + 1] : R, lam, c);
    }
    if (f.n_iters == 0) {
#pragma unroll
        for (int k = 0; k < SC; ++k)
            n[k] = S.a[k];
    }
    float o[SC];
#pragma unroll
    for (int k = 0; k < SC; ++k)
        o[k] = DST_LO ? n[k].y : depth_out(n[k]);
    float *drow = f.dst + (long long)y * f.w;
    if (PM_INB(y, f.h)) {
        if (vdst && x0 + SC <= f.w && PM_INB(x0, f.w)) {
#pragma unroll
            for (int q = 0; q < SC / 4; ++q)
                reinterpret_cast<float4 *>(drow + x0)[q] =
                    make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < SC; ++k)
                if (x0 + k < f.w)
                    drow[x0 + k] = o[k];
        }
    }
#pragma unroll
    for (int k = 0; k < SC; ++k) {
        S.u[k] = S.a[k];
        S.a[k] = d[k];
    }
    S.ae = de;
}

// Row y with its row below already read into `below`, which is refilled
// with row y + 3 (the row read two steps ahead) when `more`.
template <int MODE, int DT, bool HAS_LO, bool DST_LO, int SC>
__device__ __forceinline__ void stream_row(const DiffFrame &f, int y, int x0, int xe, bool edge,
                                           bool vsrc, bool vlo, bool vdst, int lane, float lam,
                                           float c, RowRaw<SC> &below, bool more,
                                           StreamState<SC> &S)
{
    float2 d[SC], de;
    decode_row<DT, HAS_LO, SC>(below, f.scale, d, de);
    if (more) {
        load_row<DT, HAS_LO, SC>(f, y + 3, x0, xe, edge, vsrc, vlo, below);
        // the row STREAM_PF below that into L2, one request per 128-byte line
        const int yp = y + 3 + STREAM_PF;
        if (yp < f.h && x0 < f.w) {
            constexpr int SRC_LANES = 128 / (SC * (DT == PM_F32_M ? 4 : 2));
            if (lane % SRC_LANES == 0)
                prefetch_l2((const char *)f.src + (long long)yp * f.src_pitch +
                            (long long)x0 * (DT == PM_F32_M ? 4 : 2));
            if (HAS_LO && lane % (32 / SC) == 0)
                prefetch_l2(f.lo_in + (long long)yp * f.w + x0);
        }
    }
    stream_compute<MODE, DT, DST_LO, SC>(f, y, x0, edge, vdst, lane, lam, c, d, de, S);
}

// One unit: rows y0 .. y0 + rows - 1 of the strip, by one warp.
template <int MODE, int DT, bool HAS_LO, bool DST_LO>
__device__ __forceinline__ void stream_band(const DiffFrame &f, float lam, float c, int strip,
                                            int y0, int rows)
{
    constexpr int SC = stream_cols<DT>();
    const int lane = threadIdx.x;
    const int x0 = strip * (32 * SC) + SC * lane;
    if (y0 >= f.h)
        return;
    const int y1 = min(y0 + rows, f.h);
    constexpr int VB = SC * (DT == PM_F32_M ? 4 : 2);   // bytes of a lane's encoding: 16
    const bool vsrc = ((uintptr_t)f.src % VB) == 0 && f.src_pitch % VB == 0;
    const bool vlo = ((uintptr_t)f.lo_in % 16) == 0 && f.w % 4 == 0;
    const bool vdst = ((uintptr_t)f.dst % 16) == 0 && f.w % 4 == 0;
    // the column just outside the warp: x0 - 1 for lane 0, x0 + SC for lane 31
    const int xe = lane == 0 ? x0 - 1 : x0 + SC;
    const bool edge = (lane == 0 || lane == 31) && xe >= 0 && xe < f.w;

    // two read buffers alternate: while row y is computed, rows y + 1 and
    // y + 2 are in flight
    RowRaw<SC> rA, rB;
    StreamState<SC> S;
    load_row<DT, HAS_LO, SC>(f, y0 - 1, x0, xe, edge, vsrc, vlo, rA);
    load_row<DT, HAS_LO, SC>(f, y0, x0, xe, edge, vsrc, vlo, rB);
    float2 ue;
    decode_row<DT, HAS_LO, SC>(rA, f.scale, S.u, ue);
    decode_row<DT, HAS_LO, SC>(rB, f.scale, S.a, S.ae);
    load_row<DT, HAS_LO, SC>(f, y0 + 1, x0, xe, edge, vsrc, vlo, rA);
    load_row<DT, HAS_LO, SC>(f, y0 + 2, x0, xe, edge, vsrc, vlo, rB);
    if (MODE == 0) {
        const f2 c2 = pk(c, c);
#pragma unroll
        for (int q = 0; q < SC / 2; ++q)
            S.fN[q] = link_flux2(pk(S.a[2 * q].x, S.a[2 * q + 1].x),
                                 pk(S.a[2 * q].y, S.a[2 * q + 1].y),
                                 pk(S.u[2 * q].x, S.u[2 * q + 1].x),
                                 pk(S.u[2 * q].y, S.u[2 * q + 1].y), c2);
    }
    for (int y = y0; y < y1; y += 2) {
        stream_row<MODE, DT, HAS_LO, DST_LO, SC>(f, y, x0, xe, edge, vsrc, vlo, vdst, lane, lam,
                                                 c, rA, y + 2 < y1, S);
        if (y + 1 >= y1)
            break;
        stream_row<MODE, DT, HAS_LO, DST_LO, SC>(f, y + 1, x0, xe, edge, vsrc, vlo, vdst, lane,
                                                 lam, c, rB, y + 3 < y1, S);
    }
}

template <int MODE, int DT, bool HAS_LO, bool DST_LO>
__global__ void __launch_bounds__(256, stream_min_ctas<DT>()) k_diffuse_stream(DiffFrame f,
                                                                              float lam, float c,
                                                                              int rows, int strips,
                                                                              int strip0)
{
    const int group = blockIdx.x / strips;
    stream_band<MODE, DT, HAS_LO, DST_LO>(f, lam, c, strip0 + blockIdx.x - group * strips,
                                          (group * 8 + threadIdx.y) * rows, rows);
}

// ---------------------------------------------------------------------------
// the same walk with the rows staged in shared memory by asynchronous copies
// ---------------------------------------------------------------------------
// For FP32 frames whose strips are whole and whose rows are 16-byte aligned,
// each warp keeps a ring of STREAM_RING rows of its strip in shared memory,
// filled with cp.async (16-byte pieces: every lane copies its own encoding,
// lo parts and, for lanes 0 and 31, the 4-byte word of the column outside the
// warp): STREAM_RING - 1 rows are in flight while a row is computed, without
// holding them in registers.  A lane reads back only what it copied itself,
// so cp.async.wait_group alone orders the copies and the reads.  The rows
// read back are exactly those load_row returns, so the arithmetic and the
// results are those of the register walk.  (Timed on 8192 x 8192, 10
// iterations: FP32 0.563 of the HBM peak on algorithmic bytes with registers,
// 0.623 with a 4-row ring, 0.605 with 6, 0.558 with 8; the 2-byte encodings
// reached 0.58 with a ring against 0.63 with registers in one wave, so they
// keep the register walk.)
constexpr int STREAM_RING = 4;

template <int SC>
struct RingSlot {
    static constexpr int SRC = 32 * 16;       // the lanes' encoding, 16 bytes each
    static constexpr int LO = 32 * SC * 4;    // lo parts: SC / 4 planes of 32 x 16 bytes
    static constexpr int EDGE = 32 * 8;       // container word and lo part of the outside column
    static constexpr int BYTES = SRC + LO + EDGE;
};

template <int DT>
constexpr size_t stream_ring_smem() { return (size_t)8 * STREAM_RING * RingSlot<stream_cols<DT>()>::BYTES; }

// resident CTAs per SM the ring kernel's registers are fitted to
template <int DT>
__host__ __device__ constexpr int stream_ring_ctas() { return DT == PM_F32_M ? 3 : 2; }

__device__ __forceinline__ void cp_async16(unsigned saddr, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}

__device__ __forceinline__ void cp_async4(unsigned saddr, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(g) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Row y of the lane's columns into the ring slot at shared address sb (rows
// outside the image are not copied: ring_read returns zeros for them).
template <int DT, bool HAS_LO, int SC>
__device__ __forceinline__ void ring_issue(const DiffFrame &f, int y, int x0, int xe, bool edge,
                                           int lane, unsigned sb)
{
    if (y < 0 || y >= f.h || !PM_INB(x0 + SC - 1, f.w))
        return;
    constexpr int ES = DT == PM_F32_M ? 4 : 2;
    const char *row = (const char *)f.src + (long long)y * f.src_pitch;
    cp_async16(sb + lane * 16, row + (long long)x0 * ES);
    if (HAS_LO) {
        const float *lrow = f.lo_in + (long long)y * f.w + x0;
#pragma unroll
        for (int q = 0; q < SC / 4; ++q)
            cp_async16(sb + RingSlot<SC>::SRC + q * 512 + lane * 16, lrow + 4 * q);
    }
    if (edge && PM_INB(xe, f.w)) {
        // the aligned 4-byte word holding column xe (for a 2-byte encoding the
        // frame's width is a multiple of 8, so the word lies inside the row)
        const long long xb = ((long long)xe * ES) & ~3ll;
        const unsigned se = sb + RingSlot<SC>::SRC + RingSlot<SC>::LO + lane * 8;
        cp_async4(se, row + xb);
        if (HAS_LO)
            cp_async4(se + 4, f.lo_in + (long long)y * f.w + xe);
    }
}

// Row y from the ring slot at sp, as load_row would read it.
template <int DT, bool HAS_LO, int SC>
__device__ __forceinline__ void ring_read(const DiffFrame &f, int y, int xe, bool edge, int lane,
                                          const unsigned char *sp, RowRaw<SC> &o)
{
#pragma unroll
    for (int k = 0; k < SC; ++k) {
        o.r[k] = 0u;
        o.l[k] = 0.0f;
    }
    o.re = 0u;
    o.le = 0.0f;
    if (y < 0 || y >= f.h)
        return;
    const uint4 v = *reinterpret_cast<const uint4 *>(sp + lane * 16);
    const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < SC; ++k)
        o.r[k] = SC == 8 ? ((k & 1) ? u[k >> 1] >> 16 : u[k >> 1] & 0xffffu) : u[k];
    if (HAS_LO) {
#pragma unroll
        for (int q = 0; q < SC / 4; ++q) {
            const float4 l = *reinterpret_cast<const float4 *>(sp + RingSlot<SC>::SRC + q * 512 +
                                                               lane * 16);
            o.l[4 * q] = l.x;
            o.l[4 * q + 1] = l.y;
            o.l[4 * q + 2] = l.z;
            o.l[4 * q + 3] = l.w;
        }
    }
    if (edge) {
        const unsigned char *e = sp + RingSlot<SC>::SRC + RingSlot<SC>::LO + lane * 8;
        const unsigned wv = *reinterpret_cast<const unsigned *>(e);
        o.re = DT == PM_F32_M ? wv : ((xe & 1) ? wv >> 16 : wv & 0xffffu);
        if (HAS_LO)
            o.le = *reinterpret_cast<const float *>(e + 4);
    }
}

// One band of a whole strip through the warp's ring (ring: shared address,
// sp: the same memory as a generic pointer).  Row r lives in slot
// (r - y0 + 1) % STREAM_RING; one copy group is committed per row, so
// waiting for all but the STREAM_RING - 2 newest groups completes the row
// below the one computed.
template <int MODE, int DT, bool HAS_LO, bool DST_LO>
__device__ __forceinline__ void stream_band_ring(const DiffFrame &f, float lam, float c, int strip,
                                                 int y0, int rows, unsigned ring,
                                                 const unsigned char *sp)
{
    constexpr int SC = stream_cols<DT>();
    constexpr int P = STREAM_RING;
    constexpr int SB = RingSlot<SC>::BYTES;
    const int lane = threadIdx.x;
    const int x0 = strip * (32 * SC) + SC * lane;
    if (y0 >= f.h)
        return;
    const int y1 = min(y0 + rows, f.h);
    const int xe = lane == 0 ? x0 - 1 : x0 + SC;
    const bool edge = (lane == 0 || lane == 31) && xe >= 0 && xe < f.w;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        if (y0 - 1 + i <= y1)
            ring_issue<DT, HAS_LO, SC>(f, y0 - 1 + i, x0, xe, edge, lane, ring + i * SB);
        cp_async_commit();
    }
    cp_async_wait<P - 2>();
    RowRaw<SC> r;
    StreamState<SC> S;
    float2 ue;
    ring_read<DT, HAS_LO, SC>(f, y0 - 1, xe, edge, lane, sp, r);
    decode_row<DT, HAS_LO, SC>(r, f.scale, S.u, ue);
    ring_read<DT, HAS_LO, SC>(f, y0, xe, edge, lane, sp + SB, r);
    decode_row<DT, HAS_LO, SC>(r, f.scale, S.a, S.ae);
    if (y0 + P - 1 <= y1)
        ring_issue<DT, HAS_LO, SC>(f, y0 + P - 1, x0, xe, edge, lane, ring);
    cp_async_commit();
    if (MODE == 0) {
        const f2 c2 = pk(c, c);
#pragma unroll
        for (int q = 0; q < SC / 2; ++q)
            S.fN[q] = link_flux2(pk(S.a[2 * q].x, S.a[2 * q + 1].x),
                                 pk(S.a[2 * q].y, S.a[2 * q + 1].y),
                                 pk(S.u[2 * q].x, S.u[2 * q + 1].x),
                                 pk(S.u[2 * q].y, S.u[2 * q + 1].y), c2);
    }
    int sl = 2 % P;   // slot of row y + 1
    for (int y = y0; y < y1; ++y) {
        cp_async_wait<P - 2>();
        ring_read<DT, HAS_LO, SC>(f, y + 1, xe, edge, lane, sp + sl * SB, r);
        // row y's slot (read one step earlier) takes row y + P
        const int sr = sl == 0 ? P - 1 : sl - 1;
        if (y + P <= y1)
            ring_issue<DT, HAS_LO, SC>(f, y + P, x0, xe, edge, lane, ring + sr * SB);
        cp_async_commit();
        float2 d[SC], de;
        decode_row<DT, HAS_LO, SC>(r, f.scale, d, de);
        stream_compute<MODE, DT, DST_LO, SC>(f, y, x0, edge, true, lane, lam, c, d, de, S);
        sl = sl + 1 == P ? 0 : sl + 1;
    }
    cp_async_wait<0>();
}

template <int MODE, int DT, bool HAS_LO, bool DST_LO>
__global__ void __launch_bounds__(256, stream_ring_ctas<DT>())
    k_diffuse_stream_ring(DiffFrame f, float lam, float c, int rows, int strips)
{
    extern __shared__ __align__(16) unsigned char ring_sm[];
    constexpr int SB = RingSlot<stream_cols<DT>()>::BYTES;
    const int group = blockIdx.x / strips;
    const unsigned char *sp = ring_sm + threadIdx.y * STREAM_RING * SB;
    stream_band_ring<MODE, DT, HAS_LO, DST_LO>(
        f, lam, c, blockIdx.x - group * strips, (group * 8 + threadIdx.y) * rows, rows,
        (unsigned)__cvta_generic_to_shared(sp), sp);
}

static inline float conductance_scale(float K)
{
    // exp(-(x/K)^2) = 2^(x^2 * c) with c = -log2(e) / K^2
    return (float)(-1.4426950408889634 / ((double)K * (double)K));
}

int regs_rows(int mode, int T, int dx, int dy)
{
    if (mode != 0 || T < 1 || dx != 128 - 2 * T)
        return 0;
    for (int R = 4; R <= 8; R += 2)
        if (dy == 8 * R - 2 * T)
            return R;
    return 0;
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
    const int R = regs_rows(mode, T, dx, dy);
    if (R == 4)
        k_diffuse_regs<4><<<total_tiles, block, 0, s>>>(d_frames, n_frames, T, lambda, c);
    else if (R == 6)
        k_diffuse_regs<6><<<total_tiles, block, 0, s>>>(d_frames, n_frames, T, lambda, c);
    else if (R == 8)
        k_diffuse_regs<8><<<total_tiles, block, 0, s>>>(d_frames, n_frames, T, lambda, c);
    else if (mode == 0)
        k_diffuse_tiles<0><<<total_tiles, block, smem, s>>>(d_frames, n_frames, T, dx, dy, lambda, c);
    else
        k_diffuse_tiles<1><<<total_tiles, block, smem, s>>>(d_frames, n_frames, T, dx, dy, lambda, c);
    return cudaGetLastError();
}

// The streaming kernel for the launch's iterate input and output (lo parts
// read or not, lo parts or depth written).
// The launch shape of the streaming kernel.  one_wave: bands of at least 8
// rows, as tall as it takes for the blocks to fit the resident CTAs
// (ctas_per_sm on each of the sms SMs) at once.  Otherwise the band height
// in [32, 256] rows whose grid of strips x ceil(h / (8 rows)) blocks fills
// the resident CTAs in whole waves most nearly, the smallest such height on
// ties (images too small to fill one wave with 32-row bands as in one_wave).
// (Timed on 8192 x 8192 u16: one wave of 114-row bands 0.632 of the HBM peak
// on algorithmic bytes, 38-row bands in 2.9 waves 0.588, 32-row bands in 3.5
// waves 0.557.)
struct StreamShape {
    int rows, strips, blocks;
};

StreamShape stream_shape(int w, int h, int sc, int sms, int ctas_per_sm, bool one_wave)
{
    StreamShape sh;
    sh.strips = (w + 32 * sc - 1) / (32 * sc);
    const long long resident = (long long)sms * ctas_per_sm;
    if (one_wave || (long long)sh.strips * ((h + 8LL * 32 - 1) / (8LL * 32)) < resident) {
        const long long per_strip = resident / sh.strips > 0 ? resident / sh.strips : 1;
        long long r = (h + 8 * per_strip - 1) / (8 * per_strip);
        r = r < 8 ? 8 : r;
        sh.rows = (int)(r < h ? r : h);
        sh.blocks = (int)((long long)sh.strips * ((h + 8LL * sh.rows - 1) / (8LL * sh.rows)));
        return sh;
    }
    double best = -1.0;
    sh.rows = 32;
    for (int r = 32; r <= 256; ++r) {
        const long long blocks = (long long)sh.strips * ((h + 8LL * r - 1) / (8LL * r));
        const long long waves = (blocks + resident - 1) / resident;
        const double fill = (double)blocks / (double)(waves * resident);
        if (fill > best + 1e-9) {
            best = fill;
            sh.rows = r;
        }
        if ((h + 8LL * r - 1) / (8LL * r) == 1)
            break;   // one block per strip: taller bands change nothing
    }
    sh.blocks = (int)((long long)sh.strips * ((h + 8LL * sh.rows - 1) / (8LL * sh.rows)));
    return sh;
}

// One launch of the register walk (strips [strip0, strip0 + strips)) or of
// the ring walk, for the launch's iterate input and output (lo parts read or
// not, lo parts or depth written).
template <int M, int DT, bool RING>
static void launch_stream_io(const DiffFrame &f, float lam, float c, const StreamShape &sh,
                             int strip0, cudaStream_t s)
{
    const dim3 block(32, 8);
    const size_t smem = RING ? stream_ring_smem<DT>() : 0;
#define PM_STREAM_LAUNCH(LO, DLO)                                                              \
    do {                                                                                       \
        if constexpr (RING)                                                                    \
            k_diffuse_stream_ring<M, DT, LO, DLO><<<sh.blocks, block, smem, s>>>(             \
                f, lam, c, sh.rows, sh.strips);                                                \
        else                                                                                   \
            k_diffuse_stream<M, DT, LO, DLO><<<sh.blocks, block, 0, s>>>(f, lam, c, sh.rows,  \
                                                                         sh.strips, strip0);   \
    } while (0)
    if (f.lo_in) {
        if (f.dst_lo)
            PM_STREAM_LAUNCH(true, true);
        else
            PM_STREAM_LAUNCH(true, false);
    } else {
        if (f.dst_lo)
            PM_STREAM_LAUNCH(false, true);
        else
            PM_STREAM_LAUNCH(false, false);
    }
#undef PM_STREAM_LAUNCH
}

// FP32 frames with whole, aligned strips: the ring walk over those strips;
// every other strip (and every 2-byte encoding): the register walk in one
// wave.
template <int M, int DT>
static cudaError_t launch_stream_dt(const DiffFrame &f, float lam, float c, int sms,
                                    cudaStream_t s)
{
    constexpr int SC = stream_cols<DT>();
    static_assert(stream_ring_smem<PM_F32_M>() <= 48 * 1024, "ring within the default shared memory");
    const bool aligned = DT == PM_F32_M && ((uintptr_t)f.src % 16) == 0 &&
                         f.src_pitch % 16 == 0 && ((uintptr_t)f.lo_in % 16) == 0 &&
                         ((uintptr_t)f.dst % 16) == 0 && f.w % 4 == 0;
    const int whole = aligned ? f.w / (32 * SC) : 0;
    if (whole > 0) {
        const StreamShape sh =
            stream_shape(whole * 32 * SC, f.h, SC, sms, stream_ring_ctas<DT>(), false);
        launch_stream_io<M, PM_F32_M, true>(f, lam, c, sh, 0, s);
    }
    if (whole * 32 * SC < f.w) {
        const StreamShape sh =
            stream_shape(f.w - whole * 32 * SC, f.h, SC, sms, stream_min_ctas<DT>(), true);
        launch_stream_io<M, DT, false>(f, lam, c, sh, whole, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_diffuse_stream(const DiffFrame &f, float lambda, float K, int mode,
                                  cudaStream_t s)
{
    const float c = conductance_scale(K);
    if (f.src_dtype != PM_U16_MM && f.src_dtype != PM_F16_M && f.src_dtype != PM_F32_M)
        return cudaErrorInvalidValue;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    const int dt = f.src_dtype;
    if (mode == 0) {
        if (dt == PM_U16_MM)
            return launch_stream_dt<0, PM_U16_MM>(f, lambda, c, sms, s);
        if (dt == PM_F16_M)
            return launch_stream_dt<0, PM_F16_M>(f, lambda, c, sms, s);
        return launch_stream_dt<0, PM_F32_M>(f, lambda, c, sms, s);
    }
    if (dt == PM_U16_MM)
        return launch_stream_dt<1, PM_U16_MM>(f, lambda, c, sms, s);
    if (dt == PM_F16_M)
        return launch_stream_dt<1, PM_F16_M>(f, lambda, c, sms, s);
    return launch_stream_dt<1, PM_F32_M>(f, lambda, c, sms, s);
}

PM_BOUNDS_QUERY(bounds_diffuse)

}  // namespace pm

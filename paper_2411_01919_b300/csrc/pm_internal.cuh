// pm_internal.cuh -- device-side structures and helpers shared by the libpm
// kernels (diffusion, normals, RANSAC) and the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/pm.h"

namespace pm {

// ---------------------------------------------------------------------------
// bounds-checking build (PM_DEBUG_BOUNDS): every instrumented global access
// checks its index against the extent of its buffer; the first index outside
// is recorded in a device status word of the translation unit (bit 63 set,
// bits 48-62 the source site: file id and line, bits 0-47 the index) and the
// access is skipped.  Nothing traps.  The release build compiles every check
// to `true`.  pm_debug_bounds (pm_api.cu) reads and clears the words.
// ---------------------------------------------------------------------------
#ifndef PM_FILE_ID
#define PM_FILE_ID 0
#endif
#ifdef PM_DEBUG_BOUNDS
static __device__ unsigned long long g_pm_bounds = 0ull;
__device__ __forceinline__ bool pm_inb(long long i, long long n, int site)
{
    if (i >= 0 && i < n)
        return true;
    atomicCAS(&g_pm_bounds, 0ull,
              0x8000000000000000ull | ((unsigned long long)(site & 0x7fff) << 48) |
                  ((unsigned long long)i & 0xffffffffffffull));
    return false;
}
#define PM_INB(i, n) ::pm::pm_inb((long long)(i), (long long)(n), (PM_FILE_ID << 12) | (__LINE__ & 0xfff))
#define PM_BOUNDS_QUERY(fn)                                                                   \
    cudaError_t fn(unsigned long long *v)                                                     \
    {                                                                                         \
        cudaError_t e = cudaMemcpyFromSymbol(v, g_pm_bounds, sizeof(*v));                     \
        const unsigned long long z = 0ull;                                                    \
        if (e == cudaSuccess && *v)                                                           \
            e = cudaMemcpyToSymbol(g_pm_bounds, &z, sizeof(z));                               \
        return e;                                                                             \
    }
#else
#define PM_INB(i, n) true
#define PM_BOUNDS_QUERY(fn)                                                                   \
    cudaError_t fn(unsigned long long *v)                                                     \
    {                                                                                         \
        *v = 0ull;                                                                            \
        return cudaSuccess;                                                                   \
    }
#endif
// status words of the kernels' translation units
cudaError_t bounds_diffuse(unsigned long long *v);
cudaError_t bounds_normals(unsigned long long *v);
cudaError_t bounds_ransac(unsigned long long *v);

// ---------------------------------------------------------------------------
// compile-time layout constants
// ---------------------------------------------------------------------------
constexpr int CHUNK = 1024;              // candidates per chunk (RANSAC work unit)
constexpr int CHUNK_WORDS = CHUNK / 32;  // keep-bitmask words per chunk
constexpr int MAX_HYP = 2048;            // hypotheses per round (score kernel register budget)
constexpr int MAX_PLANES = 64;
constexpr int NMOM = 9;                  // Sx Sy Sz Sxx Sxy Sxz Syy Syz Szz
constexpr int GROUP = 1;                 // chunks per moment record
constexpr int REMOVE_THREADS = 256;      // threads of the removal kernel (CHUNK / 4 candidates each)
constexpr int REFIT_WARPS = 8;          // warps of a refit block (the scoring and removal block size)
// per-group moment record: gated inliers then the other inliers, each NMOM
// double-float sums (h, l), then two int counts (as float bit patterns),
// padded to 40 words
constexpr int PART_WORDS = 40;

// Diffusion tiles (temporal blocking): output tile dx x dy chosen per launch
// (at most TILE_MAX_DX x TILE_MAX_DY), halo T <= DT_MAX
constexpr int TILE_MAX_DX = 144;
constexpr int TILE_MAX_DY = 64;
constexpr int DT_MAX = 8;

// ---------------------------------------------------------------------------
// per-frame descriptors
// ---------------------------------------------------------------------------

// One frame in one diffusion launch.  The iterate is the compensated pair
// (hi, lo), I = hi + lo: hi is the decoded sensor depth and never changes, so
// every launch decodes it again from the sensor encoding; only lo passes from
// one launch to the next.
struct DiffFrame {
    const void *src;      // sensor encoding, read by every launch (the hi parts)
    int src_dtype;        // PM_U16_MM / PM_F16_M / PM_F32_M
    int w, h;
    long long src_pitch;  // bytes
    const float *lo_in;   // lo parts from the previous launch [h*w], or null (first launch)
    float *dst;           // lo parts [h*w] (dst_lo) or FP32 depth [h*w]
    int dst_lo;           // 1: write the lo parts, 0: write FP32 depth (hi + lo rounded)
    int n_iters;          // iterations this launch (0 = decode only)
    int tiles_x;
    int tile_begin;       // first global tile of this frame
    float scale;          // metres per u16 unit
};

// Per-frame RANSAC state on the device.
struct RState {
    int M;            // candidates in the current list
    int M_next;       // candidates kept for the next round (written by compaction)
    int done;         // 1 once the frame stopped
    int n_planes;
    int nchunks;      // chunks of the current list (0 when done)
    int score_done;   // scoring work items finished this round
    int best_h;
    int best_count;
    // what the refit of an accepted round needs, kept per round parity: the
    // refit of round r runs beside the scoring (and selection) of round r + 1
    int rf_pending[2];  // [round & 1]: 1 from an accepted selection until its refit
    int rf_groups[2];   // moment records of that round
    int rf_h[2];        // its winning hypothesis
    int rf_count[2];    // and the winner's inlier count
    float4 rf_p0[2];    // its first sample point (the moment origin)
    float4 best_plane;
    float4 p0;        // first sample point of the winner (moment origin)
    int m_hist[MAX_PLANES];  // candidates scored in each round (0 once stopped)
    unsigned long long pairs_eval;  // hypothesis-candidate pairs evaluated (not culled)
};

struct RFrame {
    const float *P;           // SoA points [3][npx]
    const float *N;           // SoA normals [3][npx] or nullptr
    const unsigned char *valid;
    short *labels;            // [npx]
    int w, h, npx;
    unsigned long long frame_idx;
    float4 *cpt[2];           // candidates (x, y, z, pixel index as int bits)
    float4 *hyp;              // [H] hypothesis planes (nx, ny, nz, d); d = +inf when degenerate
    float4 *hyp_p0;           // [H] first sample point
    int *counts;              // [H]
    int *kept;                // [max_chunks]
    unsigned *keepbits;       // [max_chunks * CHUNK_WORDS]
    float *partial;           // [ceil(max_chunks / GROUP) * PART_WORDS]
    RState *st;
    pm_plane *planes;         // device [MAX_PLANES]
};

struct RParams {
    int H;
    float thr2;          // thr*thr rounded to FP32
    int max_planes;
    int min_inliers;
    unsigned long long seed;
    float cos_gate;
    float cull_thr;      // >= sqrt(thr2) (1 + 2^-20): box test, no inlier beyond it
    float incl_thr;      // <= sqrt(thr2) (1 - 2^-20): box test, every point inlier below it
};

// ---------------------------------------------------------------------------
// Exactly specified FP32 arithmetic.  The inlier decision decides integers
// (counts, argmax, labels), so it is spelled out operation by operation with
// round-to-nearest intrinsics that the compiler never contracts or reorders.
// ---------------------------------------------------------------------------

// Hypothesis plane through p0, p1, p2: n = (p1-p0) x (p2-p0), |n|^2 summed
// as (x^2 + y^2) + z^2, degenerate if |n|^2 <= 1e-18, n /= sqrt(|n|^2),
// d = -((n.x p0.x + n.y p0.y) + n.z p0.z).
__device__ __forceinline__ bool hyp_plane(float3 a, float3 b, float3 c, float4 &out)
{
    float e1x = __fsub_rn(b.x, a.x), e1y = __fsub_rn(b.y, a.y), e1z = __fsub_rn(b.z, a.z);
    float e2x = __fsub_rn(c.x, a.x), e2y = __fsub_rn(c.y, a.y), e2z = __fsub_rn(c.z, a.z);
    float nx = __fsub_rn(__fmul_rn(e1y, e2z), __fmul_rn(e1z, e2y));
    float ny = __fsub_rn(__fmul_rn(e1z, e2x), __fmul_rn(e1x, e2z));
    float nz = __fsub_rn(__fmul_rn(e1x, e2y), __fmul_rn(e1y, e2x));
    float nn = __fadd_rn(__fadd_rn(__fmul_rn(nx, nx), __fmul_rn(ny, ny)), __fmul_rn(nz, nz));
    if (!(nn > 1e-18f)) {
        // degenerate: every residual is +inf, so no point is ever an inlier
        out = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
        return false;
    }
    float s = __fsqrt_rn(nn);
    nx = __fdiv_rn(nx, s);
    ny = __fdiv_rn(ny, s);
    nz = __fdiv_rn(nz, s);
    float dot = __fadd_rn(__fadd_rn(__fmul_rn(nx, a.x), __fmul_rn(ny, a.y)), __fmul_rn(nz, a.z));
    out = make_float4(nx, ny, nz, -dot);
    return true;
}

// Residual r = fma(nz, pz, fma(ny, py, fma(nx, px, d))); inlier iff
// fma(r, r, -thr2) < 0 (the square is exact inside the fused operation).
__device__ __forceinline__ bool is_inlier(float4 pl, float px, float py, float pz, float thr2)
{
    float r = __fmaf_rn(pl.x, px, pl.w);
    r = __fmaf_rn(pl.y, py, r);
    r = __fmaf_rn(pl.z, pz, r);
    return __fmaf_rn(r, r, -thr2) < 0.0f;
}

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files); all return cudaGetLastError()
// ---------------------------------------------------------------------------
cudaError_t launch_diffuse_tiles(const DiffFrame *d_frames, int n_frames, int total_tiles,
                                 int T, int dx, int dy, float lambda, float K, int mode,
                                 cudaStream_t s);
cudaError_t launch_diffuse_stream(const DiffFrame &f, float lambda, float K, int mode,
                                  cudaStream_t s);
cudaError_t diffuse_init();   // opt the tile kernels into > 48 KB of shared memory
// Rows per warp R of the register-blocked fused kernel for this tiling (PM4,
// output tile (128 - 2T) x (8R - 2T), R in {4, 6, 8}), or 0: the shared-memory
// tile kernel runs it.
int regs_rows(int mode, int T, int dx, int dy);
pm_status set_last_error(pm_status s, const char *msg);

// Record `e` on `s` as a real event: during stream capture a plain
// cudaEventRecord only expresses a dependency, so captured timing events are
// recorded as external event nodes of the graph.
inline cudaError_t record_event(cudaEvent_t e, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(s, &cs);
    if (err != cudaSuccess)
        return err;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                              : cudaEventRecord(e, s);
}
cudaError_t launch_normals(const float *depth, int w, int h, float fx, float fy, float cx,
                           float cy, int stencil, float *P, float *N, unsigned char *valid,
                           cudaStream_t s);
cudaError_t launch_normals_batch(const void *d_desc, int n_frames, int max_w, int max_h,
                                 int stencil, cudaStream_t s);

struct NormFrame {
    const float *depth;
    float *P, *N;
    unsigned char *valid;
    int w, h;
    float fx, fy, cx, cy;
    float ifx, ify;          // 1/fx, 1/fy (rounded from FP64)
};

// RANSAC round structure (ransac.cu)
struct RansacLaunch {
    RFrame *d_frames;     // device array [n]
    int n;
    int *d_chunk_base;    // device [n + 1] (prefix of chunk counts, [n] = total)
    int max_total_chunks; // bound for persistent grids
    RParams prm;
    int score_blocks;     // persistent grid sizes
    int chunk_blocks;     // grid of k_mark0 / k_compact (their resident CTAs, at most one per chunk)
    int remove_blocks;    // grid of k_remove
    unsigned *d_counter;  // [0] grid-completion counter of the compaction kernel,
                          // [1 + r] work counter of round r's scoring
    bool fine_score;      // smaller hypothesis blocks, selection fused (small batches)
    // > 0: the next round's hypotheses are drawn by extra blocks of the
    // compaction launch, with a shared-memory kept-count prefix of this many
    // chunks (a frame's largest chunk count; small batches only); 0: by a
    // launch of their own
    int hyp_fold_chunks;
};
// Per-region RANSAC (regions.cu): all pointers device memory.
struct RegionLaunch {
    const float *P;                 // SoA points [3][w*h]
    const unsigned char *valid;
    const int *regions;             // [w*h]
    int w, h, R, H;
    unsigned long long frame_idx, seed;
    float thr2;
    int *cnt;                       // [R] points per region
    int *box;                       // [R][4] u0, v0, u1, v1
    int *offset, *cursor;           // [R] list offsets / scatter cursors
    int *chunk_base;                // [R + 1] prefix of scoring chunks
    float4 *list;                   // [w*h] region-grouped points
    float4 *hyp;                    // [R*H]
    unsigned char *deg;             // [R*H] degenerate hypotheses
    unsigned long long *err;        // [R*H] distance sums (units of 2^-32 m)
    int *inl;                       // [R*H] inlier counts
    pm_region_plane *out;           // [R]
};
cudaError_t ransac_regions(const RegionLaunch &L, int sms, cudaStream_t s);

// Canny edges of the normal image and the regions they bound (canny.cu); all
// pointers device memory, [w*h] unless noted.
struct EdgeLaunch {
    const float *N;                 // SoA normals [3][w*h]
    const unsigned char *valid;
    int w, h, low, high;
    unsigned char *state;           // 0 / 1 weak / 2 strong after suppression
    unsigned char *strong;          // per root: component holds a strong pixel
    unsigned char *edges;           // output, 1 = edge
    int *L;                         // union-find parents
    int *err;                       // set if a union-find walk overran (never expected)
};
cudaError_t canny_edges(const EdgeLaunch &E, cudaStream_t s);

struct SegLaunch {
    const unsigned char *edges, *valid;
    int w, h, gap, min_pixels;
    int *L, *size, *pre;            // parents, component sizes, in-block prefix of roots
    int *bsum;                      // [ceil(w*h / 1024) + 1]; [last] = number of regions
    int *labels;                    // output
    int *err;
};
cudaError_t segment_regions(const SegLaunch &S, cudaStream_t s);

cudaError_t ransac_init(const RansacLaunch &L, cudaStream_t s);
cudaError_t score_init();                  // shared-memory opt-in; occupancy of the RANSAC kernels
int score_hyp_block(bool fine, int H);     // hypotheses per scoring work item
int score_ctas_per_sm(bool fine, int H);
int remove_ctas_per_sm();                  // resident CTAs per SM of k_remove
int compact_ctas_per_sm();                 // ... of k_compact (and k_mark0)
// ev_score: optional event pair recorded around the scoring launch.
cudaError_t ransac_round(const RansacLaunch &L, int round, bool last, cudaStream_t s,
                         cudaEvent_t ev_before = nullptr, cudaEvent_t ev_after = nullptr);
constexpr int RANSAC_INIT_LAUNCHES = 3;
// chunk count up to which the hypotheses are drawn inside the compaction
// launch (the kept-count prefix of a frame's chunks held in shared memory)
constexpr int HYP_FOLD_MAX_CHUNKS = 4096;
// launches per round: scoring (with the selection fused for small batches,
// else a selection launch), removal and compaction, plus a hypothesis launch
// unless the hypotheses are drawn inside the compaction; the last round
// launches its refit in place of the compaction
inline int ransac_round_launches(bool fine, bool hyp_fold)
{
    return (fine ? 3 : 4) + (hyp_fold ? 0 : 1);
}

}  // namespace pm

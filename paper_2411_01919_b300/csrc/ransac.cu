// ransac.cu -- sequential multi-plane RANSAC (Sec. III-D, Eq. 3, Alg. 2) for
// sm_103a, batched over frames.
//
// One plane round of every frame still running:
//   hypotheses: Philox4x64-10 -> three candidate indices -> FP32 plane (Alg. 2
//               "select random subset of 3 points", "fit plane model").  Drawn
//               by extra blocks of the previous compaction launch, which find
//               candidate i of the list being built in the list it is built
//               from (kept-count prefix, then the keep bits of one chunk);
//               k_hyp draws them from the compacted list for frames of more
//               than HYP_FOLD_MAX_CHUNKS chunks.
//   k_score   : every hypothesis against every candidate on FP32 CUDA cores
//               (Alg. 2 inner parallel loop); a box test per 32-candidate
//               segment settles the pairs it proves to hold no inlier or
//               only inliers without evaluating them; integer counters, one atomic
//               add per (work item, hypothesis).  For small batches the CTA
//               that finishes a frame's last work item picks the frame's
//               winner (maximum count, ties to the lowest index: an integer
//               key); for large ones k_select does, one block per frame.
//   k_remove  : labels of the winner's inliers, keep bitmask of the rest,
//               compensated-FP32 moments of the inliers, one record per chunk.
//   refit     : the group records reduced in compensated FP32 in a fixed
//               order, the 3x3 eigenproblem solved in FP64 -> plane.  A round's
//               refit runs in n extra blocks of the next round's scoring
//               launch (its inputs are kept per round parity, so the next
//               selection does not overwrite them); only the last round's
//               refit is a launch of its own (k_refit).
//   k_compact : order-preserving compaction of the kept candidates (and the
//               next round's hypotheses); the last CTA of the grid plans the
//               next round (candidate counts, stop rule, cross-frame prefix of
//               chunks).
// "Last CTA" is detected with a __threadfence() and an atomic counter; no CTA
// ever waits for another.  Work is split into chunks of CHUNK candidates; a
// frame's chunking never depends on the other frames of the batch, and every
// reduction runs in a fixed order, so a frame's result is bit-identical alone
// and in a batch.
#define PM_FILE_ID 3
#include "pm_internal.cuh"

namespace pm {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1)
{
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
        unsigned long long lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
        unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0; k1 += W1;
    }
}

// Frame owning global work item `wi` (chunk_base has n + 1 entries).
__device__ __forceinline__ int frame_of(const int *__restrict__ base, int n, int wi)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= wi)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The batch's chunk prefix (chunk_base, n + 1 entries) staged in shared
// memory by the whole block when it fits, so that finding a work item's frame
// (a binary search) costs shared-memory loads instead of a chain of dependent
// global loads; larger batches search the global table.
constexpr int BASE_SMEM = 256;

__device__ __forceinline__ const int *stage_base(const int *chunk_base, int n, int *sb)
{
    if (n + 1 > BASE_SMEM)
        return chunk_base;
    for (int i = threadIdx.x; i <= n; i += blockDim.x)
        sb[i] = chunk_base[i];
    __syncthreads();
    return sb;
}

// Chunks of a frame's largest candidate list (all its pixels).
__device__ __forceinline__ int nchunks_of(const RFrame &F) { return (F.npx + CHUNK - 1) / CHUNK; }

// Candidate order: the pixel at position `pos` of the enumeration in strips
// of two rows (rows 2s, 2s + 1; one row when h is odd and the strip is the
// last), each strip column by column, the upper pixel first.  A bijection of
// [0, npx).  Thirty-two consecutive candidates then lie in a patch of about
// 16 x 2 pixels instead of 32 x 1, whose 3-D box is tighter on the surfaces
// of a depth image, so the scoring's box test settles more of their pairs.
__device__ __forceinline__ int strip_pixel(const RFrame &F, int pos)
{
    const int s = pos / (2 * F.w);
    const int y0 = 2 * s;
    const int off = pos - y0 * F.w;
    const bool two = y0 + 1 < F.h;
    const int x = two ? off >> 1 : off;
    const int y = y0 + (two ? off & 1 : 0);
    return y * F.w + x;
}

// ---------------------------------------------------------------------------
// round planning (run by one block of any size that is a multiple of 32)
// ---------------------------------------------------------------------------

// Exclusive prefix over the threads of the block; *total gets the sum.
__device__ int block_exscan(int v, int *total)
{
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    __syncthreads();
    if (lane == 31)
        warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    const int incl = x + (wid > 0 ? warp_tot[wid - 1] : 0);
    *total = warp_tot[nw - 1];
    __syncthreads();
    return incl - v;
}

// Per-frame chunk counts for the next round and their cross-frame prefix.
// initial: chunks over the frame's pixels and a fresh per-frame state;
// otherwise: the candidates kept by the last compaction, the stop rule, and
// the candidate count of `round` recorded for the statistics.
__device__ void plan_round(RFrame *frames, int n, int *chunk_base, int min_inliers, int round,
                           bool initial)
{
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int f0 = threadIdx.x * per, f1 = min(f0 + per, n);
    int mine = 0;
    for (int f = f0; f < f1; ++f) {
        RFrame &F = frames[f];
        RState *st = F.st;
        int nc;
        if (initial) {
            st->M = 0;
            st->M_next = 0;
            st->done = 0;
            st->n_planes = 0;
            st->best_h = -1;
            st->best_count = -1;
            st->rf_pending[0] = 0;
            st->rf_pending[1] = 0;
            st->rf_groups[0] = 0;
            st->rf_groups[1] = 0;
            st->score_done = 0;
            for (int r = 0; r < MAX_PLANES; ++r)
                st->m_hist[r] = 0;
            st->pairs_eval = 0ull;
            nc = (F.npx + CHUNK - 1) / CHUNK;
        } else {
            if (!st->done) {
                st->M = __ldcg(&st->M_next);
                if (st->M < 3 || st->M < min_inliers)
                    st->done = 1;
            }
            nc = st->done ? 0 : (st->M + CHUNK - 1) / CHUNK;
            st->m_hist[round] = st->done ? 0 : st->M;
            st->score_done = 0;
        }
        st->nchunks = nc;
        mine += nc;
    }
    int total;
    int off = block_exscan(mine, &total);
    for (int f = f0; f < f1; ++f) {
        chunk_base[f] = off;
        off += frames[f].st->nchunks;
    }
    if (threadIdx.x == 0)
        chunk_base[n] = total;
}

__global__ void __launch_bounds__(1024) k_plan0(RFrame *frames, int n, int *chunk_base,
                                                unsigned *grid_counter)
{
    if (threadIdx.x == 0)
        *grid_counter = 0u;
    if (threadIdx.x < MAX_PLANES)
        grid_counter[1 + threadIdx.x] = 0u;   // the scoring rounds' work counters
    plan_round(frames, n, chunk_base, 0, 0, true);
}

// Whether this CTA is the last of the grid to get here (then after a fence it
// sees every other CTA's writes).  Resets the counter for the next launch.
__device__ bool last_cta_of_grid(unsigned *counter)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(counter, 1u);
        last = prev == gridDim.x - 1;
        if (last)
            *counter = 0u;
    }
    __syncthreads();
    if (last)
        __threadfence();
    return last;
}

// Whether this CTA finished the last of the `items` work items of a frame.
__device__ bool last_item_of_frame(int *counter, int items)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        last = atomicAdd(counter, 1) == items - 1;
    __syncthreads();
    if (last)
        __threadfence();
    return last;
}

// ---------------------------------------------------------------------------
// round 0 candidate list: valid pixels in the strip order of strip_pixel()
// ---------------------------------------------------------------------------
constexpr int MARK_THREADS = 256;

__global__ void __launch_bounds__(MARK_THREADS) k_mark0(RFrame *frames, int n,
                                                        const int *chunk_base)
{
    __shared__ int wsum[MARK_THREADS / 32];
    __shared__ int sbase[BASE_SMEM];
    constexpr int PER = CHUNK / MARK_THREADS;
    const int *cb = stage_base(chunk_base, n, sbase);
    const int total = cb[n];
    for (int wi = blockIdx.x; wi < total; wi += gridDim.x) {
        const int f = frame_of(cb, n, wi);
        const RFrame &F = frames[f];
        const int c = wi - cb[f];
        const int base = c * CHUNK;
        // the thread's PER pixels loaded together, then marked
        unsigned char vb[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int pos = base + threadIdx.x + u * MARK_THREADS;
            vb[u] = pos < F.npx ? F.valid[strip_pixel(F, pos)] : 0;
        }
        int kept = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int j = threadIdx.x + u * MARK_THREADS;
            const int pix = base + j;
            if (pix < F.npx)
                F.labels[pix] = -1;
            const unsigned word = __ballot_sync(0xffffffffu, (vb[u] & 1) != 0);
            if ((threadIdx.x & 31) == 0 &&
                PM_INB((long long)c * CHUNK_WORDS + (j >> 5), (long long)nchunks_of(F) * CHUNK_WORDS)) {
                F.keepbits[(long long)c * CHUNK_WORDS + (j >> 5)] = word;
                kept += __popc(word);
            }
        }
        if ((threadIdx.x & 31) == 0)
            wsum[threadIdx.x >> 5] = kept;
        __syncthreads();
        if (threadIdx.x == 0 && PM_INB(c, nchunks_of(F))) {
            int s = 0;
            for (int w = 0; w < MARK_THREADS / 32; ++w)
                s += wsum[w];
            F.kept[c] = s;
        }
        __syncthreads();
    }
}

// Order-preserving compaction of chunk c of the source list into list `dst`;
// `off` is the number of candidates kept in the frame's chunks before c.
// Every warp scans the chunk's 32 keep words itself (lane = word) and moves
// the candidates of words wid, wid + 8, ...: no block barrier per chunk.
// src_image: the source is the pixel array itself (round 0).
__device__ void compact_chunk(const RFrame &F, int c, int nchunks, int src, int dst,
                              bool src_image, int off)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned mine = PM_INB((long long)c * CHUNK_WORDS + lane, (long long)nchunks_of(F) * CHUNK_WORDS)
                              ? F.keepbits[(long long)c * CHUNK_WORDS + lane] : 0u;
    const int x = __popc(mine);
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    const int excl = incl - x;
    const long long base = (long long)c * CHUNK;
    const long long npx = F.npx;
    const unsigned lt = (1u << lane) - 1u;
    for (int w = wid; w < CHUNK_WORDS; w += (int)(blockDim.x >> 5)) {
        const unsigned word = __shfl_sync(0xffffffffu, mine, w);
        const int wpre = __shfl_sync(0xffffffffu, excl, w);
        if (word >> lane & 1u) {
            const int pos = off + wpre + __popc(word & lt);
            const long long j = base + 32 * w + lane;
            if (!(PM_INB(j, npx) && PM_INB(pos, npx)))
                continue;
            float4 pt;
            if (src_image) {
                const int q = strip_pixel(F, (int)j);
                pt = make_float4(F.P[q], F.P[npx + q], F.P[2 * npx + q], __int_as_float(q));
            } else
                pt = F.cpt[src][j];
            F.cpt[dst][pos] = pt;
        }
    }
    if (threadIdx.x == 31 && c == nchunks - 1)
        F.st->M_next = off + incl;
}

// Kept candidates of chunks [0, c) of a frame, summed by the whole block.
__device__ int kept_before(const RFrame &F, int c)
{
    __shared__ int s_part[32];
    __shared__ int s_sum;
    int s = 0;
    for (int k = threadIdx.x; k < c; k += blockDim.x)
        s += F.kept[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0)
        s_part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = (int)threadIdx.x < (int)(blockDim.x >> 5) ? s_part[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0)
            s_sum = t;
    }
    __syncthreads();
    return s_sum;
}

// ---------------------------------------------------------------------------
// hypotheses
// ---------------------------------------------------------------------------
// Candidate index k (0..2) of hypothesis h of round `round` in the round's list
// of M: a Philox4x64-10 draw on (h, round, frame index), index umulhi(draw, M).
__device__ __forceinline__ unsigned long long sample_index(const RFrame &F, const RParams &prm,
                                                           int round, int h, int k,
                                                           unsigned long long M)
{
    unsigned long long c[4] = {(unsigned long long)h, (unsigned long long)round, F.frame_idx, 0ull};
    philox4x64_10(c, prm.seed, 0ull);
    return __umul64hi(k == 0 ? c[0] : k == 1 ? c[1] : c[2], M);
}

// The FP32 plane through the three candidates of hypothesis h; degenerate
// triples get count -1.
__device__ __forceinline__ void store_hypothesis(const RFrame &F, int h, float4 q0, float4 q1,
                                                 float4 q2)
{
    float4 pl;
    const bool ok = hyp_plane(make_float3(q0.x, q0.y, q0.z), make_float3(q1.x, q1.y, q1.z),
                              make_float3(q2.x, q2.y, q2.z), pl);
    F.hyp[h] = pl;
    F.hyp_p0[h] = q0;
    F.counts[h] = ok ? 0 : -1;
}

// The round's hypotheses from its compacted list (frames larger than the
// compaction launch's shared-memory prefix).
__global__ void __launch_bounds__(128) k_hyp(RFrame *frames, RParams prm, int round)
{
    const RFrame &F = frames[blockIdx.y];
    if (F.st->done)
        return;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= prm.H)
        return;
    const float4 *pts = F.cpt[round & 1];
    const unsigned long long M = (unsigned long long)F.st->M;
    float4 q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const unsigned long long i = sample_index(F, prm, round, h, k, M);
        q[k] = PM_INB(i, F.npx) ? pts[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    store_hypothesis(F, h, q[0], q[1], q[2]);
}

constexpr int COMPACT_THREADS = 256;
constexpr int HYP_PER_BLOCK = 85;   // hypotheses per drawing block (3 threads each of 256)

// Candidate i of the compacted list, read from the source list before the
// compaction: the chunk c with pre[c] <= i < pre[c + 1] (pre: exclusive prefix
// of the frame's kept counts over its nc chunks), then the (i - pre[c])-th set
// bit of the chunk's keep words -- the same candidate the compaction moves to
// position i.
__device__ float4 kept_candidate(const RFrame &F, const int *pre, int nc, bool src_image, int src,
                                 unsigned long long i)
{
    int lo = 0, hi = nc - 1;   // the last chunk whose prefix is <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((unsigned long long)pre[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    int r = (int)(i - (unsigned long long)pre[lo]);
    unsigned kw[CHUNK_WORDS];
    const long long wbase = (long long)lo * CHUNK_WORDS;
    if (PM_INB(wbase + CHUNK_WORDS - 1, (long long)nchunks_of(F) * CHUNK_WORDS)) {
        const uint4 *k4 = reinterpret_cast<const uint4 *>(F.keepbits + wbase);
#pragma unroll
        for (int q = 0; q < CHUNK_WORDS / 4; ++q) {
            const uint4 v = __ldcg(k4 + q);
            kw[4 * q] = v.x;
            kw[4 * q + 1] = v.y;
            kw[4 * q + 2] = v.z;
            kw[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < CHUNK_WORDS; ++q)
            kw[q] = 0u;
    }
    // the word holding the r-th kept candidate of the chunk, then the bit
    int w = 0;
    unsigned word = 0u;
    bool found = false;
#pragma unroll
    for (int q = 0; q < CHUNK_WORDS; ++q) {
        const int pc = __popc(kw[q]);
        if (!found) {
            if (r < pc) {
                found = true;
                w = q;
                word = kw[q];
            } else {
                r -= pc;
            }
        }
    }
    int bit = 0;
#pragma unroll
    for (int width = 16; width > 0; width >>= 1) {
        const unsigned low = word & ((1u << width) - 1u);
        const int pc = __popc(low);
        if (r >= pc) {
            r -= pc;
            word >>= width;
            bit += width;
        } else {
            word = low;
        }
    }
    const long long j = (long long)lo * CHUNK + 32 * w + bit;
    const long long npx = F.npx;
    if (!PM_INB(j, npx))
        return make_float4(0.f, 0.f, 0.f, 0.f);
    if (src_image) {
        const int q = strip_pixel(F, (int)j);
        return make_float4(F.P[q], F.P[npx + q], F.P[2 * npx + q], __int_as_float(q));
    }
    return F.cpt[src][j];
}

// The hypotheses [hb * HYP_PER_BLOCK, hb * HYP_PER_BLOCK + HYP_PER_BLOCK) of
// round `next` of a frame, drawn beside the compaction that builds that
// round's list (same draws and the same candidates as from the compacted
// list): thread t finds candidate t % 3 of hypothesis t / 3, and the planes
// are formed from shared memory.  pre: shared memory for cap + 1 prefix
// entries.
__device__ void hyp_block(const RFrame &F, const RParams &prm, int next, int hb, bool src_image,
                          int src, int min_inliers, int *pre, int cap)
{
    __shared__ float4 q[3 * HYP_PER_BLOCK];
    RState *st = F.st;
    const int nc = st->nchunks;
    if (st->done || nc < 1 || !PM_INB(nc, cap + 1))   // (block-uniform; cap bounds every frame)
        return;
    const int per = (nc + blockDim.x - 1) / blockDim.x;
    const int c0 = threadIdx.x * per, c1 = min(nc, c0 + per);
    int mine = 0;
    for (int c = c0; c < c1; ++c)
        mine += __ldcg(F.kept + c);
    int total;
    int off = block_exscan(mine, &total);
    for (int c = c0; c < c1; ++c) {
        pre[c] = off;
        off += __ldcg(F.kept + c);
    }
    if (threadIdx.x == 0)
        pre[nc] = total;
    __syncthreads();
    // the stop rule of the next round's planning: no round, no hypotheses
    if (total < 3 || total < min_inliers)
        return;
    const int t = (int)threadIdx.x;
    const int h0 = hb * HYP_PER_BLOCK;
    if (t < 3 * HYP_PER_BLOCK && h0 + t / 3 < prm.H) {
        const unsigned long long i =
            sample_index(F, prm, next, h0 + t / 3, t % 3, (unsigned long long)total);
        q[t] = PM_INB(i, (unsigned long long)total) ? kept_candidate(F, pre, nc, src_image, src, i)
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (t < HYP_PER_BLOCK && h0 + t < prm.H)
        store_hypothesis(F, h0 + t, q[3 * t], q[3 * t + 1], q[3 * t + 2]);
}

// Compaction by block b of nb: each takes a contiguous run of chunks, so the
// running offset within a frame is summed once per run and then advanced
// chunk by chunk.
__device__ void compact_run(RFrame *frames, int n, const int *chunk_base, int src, int dst,
                            bool src_image, int b, int nb)
{
    __shared__ int sbase[BASE_SMEM];
    const int *cb = stage_base(chunk_base, n, sbase);
    const int total = cb[n];
    const int per = (total + nb - 1) / nb;
    const int w0 = b * per, w1 = min(total, w0 + per);
    int cur_f = -1, off = 0;
    for (int wi = w0; wi < w1; ++wi) {
        const int f = frame_of(cb, n, wi);
        const RFrame &F = frames[f];
        if (F.st->done)
            continue;
        const int c = wi - cb[f];
        if (f != cur_f) {
            off = kept_before(F, c);
            cur_f = f;
        }
        compact_chunk(F, c, F.st->nchunks, src, dst, src_image, off);
        off += __ldcg(F.kept + c);
    }
}

// Compaction of every chunk; the last CTA of the grid plans round `next`.
// src_image: round 0 (the source list is the pixel array itself).  With
// hyp_cap > 0 the first n * ceil(H / HYP_PER_BLOCK) blocks draw round
// `next`'s hypotheses instead (hyp_cap: the largest chunk count of a frame,
// for the dynamic shared memory of the prefix) and the other ncompact blocks
// compact.
__global__ void __launch_bounds__(COMPACT_THREADS)
    k_compact(RFrame *frames, int n, int *chunk_base, int round, bool src_image, int next,
              int min_inliers, unsigned *grid_counter, RParams prm, int hyp_cap, int ncompact)
{
    extern __shared__ int pre_sm[];
    const int src = round & 1, dst = src_image ? 0 : src ^ 1;
    const int per_frame = hyp_cap > 0 ? (prm.H + HYP_PER_BLOCK - 1) / HYP_PER_BLOCK : 0;
    const int nhyp = n * per_frame;
    if ((int)blockIdx.x < nhyp) {
        const int f = (int)blockIdx.x / per_frame;
        hyp_block(frames[f], prm, next, (int)blockIdx.x - f * per_frame, src_image, src,
                  min_inliers, pre_sm, hyp_cap);
    } else {
        compact_run(frames, n, chunk_base, src, dst, src_image, (int)blockIdx.x - nhyp, ncompact);
    }
    if (last_cta_of_grid(grid_counter))
        plan_round(frames, n, chunk_base, min_inliers, next, false);
}

// ---------------------------------------------------------------------------
// selection: argmax of (count, -h) by one block
// ---------------------------------------------------------------------------
__device__ void select_winner(const RFrame &F, const RParams &prm, int round)
{
    __shared__ unsigned long long wk[32];
    RState *st = F.st;
    unsigned long long key = 0;
    for (int h = threadIdx.x; h < prm.H; h += blockDim.x) {
        const int cnt = __ldcg(F.counts + h);
        const unsigned long long k = ((unsigned long long)(unsigned)(cnt + 1) << 32) |
                                     (unsigned long long)(0xffffffffu - (unsigned)h);
        key = k > key ? k : key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
        key = y > key ? y : key;
    }
    if ((threadIdx.x & 31) == 0)
        wk[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            key = wk[w] > key ? wk[w] : key;
        const int best_h = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
        const int best_count = (int)(key >> 32) - 1;
        if (best_count < prm.min_inliers || best_count < 3) {
            st->done = 1;
        } else {
            st->best_h = best_h;
            st->best_count = best_count;
            st->best_plane = __ldcg(F.hyp + best_h);
            st->p0 = __ldcg(F.hyp_p0 + best_h);
            // what this round's refit needs, in this round's parity slot: the
            // refit runs beside the next round's selection, which fills the
            // other slot
            const int slot = round & 1;
            st->rf_groups[slot] = (st->nchunks + GROUP - 1) / GROUP;
            st->rf_h[slot] = best_h;
            st->rf_count[slot] = best_count;
            st->rf_p0[slot] = st->p0;
            st->rf_pending[slot] = 1;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// scoring with exact box culling and inclusion.
//
// A work item is (frame, chunk of CHUNK candidates, block of HB hypotheses).
// The chunk is cut into segments of SEG consecutive candidates (in the strip
// order, a patch of about 16 x 2 pixels, so a small patch of one surface);
// large batches also into parents of PSEG segments; each segment gets an
// axis-aligned box [c - e, c + e] that holds its points.  A hypothesis whose
// plane stays farther than the threshold from the whole box, by a margin that
// covers every rounding of the FP32 residual and of the test, has no inlier
// in the segment: its count there is exactly 0.  A hypothesis whose slab
// holds the whole box, by the same margin, has every point of the segment as
// an inlier: its count there is exactly the segment's size.  Neither kind of
// pair is evaluated; the counts, and every decision taken from them, are the
// ones of evaluating all pairs.
//
// The margin.  u = 2^-24, s = 2^-18 (64 u), T = sqrt(thr2) (real).  The
// residual r~ = fma(nz,pz,fma(ny,py,fma(nx,px,d))) of a point p of the box is
// within 3.0000004 u (|n|.|p| + |d|) of n.p + d, and |p_k| <= |c_k| + e_k.
// The box test computes, each step rounded to nearest,
//     t~ = fma(nz,cz,fma(ny,cy,fma(nx,cx,d))),
//     A~ = fma(|nz|,gz,fma(|ny|,gy,fma(|nx|,gx,s|d|))),
// with g_k = e_k + s (|c_k| + e_k) and s|d| rounded up.  t~ is within
// 3.0000004 u (|n|.|c| + |d|) of n.c + d; the slack s in g and s|d| covers
// both residual errors and the three roundings of A~ (all terms >= 0), so
//     | |r~| - |t~| |  <=  |n|.e + 6.000001 u (|n|.(|c| + e) + |d|)  <=  A~
// for every point of the box.  Rounding is monotone and the thresholds are
// FP32 numbers, so
//     fl(|t~| - A~) > thr_c   gives  |r~| > thr_c >= T:  r~ r~ - thr2 > 0;
//     fl(|t~| + A~) < thr_i   gives  |r~| < thr_i <= T:  r~ r~ - thr2 < 0;
// with thr_c >= T (1 + 2^-20) and thr_i <= T (1 - 2^-20) from the host.  A
// degenerate hypothesis (n = 0, d = +inf) has t~ = inf, A~ = 0: culled.  A
// NaN anywhere keeps the pair for evaluation.
//
// Per segment a warp tests all HB hypotheses (one per lane): included ones
// add the segment's size to their shared-memory count, the rest that the
// cull does not prove empty go to a list of survivors (ballot), which is
// scored up to four hypotheses per lane against the segment's points
// (broadcast 16-byte loads from shared memory).  Per pair: three residual
// FMAs, one FMA for r*r - thr2 and one integer add of its sign bit, which is
// set iff it is negative (an exact zero rounds to +0): the decision of
// is_inlier().  Counts go to shared memory, then once per work item to
// global memory.
// ---------------------------------------------------------------------------
constexpr int SEG = 32;
constexpr int NSEG = CHUNK / SEG;
constexpr int PSEG = 4;                  // segments per parent (a 128-candidate box)
constexpr int NPAR = NSEG / PSEG;
constexpr int SCORE_THREADS = 256;
constexpr int SCORE_WARPS = SCORE_THREADS / 32;
constexpr float CULL_SLACK = 0x1p-18f;
static_assert(NPAR == SCORE_WARPS, "one parent per warp in the parent pass");

// TWO: the two-level box test (parents' unsettled lists in shared memory).
template <int HB, bool TWO>
constexpr size_t score_smem_bytes()
{
    return (size_t)CHUNK * 16 + (size_t)HB * 16 + (size_t)HB * 4 + (size_t)NSEG * 32 +
           (size_t)NPAR * 32 + (size_t)HB * 4 + (size_t)SCORE_WARPS * HB * 2 +
           (TWO ? (size_t)NPAR * HB * 2 : 0);
}

// The box [c - g, c + g] of candidates [b0, b0 + n) of the chunk (n >= 1),
// written by lanes 0-2 (axis k by lane k) to out[0] (centre) and out[1]
// (widened half-size): the centre, the half-size rounded up and widened by
// the centre's rounding, then g = e + s (|c| + e) (the margin derived above).
template <int PER>
__device__ __forceinline__ void candidate_box(const float4 *pts, int b0, int n, float4 *out,
                                              int lane)
{
    float lx = INFINITY, ly = INFINITY, lz = INFINITY;
    float ux = -INFINITY, uy = -INFINITY, uz = -INFINITY;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const float4 p = pts[b0 + min(lane + 32 * i, n - 1)];
        lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
        ux = fmaxf(ux, p.x); uy = fmaxf(uy, p.y); uz = fmaxf(uz, p.z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        ux = fmaxf(ux, __shfl_xor_sync(0xffffffffu, ux, o));
        uy = fmaxf(uy, __shfl_xor_sync(0xffffffffu, uy, o));
        uz = fmaxf(uz, __shfl_xor_sync(0xffffffffu, uz, o));
    }
    if (lane < 3) {
        const float lo = lane == 0 ? lx : lane == 1 ? ly : lz;
        const float hi = lane == 0 ? ux : lane == 1 ? uy : uz;
        const float cc = __fmul_rn(__fadd_rn(lo, hi), 0.5f);
        const float e = __fadd_ru(__fmul_ru(__fsub_ru(hi, lo), 0.5f),
                                  __fmul_ru(fabsf(cc), 0x1p-23f));
        const float g = __fmaf_ru(CULL_SLACK, __fadd_ru(fabsf(cc), e), e);
        float *b = reinterpret_cast<float *>(out);
        b[lane] = cc;
        b[4 + lane] = g;
    }
}

// Box test of hypotheses against the box (bc, bg) of sc candidates, by one
// warp: hypotheses whose slab holds the box add sc to their count; those the
// test cannot settle are appended to `out`; returns their number.  LIST:
// the hypotheses are in[0, nin); otherwise they are 0 .. nin - 1 (hpl and
// hsd padded to a multiple of 32 with planes that are always culled).
template <bool LIST>
__device__ __forceinline__ int box_pass(const float4 *hpl, const float *hsd,
                                        const unsigned short *in, int nin, float4 bc, float4 bg,
                                        int sc, int *hcnt, unsigned short *out, float cull_thr,
                                        float incl_thr, int lane)
{
    const unsigned lt = (1u << lane) - 1u;
    int len = 0;
    for (int e = lane; e < nin + ((32 - (nin & 31)) & 31); e += 32) {
        const bool live = !LIST || e < nin;
        const int k = LIST ? (live ? (int)in[e] : 0) : e;
        const float4 pl = hpl[k];
        float t = __fmaf_rn(pl.x, bc.x, pl.w);
        t = __fmaf_rn(pl.y, bc.y, t);
        t = __fmaf_rn(pl.z, bc.z, t);
        float a = __fmaf_rn(fabsf(pl.x), bg.x, hsd[k]);
        a = __fmaf_rn(fabsf(pl.y), bg.y, a);
        a = __fmaf_rn(fabsf(pl.z), bg.z, a);
        const float at = fabsf(t);
        const bool inc = live && __fadd_rn(at, a) < incl_thr;
        if (inc)
            atomicAdd(hcnt + k, sc);
        const bool keep = live && !inc && !(__fsub_rn(at, a) > cull_thr);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep)
            out[len + __popc(m & lt)] = (unsigned short)k;
        len += __popc(m);
    }
    return len;
}

// E surviving hypotheses per lane (list entries e0 + lane + 32 i) against the
// sc points of one segment; counts added to shared memory.
template <int E, bool FULL>
__device__ __forceinline__ void score_batch(const float4 *__restrict__ hpl,
                                            const unsigned short *__restrict__ lst, int e0,
                                            int len, const float4 *__restrict__ sp, int sc,
                                            float nthr2, int *hcnt, int lane)
{
    const float4 none = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
    int k[E];
    float4 pl[E];
    unsigned acc[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int e = e0 + lane + 32 * i;
        k[i] = e < len ? (int)lst[e] : -1;
        pl[i] = k[i] >= 0 ? hpl[k[i]] : none;
        acc[i] = 0u;
    }
    const int n = FULL ? SEG : sc;
#pragma unroll(FULL ? 8 : 1)
    for (int j = 0; j < n; ++j) {
        const float4 p = sp[j];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            float r = __fmaf_rn(pl[i].x, p.x, pl[i].w);
            r = __fmaf_rn(pl[i].y, p.y, r);
            r = __fmaf_rn(pl[i].z, p.z, r);
            acc[i] += __float_as_uint(__fmaf_rn(r, r, nthr2)) >> 31;
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i)
        if (acc[i])
            atomicAdd(hcnt + k[i], (int)acc[i]);
}

template <bool FULL>
__device__ __forceinline__ void score_list(const float4 *hpl, const unsigned short *lst, int len,
                                           const float4 *sp, int sc, float nthr2, int *hcnt,
                                           int lane)
{
    int e0 = 0;
    while (len - e0 >= 128) {
        score_batch<4, FULL>(hpl, lst, e0, len, sp, sc, nthr2, hcnt, lane);
        e0 += 128;
    }
    while (len - e0 > 32) {
        score_batch<2, FULL>(hpl, lst, e0, len, sp, sc, nthr2, hcnt, lane);
        e0 += 64;
    }
    if (len - e0 > 0)
        score_batch<1, FULL>(hpl, lst, e0, len, sp, sc, nthr2, hcnt, lane);
}

// Block-shared scratch of a refit (the scoring kernel lends it part of its
// dynamic shared memory).
struct RefitShared {
    float ss[REFIT_WARPS][2 * NMOM];   // per-warp double-float sums
    float sc[REFIT_WARPS][2 * NMOM];
    int sn[REFIT_WARPS][2];            // per-warp counts of the two sets
    double acc[2 * NMOM];
    long long cnt[2];
};

static_assert(SCORE_THREADS == 32 * REFIT_WARPS && REMOVE_THREADS == 32 * REFIT_WARPS,
              "a refit runs in scoring and in removal-sized blocks");
static_assert(sizeof(RefitShared) <= score_smem_bytes<256, false>(), "refit scratch fits the scoring smem");

__device__ __noinline__ void refit_frame(const RFrame &F, const RParams &prm, int round, RefitShared &rs);

// INNER: a work item is a whole chunk, its hypothesis blocks scored one
// after another on the same points and boxes (large batches); otherwise a
// work item is one (chunk, hypothesis block) pair (more items for small
// batches).  Blocks take work items from a counter (`work`, zeroed when the
// batch starts), so a grid of the resident CTAs ends together whatever the
// items cost.  From the second round on, the blocks first refit the previous
// round's winners (frame f by block f mod grid): the refit reads only that
// round's moment records and its parity slot of the state, which nothing in
// this round's scoring and selection writes.
template <int HB, bool FUSE, bool INNER>
__global__ void __launch_bounds__(SCORE_THREADS) k_score(RFrame *frames, int n,
                                                         const int *chunk_base, RParams prm,
                                                         int round, unsigned *work)
{
    extern __shared__ float4 sm[];
    float4 *pts = sm;                  // [CHUNK] candidates of the chunk
    float4 *hpl = pts + CHUNK;         // [HB] planes (nx, ny, nz, d)
    float4 *box = hpl + HB;            // [NSEG][2] centre c; widened half-size g
    float4 *pbox = box + 2 * NSEG;     // [NPAR][2] the same for each parent
    float *hsd = reinterpret_cast<float *>(pbox + 2 * NPAR);             // [HB] s |d|
    int *hcnt = reinterpret_cast<int *>(hsd + HB);                       // [HB]
    unsigned short *lst = reinterpret_cast<unsigned short *>(hcnt + HB);  // [warps][HB]
    unsigned short *psurv = lst + SCORE_WARPS * HB;                       // [NPAR][HB]
    __shared__ int plen[NPAR];
    constexpr bool TWO = INNER;
    __shared__ int next_seg;
    __shared__ unsigned long long evaluated;
    const int nhb = (prm.H + HB - 1) / HB;
    const int per_chunk = INNER ? 1 : nhb;
    const int total = chunk_base[n] * per_chunk;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float nthr2 = -prm.thr2;
    const float cull_thr = prm.cull_thr, incl_thr = prm.incl_thr;
    unsigned short *my = lst + wid * HB;
    __shared__ int s_item;
    if (round > 0) {
        for (int f = blockIdx.x; f < n; f += gridDim.x) {
            const RFrame &F = frames[f];
            if (F.st->rf_pending[(round - 1) & 1])   // (block-uniform)
                refit_frame(F, prm, round - 1, *reinterpret_cast<RefitShared *>(sm));
            __syncthreads();   // thread 0 ends the refit before the scratch is reused
        }
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_item = (int)atomicAdd(work, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= total)
            break;
        const int wi = it / per_chunk;
        const int hb_first = INNER ? 0 : it - wi * nhb, hb_end = INNER ? nhb : hb_first + 1;
        const int f = frame_of(chunk_base, n, wi);
        const RFrame &F = frames[f];
        RState *st = F.st;
        const int c = wi - chunk_base[f];
        const int base = c * CHUNK;
        const int cnt = max(0, min(CHUNK, st->M - base));
        const float4 *src = F.cpt[round & 1] + base;
        // the removal adds the chunk's kept candidates warp by warp
        if (threadIdx.x == 0 && hb_first == 0 && PM_INB(c, nchunks_of(F)))
            F.kept[c] = 0;
        const int nseg = (cnt + SEG - 1) / SEG;
        const int npar = (nseg + PSEG - 1) / PSEG;
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += SCORE_THREADS)
            pts[j] = PM_INB(base + j, F.npx) ? src[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int hb = hb_first; hb < hb_end; ++hb) {
            const int h0 = hb * HB;
            const int nh = min(HB, prm.H - h0);
            for (int k = threadIdx.x; k < HB; k += SCORE_THREADS) {
                float4 pl = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
                float sd = 0.0f;                     // n = 0, d = inf: culled everywhere
                if (k < nh && PM_INB(h0 + k, prm.H)) {
                    const float4 q = F.hyp[h0 + k];
                    if (fabsf(q.w) <= 3.0e38f) {     // degenerate planes carry d = +inf
                        pl = q;
                        sd = __fmul_ru(CULL_SLACK, fabsf(q.w));
                    }
                }
                hpl[k] = pl;
                hsd[k] = sd;
                hcnt[k] = 0;
            }
            if (threadIdx.x == 0) {
                next_seg = 0;
                evaluated = 0ull;
            }
            __syncthreads();
            if (hb == hb_first) {
                for (int sg = wid; sg < nseg; sg += SCORE_WARPS)
                    candidate_box<1>(pts, sg * SEG, min(SEG, cnt - sg * SEG), box + 2 * sg, lane);
                for (int pg = wid; TWO && pg < npar; pg += SCORE_WARPS)
                    candidate_box<PSEG>(pts, pg * PSEG * SEG, min(PSEG * SEG, cnt - pg * PSEG * SEG),
                                        pbox + 2 * pg, lane);
                __syncthreads();
            }
            // Two levels (large batches): each parent (PSEG segments) against
            // every hypothesis; then each segment against its parent's unsettled
            // hypotheses only.  A parent's box holds its segments' points, so a
            // hypothesis that the parent's test settles has the same answer for
            // every one of them.  (Small batches, whose items are short and
            // latency-bound, test each segment against every hypothesis.)
            if (TWO) {
                for (int pg = wid; pg < npar; pg += SCORE_WARPS) {
                    const int pc = min(PSEG * SEG, cnt - pg * PSEG * SEG);
                    const int len = box_pass<false>(hpl, hsd, nullptr, nh, pbox[2 * pg],
                                                    pbox[2 * pg + 1], pc, hcnt, psurv + pg * HB,
                                                    cull_thr, incl_thr, lane);
                    if (lane == 0)
                        plen[pg] = len;
                }
                __syncthreads();
            }
            unsigned long long mine = 0ull;
            for (;;) {
                int sg = 0;
                if (lane == 0)
                    sg = atomicAdd(&next_seg, 1);
                sg = __shfl_sync(0xffffffffu, sg, 0);
                if (sg >= nseg)
                    break;
                const int pg = sg / PSEG;
                const int sc = min(SEG, cnt - sg * SEG);
                const int len =
                    TWO ? box_pass<true>(hpl, hsd, psurv + pg * HB, plen[pg], box[2 * sg],
                                         box[2 * sg + 1], sc, hcnt, my, cull_thr, incl_thr, lane)
                        : box_pass<false>(hpl, hsd, nullptr, nh, box[2 * sg], box[2 * sg + 1], sc,
                                          hcnt, my, cull_thr, incl_thr, lane);
                __syncwarp();
                mine += (unsigned long long)len * (unsigned)sc;
                if (sc == SEG)
                    score_list<true>(hpl, my, len, pts + sg * SEG, sc, nthr2, hcnt, lane);
                else
                    score_list<false>(hpl, my, len, pts + sg * SEG, sc, nthr2, hcnt, lane);
                __syncwarp();   // the list is rewritten for the next segment
            }
            if (lane == 0 && mine)
                atomicAdd(&evaluated, mine);
            __syncthreads();
            for (int k = threadIdx.x; k < nh; k += SCORE_THREADS) {
                const int v = hcnt[k];
                if (v)
                    atomicAdd(F.counts + h0 + k, v);
            }
            if (threadIdx.x == 0 && evaluated)
                atomicAdd(&st->pairs_eval, evaluated);
            __syncthreads();   // hpl, hw, hcnt are refilled for the next block
        }
        if (FUSE && last_item_of_frame(&st->score_done, st->nchunks * per_chunk))
            select_winner(F, prm, round);
    }
}

// ---------------------------------------------------------------------------
// removal + compensated moments; refit of each frame's plane
// ---------------------------------------------------------------------------

// Knuth's TwoSum: s = fl(a + b) and e with a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// Double-float accumulation (compensated FP32): the sum is h + l, h the
// rounded running sum and l the sum of the exact rounding errors of h's
// additions.  (h, l) += x + t, where x + t is exact (a float and 0, or an
// error-free product).
__device__ __forceinline__ void df_add(float &h, float &l, float x, float t)
{
    float s, e;
    two_sum(h, x, s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, t));
}

// (h, l) += (h2, l2) for two double-float sums.
__device__ __forceinline__ void df_merge(float &h, float &l, float h2, float l2)
{
    float s, e;
    two_sum(h, h2, s, e);
    h = s;
    l = __fadd_rn(__fadd_rn(l, l2), e);
}

// The nine moment values of a centred inlier -- x, y, z and the products xx
// xy xz yy yz zz, each product split exactly into its rounded value and
// tail (fma(a, b, -fl(a b)) is exact) -- added to the double-float sums
// (H, L)[off ..]: no rounding error is dropped, so the covariance
// E[xx] - E[x]^2 of a thin cluster of inliers far from the moment origin,
// where the two terms nearly cancel, keeps its precision.
__device__ __forceinline__ void mom_values(float (&H)[2 * NMOM], float (&L)[2 * NMOM], int off, float x,
                                           float y, float z)
{
    const float a[6] = {x, x, x, y, y, z}, b[6] = {x, y, z, y, z, z};
    const float lin[3] = {x, y, z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (off == 0)
            df_add(H[k], L[k], lin[k], 0.0f);
        else
            df_add(H[NMOM + k], L[NMOM + k], lin[k], 0.0f);
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const float p = __fmul_rn(a[j], b[j]);
        const float t = __fmaf_rn(a[j], b[j], -p);
        if (off == 0)
            df_add(H[3 + j], L[3 + j], p, t);
        else
            df_add(H[NMOM + 3 + j], L[NMOM + 3 + j], p, t);
    }
}

// One halving step of warp_reduce18 at lane offset o: S slots out of 2 S
// (slots at or beyond n hold zeros), the lane keeping the half its bit o
// selects and adding the partner's copy of it.
template <int S>
__device__ __forceinline__ void reduce_half(const float *H, const float *L, int n, int lane, int o,
                                            float (&KH)[S], float (&KL)[S])
{
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        const float ah = H[i], al = L[i];
        const float bh = S + i < n ? H[S + i] : 0.0f, bl = S + i < n ? L[S + i] : 0.0f;
        float kh = up ? bh : ah, kl = up ? bl : al;
        const float sh = up ? ah : bh, sl = up ? al : bl;
        df_merge(kh, kl, __shfl_xor_sync(0xffffffffu, sh, o), __shfl_xor_sync(0xffffffffu, sl, o));
        KH[i] = kh;
        KL[i] = kl;
    }
}

// Sum over the warp of each of a lane's 18 double-float values (the two
// moment sets): five halving steps, 18 -> 9 -> 5 -> 3 -> 2 -> 1 slots (an odd
// count padded with a zero slot), 20 merges and 40 shuffles.  Lane l returns
// the sum of value moment_lane_value(l), or of a padding slot (then < 0).
// The order of the additions is fixed by the lane, not by the data.
__device__ __forceinline__ void warp_reduce18(const float (&H)[2 * NMOM], const float (&L)[2 * NMOM],
                                              int lane, float &h, float &l)
{
    static_assert(2 * NMOM == 18, "the halving steps are laid out for 18 values");
    float h9[9], l9[9], h5[5], l5[5], h3[3], l3[3], h2[2], l2[2], h1[1], l1[1];
    reduce_half<9>(H, L, 18, lane, 16, h9, l9);
    reduce_half<5>(h9, l9, 9, lane, 8, h5, l5);
    reduce_half<3>(h5, l5, 5, lane, 4, h3, l3);
    reduce_half<2>(h3, l3, 3, lane, 2, h2, l2);
    reduce_half<1>(h2, l2, 2, lane, 1, h1, l1);
    h = h1[0];
    l = l1[0];
}

// The value whose warp sum lane `lane` holds after warp_reduce18, or -1 for
// a padding slot: follow the lane's bits down the halving steps.
__device__ __forceinline__ int moment_lane_value(int lane)
{
    const int half[5] = {9, 5, 3, 2, 1};
    int start = 0, n = 2 * NMOM;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (lane & (16 >> k)) {
            start += half[k];
            n -= half[k];
        } else {
            n = min(n, half[k]);
        }
        if (n <= 0)
            return -1;
    }
    return start;
}

// ---------------------------------------------------------------------------
// refit: FP64 reduction + smallest eigenpair of the 3x3 covariance.
// The smallest eigenvalue is the smallest root of the characteristic cubic
//   f(l) = det - c1 l + tr l^2 - l^3   (c1 = sum of the principal 2x2 minors),
// found by Newton's method from l = 0: on [0, l_min] f is decreasing and
// convex (f'' = 2 tr - 6 l > 0 below tr / 3), so the iterates rise
// monotonically to l_min.  Its eigenvector is orthogonal to every row of
// A - l_min I: the largest of the three pairwise cross products of the rows.
// No transcendental functions: FP64 is a narrow unit on this GPU.
// ---------------------------------------------------------------------------
__device__ void smallest_eigenpair(const double a[3][3], double &lmin, double v[3])
{
    const double tr = a[0][0] + a[1][1] + a[2][2];
    const double c1 = a[0][0] * a[1][1] + a[0][0] * a[2][2] + a[1][1] * a[2][2] -
                      a[0][1] * a[0][1] - a[0][2] * a[0][2] - a[1][2] * a[1][2];
    const double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[1][2]) -
                       a[0][1] * (a[0][1] * a[2][2] - a[1][2] * a[0][2]) +
                       a[0][2] * (a[0][1] * a[1][2] - a[1][1] * a[0][2]);
    double l = 0.0;
    for (int it = 0; it < 64; ++it) {
        const double f = det - l * (c1 - l * (tr - l));
        const double fp = -c1 + l * (2.0 * tr - 3.0 * l);
        if (!(fp < 0.0))
            break;
        const double nl = l - f / fp;
        if (!(nl > l))
            break;
        l = nl;
    }
    lmin = l;
    double r[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            r[i][j] = a[i][j] - (i == j ? l : 0.0);
    double best = -1.0;
    v[0] = 0.0;
    v[1] = 0.0;
    v[2] = 1.0;
    for (int pq = 0; pq < 3; ++pq) {
        const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
        const double x = r[p][1] * r[q][2] - r[p][2] * r[q][1];
        const double y = r[p][2] * r[q][0] - r[p][0] * r[q][2];
        const double z = r[p][0] * r[q][1] - r[p][1] * r[q][0];
        const double n2 = x * x + y * y + z * z;
        if (n2 > best) {
            best = n2;
            v[0] = x;
            v[1] = y;
            v[2] = z;
        }
    }
    const double ln = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (ln > 0.0) {
        v[0] /= ln;
        v[1] /= ln;
        v[2] /= ln;
    } else {
        v[0] = 0.0;
        v[1] = 0.0;
        v[2] = 1.0;
    }
}

// FP64 reduction of a frame's group records in a fixed order and the refit
// of round `round`'s winner; run by one block of REFIT_WARPS warps.
__device__ __noinline__ void refit_frame(const RFrame &F, const RParams &prm, int round, RefitShared &rs)
{
    // The group records are reduced in compensated FP32, in a fixed order
    // (warp w takes records w, w + 8, ...; lane v value v; then the warps in
    // order); only the final sums are widened to FP64 for the eigen-solve.
    RState *st = F.st;
    const int slot = round & 1;
    const int ngroups = st->rf_groups[slot];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = REFIT_WARPS;
    float vs = 0.0f, vc = 0.0f;
    int vn = 0;
    // lane v < 2 NMOM: double-float sum (h, l) of value v; lanes 2 NMOM, +1: counts
    const int word = lane < 2 * NMOM ? 2 * lane : 4 * NMOM + min(lane - 2 * NMOM, 1);
    constexpr int UNR = 4;   // records loaded together
    for (int g0 = wid * UNR; g0 < ngroups; g0 += nw * UNR) {
        float a[UNR], b[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const float *rec = F.partial + (long long)(g0 + u) * PART_WORDS;
            const bool ok = g0 + u < ngroups;
            a[u] = ok ? __ldcg(rec + word) : 0.0f;
            b[u] = ok && lane < 2 * NMOM ? __ldcg(rec + word + 1) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (g0 + u >= ngroups)
                break;
            if (lane < 2 * NMOM)
                df_merge(vs, vc, a[u], b[u]);
            else if (lane < 2 * NMOM + 2)
                vn += __float_as_int(a[u]);
        }
    }
    if (lane < 2 * NMOM) {
        rs.ss[wid][lane] = vs;
        rs.sc[wid][lane] = vc;
    } else if (lane < 2 * NMOM + 2) {
        rs.sn[wid][lane - 2 * NMOM] = vn;
    }
    __syncthreads();
    if (wid == 0) {
        if (lane < 2 * NMOM) {
            float s0 = rs.ss[0][lane], c0 = rs.sc[0][lane];
            for (int w = 1; w < nw; ++w)
                df_merge(s0, c0, rs.ss[w][lane], rs.sc[w][lane]);
            rs.acc[lane] = (double)s0 + (double)c0;
        } else if (lane < 2 * NMOM + 2) {
            long long t = 0;
            for (int w = 0; w < nw; ++w)
                t += rs.sn[w][lane - 2 * NMOM];
            rs.cnt[lane - 2 * NMOM] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0)
        return;   // (the caller does not synchronise the block after this)
    long long cnt[2] = {rs.cnt[0], rs.cnt[1]};
    // gated inliers if at least 3 pass the gate, else all inliers (set 0 + set 1)
    const bool gated = cnt[0] >= 3;
    const long long nsel = gated ? cnt[0] : cnt[0] + cnt[1];
    double S[NMOM];
    for (int k = 0; k < NMOM; ++k)
        S[k] = gated ? rs.acc[k] : rs.acc[k] + rs.acc[NMOM + k];
    const double nn = (double)nsel;
    const double mx = S[0] / nn, my = S[1] / nn, mz = S[2] / nn;
    double a[3][3], lmin, nv[3];
    a[0][0] = S[3] / nn - mx * mx;
    a[0][1] = a[1][0] = S[4] / nn - mx * my;
    a[0][2] = a[2][0] = S[5] / nn - mx * mz;
    a[1][1] = S[6] / nn - my * my;
    a[1][2] = a[2][1] = S[7] / nn - my * mz;
    a[2][2] = S[8] / nn - mz * mz;
    smallest_eigenpair(a, lmin, nv);
    double n0 = nv[0], n1 = nv[1], n2 = nv[2];
    const float4 p0 = st->rf_p0[slot];
    const double cx = (double)p0.x + mx, cy = (double)p0.y + my, cz = (double)p0.z + mz;
    double d = -(n0 * cx + n1 * cy + n2 * cz);
    if (d < 0.0) {
        n0 = -n0; n1 = -n1; n2 = -n2; d = -d;
    }
    pm_plane &out = F.planes[st->n_planes];
    out.n[0] = n0;
    out.n[1] = n1;
    out.n[2] = n2;
    out.d = d;
    out.n_inliers = st->rf_count[slot];
    out.n_refit = (int)nsel;
    out.rms = (float)sqrt(fmax(lmin, 0.0));
    out.hyp_index = st->rf_h[slot];
    st->n_planes += 1;
    st->rf_pending[slot] = 0;
    if (round + 1 >= prm.max_planes)
        st->done = 1;
}

// Removal of the winner's inliers.  A work item is a group of GROUP chunks of
// one frame (group g = chunks [g*GROUP, g*GROUP + GROUP)), fixed by the
// frame's own candidate count, so its moment record does not depend on the
// rest of the batch.  Per chunk: labels, keep bitmask and kept count.  Per
// group: one record of compensated moments of the inliers, centred at the
// winner's first sample point, in two disjoint sets -- set 0: inliers whose
// normal passes the refit gate, set 1: the other inliers.
__global__ void __launch_bounds__(REMOVE_THREADS) k_remove(RFrame *frames, int n,
                                                           const int *chunk_base, RParams prm,
                                                           int round)
{
    __shared__ float sh_s[8][2 * NMOM], sh_c[8][2 * NMOM];
    __shared__ int sh_n[8][2];
    __shared__ int sbase[BASE_SMEM];
    const int *cb = stage_base(chunk_base, n, sbase);
    const int total = cb[n];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwarps = REMOVE_THREADS >> 5;
    const int my_v = moment_lane_value(lane);   // the moment value this lane sums
    for (int wi = blockIdx.x; wi < total; wi += gridDim.x) {
        const int f = frame_of(cb, n, wi);
        const int c0 = wi - cb[f];
        if (c0 % GROUP)
            continue;
        const RFrame &F = frames[f];
        RState *st = F.st;
        if (st->done)
            continue;
        const int M = st->M;
        const int nch = st->nchunks;
        const float4 pl = st->best_plane;
        const float4 p0 = st->p0;
        const int cur = round & 1;
        const long long npx = F.npx;
        // per warp: lane l holds the double-float sum of moment value my_v (>= 0)
        // (gated inliers' values 0 .. NMOM-1, the other inliers' NMOM ..);
        // the gated / other counts are warp-uniform (ballots)
        float acc_s = 0.0f, acc_c = 0.0f;
        int cnt_g = 0, cnt_o = 0;
        const int c1 = min(c0 + GROUP, nch);
        for (int c = c0; c < c1; ++c) {
            const int base = c * CHUNK;
            const int cnt = min(CHUNK, M - base);
            // the PER_THREAD candidates of this thread, loaded together
            constexpr int PER_THREAD = CHUNK / REMOVE_THREADS;
            float4 p[PER_THREAD];
            bool inl[PER_THREAD];
#pragma unroll
            for (int u = 0; u < PER_THREAD; ++u) {
                const int j = threadIdx.x + u * REMOVE_THREADS;
                p[u] = j < cnt && PM_INB(base + j, npx) ? F.cpt[cur][base + j]
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            unsigned any = 0u;
            int kept_w = 0;
#pragma unroll
            for (int u = 0; u < PER_THREAD; ++u) {
                const int j = threadIdx.x + u * REMOVE_THREADS;
                inl[u] = j < cnt && is_inlier(pl, p[u].x, p[u].y, p[u].z, prm.thr2);
                const unsigned word = __ballot_sync(0xffffffffu, j < cnt && !inl[u]);
                any |= __ballot_sync(0xffffffffu, inl[u]);
                kept_w += __popc(word);
                if (lane == 0 && PM_INB((long long)c * CHUNK_WORDS + (j >> 5),
                                        (long long)nchunks_of(F) * CHUNK_WORDS))
                    F.keepbits[(long long)c * CHUNK_WORDS + (j >> 5)] = word;
            }
            if (lane == 0 && kept_w)
                atomicAdd(F.kept + c, kept_w);
            if (any) {
                // validity and normal of every inlier fetched together (one
                // round trip); the validity bit decides whether the normal counts
                int pix[PER_THREAD];
                unsigned char vb[PER_THREAD];
                float3 nrm[PER_THREAD];
#pragma unroll
                for (int u = 0; u < PER_THREAD; ++u) {
                    pix[u] = __float_as_int(p[u].w);
                    if (inl[u] && !PM_INB(pix[u], npx))
                        inl[u] = false;
                    const bool g = inl[u] && F.N;
                    vb[u] = g ? F.valid[pix[u]] : 0;
                    nrm[u] = g ? make_float3(F.N[pix[u]], F.N[npx + pix[u]], F.N[2 * npx + pix[u]])
                               : make_float3(0.f, 0.f, 0.f);
                }
                // this lane's candidates, summed per value in registers
                float vh[2 * NMOM], vl[2 * NMOM];
#pragma unroll
                for (int k = 0; k < 2 * NMOM; ++k) {
                    vh[k] = 0.0f;
                    vl[k] = 0.0f;
                }
                bool gated[PER_THREAD];
                int ng = 0, no = 0;
#pragma unroll
                for (int u = 0; u < PER_THREAD; ++u) {
                    gated[u] = false;
                    if (inl[u]) {
                        F.labels[pix[u]] = (short)round;
                        if (vb[u] & 2) {
                            // the gate decides an integer set: FP32 with a fixed order
                            const float dot = __fmaf_rn(nrm[u].z, pl.z,
                                                        __fmaf_rn(nrm[u].y, pl.y,
                                                                  __fmul_rn(nrm[u].x, pl.x)));
                            gated[u] = fabsf(dot) >= prm.cos_gate;
                        }
                    }
                    const int g = __popc(__ballot_sync(0xffffffffu, inl[u] && gated[u]));
                    const int o = __popc(__ballot_sync(0xffffffffu, inl[u] && !gated[u]));
                    ng += g;
                    no += o;
                }
                cnt_g += ng;
                cnt_o += no;
                // each set's sums in a pass of its own, skipped by a warp with no
                // candidate in it: the register set a value goes to is then fixed
                // at compile time, not chosen per lane
                if (ng) {
#pragma unroll
                    for (int u = 0; u < PER_THREAD; ++u)
                        if (inl[u] && gated[u])
                            mom_values(vh, vl, 0, __fsub_rn(p[u].x, p0.x),
                                       __fsub_rn(p[u].y, p0.y), __fsub_rn(p[u].z, p0.z));
                }
                if (no) {
#pragma unroll
                    for (int u = 0; u < PER_THREAD; ++u)
                        if (inl[u] && !gated[u])
                            mom_values(vh, vl, NMOM, __fsub_rn(p[u].x, p0.x),
                                       __fsub_rn(p[u].y, p0.y), __fsub_rn(p[u].z, p0.z));
                }
                float th, tl;
                warp_reduce18(vh, vl, lane, th, tl);
                if (my_v >= 0)
                    df_merge(acc_s, acc_c, th, tl);
            }
        }
        if (my_v >= 0) {
            sh_s[wid][my_v] = acc_s;
            sh_c[wid][my_v] = acc_c;
        }
        if (lane == 0) {
            sh_n[wid][0] = cnt_g;
            sh_n[wid][1] = cnt_o;
        }
        __syncthreads();
        // across warps: one thread per moment value, warps merged in order
        float *rec = F.partial + (long long)(c0 / GROUP) * PART_WORDS;
        if (!PM_INB(c0 / GROUP, nchunks_of(F))) {
            __syncthreads();
            continue;
        }
        if ((int)threadIdx.x < 2 * NMOM) {
            const int v = threadIdx.x;
            float ss = sh_s[0][v], cc = sh_c[0][v];
            for (int w = 1; w < nwarps; ++w)
                df_merge(ss, cc, sh_s[w][v], sh_c[w][v]);
            rec[2 * v] = ss;
            rec[2 * v + 1] = cc;
        } else if ((int)threadIdx.x < 2 * NMOM + 2) {
            const int set = threadIdx.x - 2 * NMOM;
            int nn = 0;
            for (int w = 0; w < nwarps; ++w)
                nn += sh_n[w][set];
            rec[4 * NMOM + set] = __int_as_float(nn);
        }
        __syncthreads();
    }
}

// Large batches: selection and refit as their own launches, one block per
// frame (fusing them costs every scoring / removal work item a fence that
// waits for its atomics, which a batch with many work items per CTA feels).
__global__ void __launch_bounds__(1024) k_select(RFrame *frames, RParams prm, int round)
{
    const RFrame &F = frames[blockIdx.x];
    if (F.st->done)
        return;
    select_winner(F, prm, round);
}

// The last round's refit (every earlier round's runs inside the next round's
// scoring launch): the frames whose selection accepted a winner that round.
__global__ void __launch_bounds__(REMOVE_THREADS) k_refit(RFrame *frames, RParams prm, int round)
{
    const RFrame &F = frames[blockIdx.x];
    __shared__ RefitShared rs;
    if (!F.st->rf_pending[round & 1])
        return;
    refit_frame(F, prm, round, rs);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// The compaction of round `round` into round `next`'s list; with the
// hypothesis fold, extra blocks draw round `next`'s hypotheses.
static void launch_compact(const RansacLaunch &L, int round, bool src_image, int next,
                           cudaStream_t s)
{
    const int cap = L.hyp_fold_chunks;
    const int nhyp = cap > 0 ? L.n * ((L.prm.H + HYP_PER_BLOCK - 1) / HYP_PER_BLOCK) : 0;
    const size_t smem = cap > 0 ? (size_t)(cap + 1) * sizeof(int) : 0;
    k_compact<<<L.chunk_blocks + nhyp, COMPACT_THREADS, smem, s>>>(
        L.d_frames, L.n, L.d_chunk_base, round, src_image, next, L.prm.min_inliers, L.d_counter,
        L.prm, cap, L.chunk_blocks);
}

cudaError_t ransac_init(const RansacLaunch &L, cudaStream_t s)
{
    k_plan0<<<1, 1024, 0, s>>>(L.d_frames, L.n, L.d_chunk_base, L.d_counter);
    k_mark0<<<L.chunk_blocks, MARK_THREADS, 0, s>>>(L.d_frames, L.n, L.d_chunk_base);
    launch_compact(L, 0, true, 0, s);
    return cudaGetLastError();
}

template <int HB, bool FUSE, bool INNER>
static void launch_score(const RansacLaunch &L, int round, cudaStream_t s)
{
    k_score<HB, FUSE, INNER><<<L.score_blocks, SCORE_THREADS, score_smem_bytes<HB, INNER>(), s>>>(
        L.d_frames, L.n, L.d_chunk_base, L.prm, round, L.d_counter + 1 + round);
}

template <int HB, bool FUSE, bool INNER>
static cudaError_t score_attr(int *ctas)
{
    cudaError_t e = cudaFuncSetAttribute(k_score<HB, FUSE, INNER>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)score_smem_bytes<HB, INNER>());
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_score<HB, FUSE, INNER>,
                                                          SCORE_THREADS, score_smem_bytes<HB, INNER>());
    return e;
}

static int g_score_ctas[3] = {1, 1, 1};   // CTAs per SM: <256,true>, <256,false>, <512,false>
static int g_remove_ctas = 1, g_compact_ctas = 1;

cudaError_t score_init()
{
    cudaError_t e = score_attr<256, true, false>(&g_score_ctas[0]);
    if (e == cudaSuccess)
        e = score_attr<256, false, true>(&g_score_ctas[1]);
    if (e == cudaSuccess)
        e = score_attr<512, false, true>(&g_score_ctas[2]);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_remove_ctas, k_remove,
                                                          REMOVE_THREADS, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_compact_ctas, k_compact, 256,
                                                          (HYP_FOLD_MAX_CHUNKS + 1) * sizeof(int));
    return e;
}

int remove_ctas_per_sm() { return g_remove_ctas > 0 ? g_remove_ctas : 1; }
int compact_ctas_per_sm() { return g_compact_ctas > 0 ? g_compact_ctas : 1; }

int score_hyp_block(bool fine, int H) { return fine || H <= 256 ? 256 : 512; }

int score_ctas_per_sm(bool fine, int H)
{
    const int v = fine ? g_score_ctas[0] : H <= 256 ? g_score_ctas[1] : g_score_ctas[2];
    return v > 0 ? v : 1;
}

cudaError_t ransac_round(const RansacLaunch &L, int round, bool last, cudaStream_t s,
                         cudaEvent_t ev_before, cudaEvent_t ev_after)
{
    const RParams &p = L.prm;
    if (L.hyp_fold_chunks == 0)
        k_hyp<<<dim3((p.H + 127) / 128, L.n), 128, 0, s>>>(L.d_frames, p, round);
    if (ev_before)
        record_event(ev_before, s);
    // coarse work items (512-hypothesis blocks, separate selection) when there
    // are enough chunks to fill the GPU; 256-hypothesis blocks with the
    // selection folded into the scoring launch for small batches.  Either
    // scoring launch also refits the previous round's winners.
    const bool fine = L.fine_score;
    if (fine)
        launch_score<256, true, false>(L, round, s);
    else if (p.H <= 256)
        launch_score<256, false, true>(L, round, s);
    else
        launch_score<512, false, true>(L, round, s);
    if (ev_after)
        record_event(ev_after, s);
    if (!fine)
        k_select<<<L.n, 1024, 0, s>>>(L.d_frames, p, round);
    k_remove<<<L.remove_blocks, REMOVE_THREADS, 0, s>>>(L.d_frames, L.n, L.d_chunk_base, p, round);
    if (!last)
        launch_compact(L, round, false, round + 1, s);
    else
        k_refit<<<L.n, REMOVE_THREADS, 0, s>>>(L.d_frames, p, round);
    return cudaGetLastError();
}

PM_BOUNDS_QUERY(bounds_ransac)

}  // namespace pm

// pm_api.cu -- the C ABI of libpm (include/pm.h): contexts, argument checks,
// scratch arena, launch orchestration, CUDA-graph capture of batches.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pm_internal.cuh"

using namespace pm;

namespace {

thread_local std::string g_err;

// An NVTX range over the lifetime of the object (entry points and the stages
// of a launch sequence), visible to profilers that record NVTX; header-only,
// inert when no tool is attached.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

pm_status fail(pm_status s, const std::string &m)
{
    g_err = m;
    return s;
}

#define PM_CK(call)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int elem_size(int dtype) { return dtype == PM_F32_M ? 4 : 2; }

// Layout of the device scratch arena: every region is 256-byte aligned.
struct Layout {
    size_t buf[2], depth, P, N, valid, labels, cpt[2], input;
    size_t hyp, hyp_p0, counts, kept, keepbits, partial, state, planes, chunk_base, counter;
    size_t total;
};

Layout make_layout(long long npx, int frames, int H, int max_chunks)
{
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t F = (size_t)frames, P = (size_t)npx;
    L.buf[0] = take(F * P * 4);   // lo parts of the compensated iterate
    L.buf[1] = take(F * P * 4);
    L.depth = take(F * P * 4);
    L.P = take(F * P * 12);
    L.N = take(F * P * 12);
    L.valid = take(F * P);
    L.labels = take(F * P * 2);
    L.cpt[0] = take(F * P * 16);
    L.cpt[1] = take(F * P * 16);
    L.input = take(F * P * 4);
    L.hyp = take(F * H * 16);
    L.hyp_p0 = take(F * H * 16);
    L.counts = take(F * H * 4);
    L.kept = take(F * max_chunks * 4);
    L.keepbits = take(F * max_chunks * CHUNK_WORDS * 4);
    L.partial = take(F * max_chunks * PART_WORDS * 4);
    L.state = take(F * sizeof(RState));
    L.planes = take(F * MAX_PLANES * sizeof(pm_plane));
    L.chunk_base = take((F + 1) * 4);
    L.counter = take(4 * (1 + MAX_PLANES));   // compaction grid counter, scoring work counters
    L.total = off;
    return L;
}

// Per-region RANSAC scratch for R regions x H hypotheses.
struct RegionLayout {
    size_t cnt, box, off, cur, cb, hyp, deg, err, inl, out, total;
};

RegionLayout region_layout(size_t R, size_t H)
{
    RegionLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align_up(o + bytes, 256);
        return r;
    };
    const size_t RH = R * H;
    L.cnt = take(R * 4);
    L.box = take(R * 16);
    L.off = take(R * 4);
    L.cur = take(R * 4);
    L.cb = take((R + 1) * 4);
    L.hyp = take(RH * 16);
    L.deg = take(RH);
    L.err = take(RH * 8);
    L.inl = take(RH * 4);
    L.out = take(R * sizeof(pm_region_plane));
    L.total = o;
    return L;
}

// Scratch of the edge and region passes for images of up to n pixels.
struct EdgeLayout {
    size_t state, strong, L, size, pre, bsum, err, total;
};

EdgeLayout edge_layout(size_t n)
{
    EdgeLayout E;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align_up(o + bytes, 256);
        return r;
    };
    const size_t nb = (n + 1023) / 1024 + 1;
    E.state = take(n);
    E.strong = take(n);
    E.L = take(n * 4);
    E.size = take(n * 4);
    E.pre = take(n * 4);
    E.bsum = take(nb * 4);
    E.err = take(4);
    E.total = o;
    return E;
}

// Regions the per-region RANSAC scratch allocated by pm_create holds (at the
// context's hypothesis count).
constexpr int CREATE_REGIONS = 256;

struct GraphEntry {
    std::vector<long long> sig;
    cudaGraphExec_t exec;
    long long launches;   // kernels in the graph
};

}  // namespace

namespace pm {
// Record `msg` as the calling thread's pm_last_error() text and return `s`.
pm_status set_last_error(pm_status s, const char *msg) { return fail(s, msg); }
}  // namespace pm

struct pm_ctx {
    pm_diffusion_params dp;
    pm_ransac_params rp;
    pm_misc_params mp;
    int max_w, max_h, max_frames;
    long long max_npx;
    int max_chunks;
    int sms;
    int device;
    Layout lay;
    char *arena = nullptr;
    char *d_tables = nullptr;
    char *h_tables = nullptr;
    size_t tables_cap = 0;
    RState *h_state = nullptr;
    pm_plane *h_planes = nullptr;
    std::vector<GraphEntry> graphs;
    int timing = 0;                       // 0 off, 1 stage events, 2 scoring-kernel events
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t kev[2 * MAX_PLANES] = {};
    float stage_ms[3] = {0, 0, 0};
    int pending_n = 0;
    char *rg = nullptr;                   // per-region RANSAC scratch (grown on demand)
    size_t rg_cap = 0;
    pm_region_plane *h_rg = nullptr;      // pinned copy of its results
    int h_rg_cap = 0;
    char *eg = nullptr;                   // edge / region scratch for max_npx (on first use)
    int *h_eg = nullptr;                  // pinned: region count, error flag
    cudaStream_t gstream = nullptr;       // graph stream when the caller passes the legacy stream
    cudaEvent_t gev[2] = {nullptr, nullptr};
    long long launches = 0;               // kernels launched by the last call
    int last_n = 0;                       // frames of the last call
    std::vector<int> geom_wh;             // w, h of each frame of the last whole-path call

    template <class T> T *at(size_t off) const { return reinterpret_cast<T *>(arena + off); }
};

namespace {

// A frame resolved against the context: pointers, sizes and iteration count.
struct FrameJob {
    const void *src;
    int dtype, w, h;
    long long pitch;
    float fx, fy, cx, cy;
    unsigned long long frame_idx;
    int iters;
    short *labels;
    float *depth_out;
};

pm_status check_params(const pm_diffusion_params *dp, const pm_ransac_params *rp,
                       const pm_misc_params *mp)
{
    if (!dp || !rp || !mp)
        return fail(PM_ERR_ARG, "null parameter struct");
    if (dp->iters < 0 || dp->iters > 100000)
        return fail(PM_ERR_ARG, "diffusion iters out of range [0, 100000]");
    if (!(dp->lambda > 0.0f) || dp->lambda > 0.25f)
        return fail(PM_ERR_ARG, "diffusion lambda must lie in (0, 0.25]");
    if (!(dp->K > 0.0f) || !std::isfinite(dp->K))
        return fail(PM_ERR_ARG, "diffusion K must be positive");
    if (dp->mode != 0 && dp->mode != 1)
        return fail(PM_ERR_ARG, "diffusion mode must be 0 (PM4) or 1 (ALG1)");
    if (dp->iters_per_launch < 0 || dp->iters_per_launch > DT_MAX)
        return fail(PM_ERR_ARG, "iters_per_launch must lie in [0, 8]");
    const int T_eff = dp->iters_per_launch > 0 ? dp->iters_per_launch : DT_MAX;
    if (dp->tile_w < 0 || dp->tile_h < 0 || dp->tile_w + 2 * T_eff > TILE_MAX_DX ||
        dp->tile_h + 2 * T_eff > TILE_MAX_DY)
        return fail(PM_ERR_ARG, "tile_w + 2 T must lie in [0, 144] and tile_h + 2 T in [0, 64] "
                                "(T = iters_per_launch, 8 when 0)");
    if (rp->hypotheses < 1 || rp->hypotheses > MAX_HYP)
        return fail(PM_ERR_ARG, "hypotheses must lie in [1, 2048]");
    if (!(rp->thr_m > 0.0f) || !std::isfinite(rp->thr_m))
        return fail(PM_ERR_ARG, "thr_m must be positive");
    if (rp->max_planes < 1 || rp->max_planes > MAX_PLANES)
        return fail(PM_ERR_ARG, "max_planes must lie in [1, 64]");
    if (rp->min_inliers < 3)
        return fail(PM_ERR_ARG, "min_inliers must be >= 3");
    if (!(rp->refit_normal_gate_deg >= 0.0f) || rp->refit_normal_gate_deg > 180.0f)
        return fail(PM_ERR_ARG, "refit_normal_gate_deg must lie in [0, 180]");
    if (mp->normal_stencil != 0 && mp->normal_stencil != 1)
        return fail(PM_ERR_ARG, "normal_stencil must be 0 (central) or 1 (Sobel)");
    if (!(mp->depth_scale > 0.0f) || !std::isfinite(mp->depth_scale))
        return fail(PM_ERR_ARG, "depth_scale must be positive");
    return PM_OK;
}

// Whether a device pointer meets the alignment of its element type (a
// misaligned element access would fault the kernel instead of failing here).
bool misaligned(const void *p, size_t align) { return ((uintptr_t)p & (align - 1)) != 0; }

pm_status check_frame(const pm_ctx *ctx, const void *depth, int dtype, int w, int h,
                      long long pitch, const pm_intrinsics *K)
{
    if (!depth)
        return fail(PM_ERR_ARG, "null depth pointer");
    if (dtype != PM_U16_MM && dtype != PM_F16_M && dtype != PM_F32_M)
        return fail(PM_ERR_ARG, "unknown depth dtype");
    if (w < 1 || h < 1)
        return fail(PM_ERR_ARG, "image size must be at least 1x1");
    if ((long long)w * h > ctx->max_npx)
        return fail(PM_ERR_ARG, "image larger than the context's max_w * max_h");
    if (pitch < (long long)w * elem_size(dtype) || pitch % elem_size(dtype) != 0)
        return fail(PM_ERR_ARG, "pitch smaller than a row or not a multiple of the element size");
    if (misaligned(depth, elem_size(dtype)))
        return fail(PM_ERR_ARG, "depth pointer not aligned to its element size");
    if (K && (!(K->fx > 0) || !(K->fy > 0) || !std::isfinite(K->fx) || !std::isfinite(K->fy) ||
              !std::isfinite(K->cx) || !std::isfinite(K->cy)))
        return fail(PM_ERR_ARG, "intrinsics must be finite with fx, fy > 0");
    return PM_OK;
}

int choose_T(const pm_ctx *ctx) { return ctx->dp.iters_per_launch > 0 ? ctx->dp.iters_per_launch : DT_MAX; }

pm_status ensure_tables(pm_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->tables_cap)
        return PM_OK;
    size_t cap = align_up(bytes * 2, 4096);
    if (ctx->d_tables)
        cudaFree(ctx->d_tables);
    if (ctx->h_tables)
        cudaFreeHost(ctx->h_tables);
    ctx->d_tables = nullptr;
    ctx->h_tables = nullptr;
    ctx->tables_cap = 0;
    PM_CK(cudaMalloc(&ctx->d_tables, cap));
    PM_CK(cudaMallocHost(&ctx->h_tables, cap));
    ctx->tables_cap = cap;
    return PM_OK;
}

// What the launch sequence of a batch depends on (the graph cache key).
std::vector<long long> signature(const std::vector<FrameJob> &jobs, int T, bool ransac)
{
    std::vector<long long> s;
    s.push_back((long long)jobs.size());
    s.push_back(T);
    s.push_back(ransac ? 1 : 0);
    for (const FrameJob &j : jobs) {
        s.push_back(j.w);
        s.push_back(j.h);
        s.push_back(j.iters);
    }
    return s;
}

struct Plan {
    size_t bytes = 0;
    int dx = 0, dy = 0;               // diffusion output tile
    std::vector<size_t> diff_off;     // table offset of each diffusion launch
    std::vector<int> diff_n, diff_tiles;
    size_t norm_off = 0, rframe_off = 0;
    int max_w = 0, max_h = 0;
    long long total_chunks = 0;
};

// Fill the pinned host tables for a batch (descriptor contents only; the
// launch sequence depends on the signature alone).
Plan build_tables(pm_ctx *ctx, const std::vector<FrameJob> &jobs, int T, bool ransac,
                  bool write)
{
    Plan pl;
    const int n = (int)jobs.size();
    std::vector<int> L(n);
    int Lmax = 0;
    long long big_tiles = 0;
    for (int f = 0; f < n; ++f) {
        L[f] = jobs[f].iters == 0 ? 1 : (jobs[f].iters + T - 1) / T;
        Lmax = L[f] > Lmax ? L[f] : Lmax;
        pl.max_w = jobs[f].w > pl.max_w ? jobs[f].w : pl.max_w;
        pl.max_h = jobs[f].h > pl.max_h ? jobs[f].h : pl.max_h;
        pl.total_chunks += ((long long)jobs[f].w * jobs[f].h + CHUNK - 1) / CHUNK;
        big_tiles += (long long)((jobs[f].w + 79) / 80) * ((jobs[f].h + 47) / 48);
    }
    // tile shape: for PM4 batches that fill the GPU twice over, the
    // register-blocked kernel's (128 - 2T) x (64 - 2T) tiles; otherwise the
    // shared-memory kernel's smaller tiles (more CTAs for small batches)
    const bool big = big_tiles >= 2LL * ctx->sms;
    const bool regs = big && ctx->dp.mode == 0;
    pl.dx = ctx->dp.tile_w > 0 ? ctx->dp.tile_w : (regs ? 128 - 2 * T : big ? 80 : 48);
    pl.dy = ctx->dp.tile_h > 0 ? ctx->dp.tile_h : (regs ? 64 - 2 * T : big ? 48 : 24);
    size_t off = 0;
    for (int k = 0; k < Lmax; ++k) {
        DiffFrame *tab = reinterpret_cast<DiffFrame *>(ctx->h_tables + off);
        pl.diff_off.push_back(off);
        int cnt = 0, tiles = 0;
        for (int f = 0; f < n; ++f) {
            if (k >= L[f])
                continue;
            const FrameJob &j = jobs[f];
            const long long slot = (long long)f * ctx->max_npx;
            const int tx = (j.w + pl.dx - 1) / pl.dx, ty = (j.h + pl.dy - 1) / pl.dy;
            if (write) {
                DiffFrame d;
                const bool first = k == 0, lastk = k == L[f] - 1;
                d.src = j.src;
                d.src_dtype = j.dtype;
                d.src_pitch = j.pitch;
                d.lo_in = first ? nullptr : ctx->at<float>(ctx->lay.buf[(k - 1) & 1]) + slot;
                d.w = j.w;
                d.h = j.h;
                d.dst = lastk ? j.depth_out : ctx->at<float>(ctx->lay.buf[k & 1]) + slot;
                d.dst_lo = lastk ? 0 : 1;
                int rem = j.iters - k * T;
                d.n_iters = rem < T ? (rem > 0 ? rem : 0) : T;
                d.tiles_x = tx;
                d.tile_begin = tiles;
                d.scale = ctx->mp.depth_scale;
                tab[cnt] = d;
            }
            tiles += tx * ty;
            ++cnt;
        }
        pl.diff_n.push_back(cnt);
        pl.diff_tiles.push_back(tiles);
        off += align_up(cnt * sizeof(DiffFrame), 256);
    }
    pl.norm_off = off;
    if (write) {
        NormFrame *nt = reinterpret_cast<NormFrame *>(ctx->h_tables + off);
        for (int f = 0; f < n; ++f) {
            const FrameJob &j = jobs[f];
            const long long slot = (long long)f * ctx->max_npx;
            nt[f] = NormFrame{j.depth_out, ctx->at<float>(ctx->lay.P) + 3 * slot,
                              ctx->at<float>(ctx->lay.N) + 3 * slot,
                              ctx->at<unsigned char>(ctx->lay.valid) + slot, j.w, j.h,
                              j.fx, j.fy, j.cx, j.cy, (float)(1.0 / (double)j.fx),
                              (float)(1.0 / (double)j.fy)};
        }
    }
    off += align_up(n * sizeof(NormFrame), 256);
    pl.rframe_off = off;
    if (write && ransac) {
        RFrame *rt = reinterpret_cast<RFrame *>(ctx->h_tables + off);
        for (int f = 0; f < n; ++f) {
            const FrameJob &j = jobs[f];
            const long long slot = (long long)f * ctx->max_npx;
            const Layout &Ly = ctx->lay;
            RFrame r;
            r.P = ctx->at<float>(Ly.P) + 3 * slot;
            r.N = ctx->at<float>(Ly.N) + 3 * slot;
            r.valid = ctx->at<unsigned char>(Ly.valid) + slot;
            r.labels = j.labels;
            r.w = j.w;
            r.h = j.h;
            r.npx = j.w * j.h;
            r.frame_idx = j.frame_idx;
            for (int b = 0; b < 2; ++b) {
                r.cpt[b] = ctx->at<float4>(Ly.cpt[b]) + slot;
            }
            r.hyp = ctx->at<float4>(Ly.hyp) + (size_t)f * ctx->rp.hypotheses;
            r.hyp_p0 = ctx->at<float4>(Ly.hyp_p0) + (size_t)f * ctx->rp.hypotheses;
            r.counts = ctx->at<int>(Ly.counts) + (size_t)f * ctx->rp.hypotheses;
            r.kept = ctx->at<int>(Ly.kept) + (size_t)f * ctx->max_chunks;
            r.keepbits = ctx->at<unsigned>(Ly.keepbits) + (size_t)f * ctx->max_chunks * CHUNK_WORDS;
            r.partial = ctx->at<float>(Ly.partial) + (size_t)f * ctx->max_chunks * PART_WORDS;
            r.st = ctx->at<RState>(Ly.state) + f;
            r.planes = ctx->at<pm_plane>(Ly.planes) + (size_t)f * MAX_PLANES;
            rt[f] = r;
        }
    }
    off += align_up(n * sizeof(RFrame), 256);
    pl.bytes = off;
    return pl;
}

RParams ransac_params(const pm_ctx *ctx)
{
    RParams p;
    p.H = ctx->rp.hypotheses;
    p.thr2 = ctx->rp.thr_m * ctx->rp.thr_m;
    p.max_planes = ctx->rp.max_planes;
    p.min_inliers = ctx->rp.min_inliers;
    p.seed = ctx->rp.seed;
    p.cos_gate = (float)std::cos((double)ctx->rp.refit_normal_gate_deg * M_PI / 180.0);
    p.cull_thr = std::nextafter((float)(std::sqrt((double)p.thr2) * (1.0 + 0x1p-20)), INFINITY);
    p.incl_thr = std::nextafter((float)(std::sqrt((double)p.thr2) * (1.0 - 0x1p-20)), 0.0f);
    return p;
}

// Enqueue the RANSAC rounds for n frames whose RFrame table is at d_rframes.
pm_status enqueue_ransac(pm_ctx *ctx, RFrame *d_rframes, int n, long long total_chunks,
                         cudaStream_t s)
{
    Range range_("ransac");
    RansacLaunch L;
    L.d_frames = d_rframes;
    L.n = n;
    L.d_chunk_base = ctx->at<int>(ctx->lay.chunk_base);
    L.max_total_chunks = (int)total_chunks;
    L.prm = ransac_params(ctx);
    L.d_counter = ctx->at<unsigned>(ctx->lay.counter);
    L.fine_score = total_chunks < (long long)ctx->sms * 32;
    // small batches draw the hypotheses inside the compaction launch (one
    // launch less per round on a latency-bound path); large ones keep the
    // hypothesis launch, whose blocks would otherwise queue behind the
    // compaction's resident grid
    L.hyp_fold_chunks =
        L.fine_score && ctx->max_chunks <= HYP_FOLD_MAX_CHUNKS ? ctx->max_chunks : 0;
    const int hb = score_hyp_block(L.fine_score, L.prm.H);
    const long long score_items = total_chunks * (L.fine_score ? (L.prm.H + hb - 1) / hb : 1);
    const long long sb = (long long)ctx->sms * score_ctas_per_sm(L.fine_score, L.prm.H);
    // persistent grids of the resident CTAs (a CTA beyond them would start
    // only when a resident one has finished all its work items)
    const long long cb = (long long)ctx->sms * compact_ctas_per_sm();
    const long long rb = (long long)ctx->sms * remove_ctas_per_sm();
    L.score_blocks = (int)(score_items < sb ? score_items : sb);
    L.chunk_blocks = (int)(total_chunks < cb ? total_chunks : cb);
    L.remove_blocks = (int)(total_chunks < rb ? total_chunks : rb);
    if (L.score_blocks < 1)
        L.score_blocks = 1;
    if (L.chunk_blocks < 1)
        L.chunk_blocks = 1;
    if (L.remove_blocks < 1)
        L.remove_blocks = 1;
    PM_CK(ransac_init(L, s));
    ctx->launches += RANSAC_INIT_LAUNCHES;
    for (int r = 0; r < ctx->rp.max_planes; ++r) {
        const bool last = r + 1 == ctx->rp.max_planes;
        cudaEvent_t a = ctx->timing == 2 ? ctx->kev[2 * r] : nullptr;
        cudaEvent_t b = ctx->timing == 2 ? ctx->kev[2 * r + 1] : nullptr;
        PM_CK(ransac_round(L, r, last, s, a, b));
        ctx->launches += ransac_round_launches(L.fine_score, L.hyp_fold_chunks > 0);
    }
    return PM_OK;
}

// The launch sequence of a batch after its tables are written: upload,
// diffusion, normals, RANSAC, result download.
pm_status enqueue_batch(pm_ctx *ctx, const Plan &pl, int n, int T, bool ransac, bool timed,
                        cudaStream_t s)
{
    PM_CK(cudaMemcpyAsync(ctx->d_tables, ctx->h_tables, pl.bytes, cudaMemcpyHostToDevice, s));
    if (timed)
        PM_CK(record_event(ctx->ev[0], s));
    Range r_diff("diffusion");
    for (size_t k = 0; k < pl.diff_off.size(); ++k) {
        if (pl.diff_n[k] == 0)
            continue;
        int Tk = T;
        PM_CK(launch_diffuse_tiles(reinterpret_cast<const DiffFrame *>(ctx->d_tables + pl.diff_off[k]),
                                   pl.diff_n[k], pl.diff_tiles[k], Tk, pl.dx, pl.dy,
                                   ctx->dp.lambda, ctx->dp.K, ctx->dp.mode, s));
        ctx->launches += 1;
    }
    if (timed)
        PM_CK(record_event(ctx->ev[1], s));
    if (!ransac)
        return PM_OK;
    Range r_norm("normals");
    PM_CK(launch_normals_batch(ctx->d_tables + pl.norm_off, n, pl.max_w, pl.max_h,
                               ctx->mp.normal_stencil, s));
    ctx->launches += 1;
    if (timed)
        PM_CK(record_event(ctx->ev[2], s));
    pm_status st = enqueue_ransac(ctx, reinterpret_cast<RFrame *>(ctx->d_tables + pl.rframe_off),
                                  n, pl.total_chunks, s);
    if (st != PM_OK)
        return st;
    if (timed)
        PM_CK(record_event(ctx->ev[3], s));
    PM_CK(cudaMemcpyAsync(ctx->h_state, ctx->at<RState>(ctx->lay.state), n * sizeof(RState),
                          cudaMemcpyDeviceToHost, s));
    PM_CK(cudaMemcpyAsync(ctx->h_planes, ctx->at<pm_plane>(ctx->lay.planes),
                          (size_t)n * MAX_PLANES * sizeof(pm_plane), cudaMemcpyDeviceToHost, s));
    return PM_OK;
}

pm_status run_batch(pm_ctx *ctx, std::vector<FrameJob> &jobs, bool ransac, bool use_graph,
                    cudaStream_t s)
{
    const int n = (int)jobs.size();
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    const int T = choose_T(ctx);
    for (int f = 0; f < n; ++f) {
        const long long slot = (long long)f * ctx->max_npx;
        if (!jobs[f].depth_out)
            jobs[f].depth_out = ctx->at<float>(ctx->lay.depth) + slot;
        if (!jobs[f].labels)
            jobs[f].labels = ctx->at<short>(ctx->lay.labels) + slot;
    }
    ctx->launches = 0;
    ctx->last_n = n;
    if (ransac) {
        ctx->geom_wh.resize(2 * (size_t)n);
        for (int f = 0; f < n; ++f) {
            ctx->geom_wh[2 * f] = jobs[f].w;
            ctx->geom_wh[2 * f + 1] = jobs[f].h;
        }
    }
    Plan pl = build_tables(ctx, jobs, T, ransac, false);
    pm_status st = ensure_tables(ctx, pl.bytes);
    if (st != PM_OK)
        return st;
    build_tables(ctx, jobs, T, ransac, true);
    if (use_graph) {
        // a stream that is being captured by the caller gets plain launches
        // (they become part of the caller's graph)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        PM_CK(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            use_graph = false;
    }
    if (use_graph) {
        // the legacy default stream cannot be captured: run the graph on the
        // context's own stream, ordered after and before the caller's work
        const bool bridge = s == nullptr;
        if (bridge) {
            if (!ctx->gstream) {
                PM_CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
                PM_CK(cudaEventCreateWithFlags(&ctx->gev[0], cudaEventDisableTiming));
                PM_CK(cudaEventCreateWithFlags(&ctx->gev[1], cudaEventDisableTiming));
            }
            PM_CK(cudaEventRecord(ctx->gev[0], s));
            PM_CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0));
            s = ctx->gstream;
        }
        std::vector<long long> sig = signature(jobs, T, ransac);
        sig.push_back(ctx->timing);
        sig.push_back(pl.dx);
        sig.push_back(pl.dy);
        cudaGraphExec_t exec = nullptr;
        long long glaunch = 0;
        for (GraphEntry &g : ctx->graphs)
            if (g.sig == sig) {
                exec = g.exec;
                glaunch = g.launches;
            }
        if (!exec) {
            PM_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            st = enqueue_batch(ctx, pl, n, T, ransac, ctx->timing == 1, s);
            glaunch = ctx->launches;
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (st != PM_OK) {
                if (graph)
                    cudaGraphDestroy(graph);
                return st;
            }
            PM_CK(e);
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            PM_CK(e);
            if (ctx->graphs.size() >= 16) {
                cudaGraphExecDestroy(ctx->graphs.front().exec);
                ctx->graphs.erase(ctx->graphs.begin());
            }
            ctx->graphs.push_back(GraphEntry{sig, exec, glaunch});
        }
        PM_CK(cudaGraphLaunch(exec, s));
        ctx->launches = glaunch;
        if (bridge) {
            PM_CK(cudaEventRecord(ctx->gev[1], s));
            PM_CK(cudaStreamWaitEvent(nullptr, ctx->gev[1], 0));
        }
        return PM_OK;
    }
    return enqueue_batch(ctx, pl, n, T, ransac, ctx->timing == 1, s);
}

pm_status finish_timing(pm_ctx *ctx, bool ransac)
{
    if (ctx->timing != 1)
        return PM_OK;
    PM_CK(cudaEventElapsedTime(&ctx->stage_ms[0], ctx->ev[0], ctx->ev[1]));
    if (ransac) {
        PM_CK(cudaEventElapsedTime(&ctx->stage_ms[1], ctx->ev[1], ctx->ev[2]));
        PM_CK(cudaEventElapsedTime(&ctx->stage_ms[2], ctx->ev[2], ctx->ev[3]));
    }
    return PM_OK;
}

pm_status copy_planes(pm_ctx *ctx, int f, pm_plane *planes, int max_planes, int *n_planes)
{
    int np = ctx->h_state[f].n_planes;
    if (np < 0 || np > MAX_PLANES)
        return fail(PM_ERR_CUDA, "corrupt plane count read back from the device");
    int k = np < max_planes ? np : max_planes;
    if (planes && k > 0)
        std::memcpy(planes, ctx->h_planes + (size_t)f * MAX_PLANES, k * sizeof(pm_plane));
    if (n_planes)
        *n_planes = k;
    return PM_OK;
}

}  // namespace

// ===========================================================================
// exported entry points
// ===========================================================================
extern "C" {

long long pm_scratch_bytes(int max_w, int max_h, int max_frames, int hypotheses, int max_planes)
{
    (void)max_planes;
    if (max_w < 1 || max_h < 1 || max_frames < 1 || hypotheses < 1)
        return -1;
    long long npx = (long long)max_w * max_h;
    int max_chunks = (int)((npx + CHUNK - 1) / CHUNK);
    return (long long)(make_layout(npx, max_frames, hypotheses, max_chunks).total +
                       edge_layout((size_t)npx).total +
                       region_layout(CREATE_REGIONS, (size_t)hypotheses).total);
}

pm_status pm_create(const pm_diffusion_params *dp, const pm_ransac_params *rp,
                    const pm_misc_params *mp, int max_w, int max_h, int max_frames, pm_ctx **out)
{
    if (!out)
        return fail(PM_ERR_ARG, "null output pointer");
    pm_status st = check_params(dp, rp, mp);
    if (st != PM_OK)
        return st;
    if (max_w < 1 || max_h < 1 || max_frames < 1 || max_frames > 1024)
        return fail(PM_ERR_ARG, "max_w, max_h >= 1 and max_frames in [1, 1024] required");
    if ((long long)max_w * max_h >= (1ll << 31) / 2)
        return fail(PM_ERR_ARG, "max_w * max_h too large for 32-bit pixel indices");
    pm_ctx *ctx = new pm_ctx();
    ctx->dp = *dp;
    ctx->rp = *rp;
    ctx->mp = *mp;
    ctx->max_w = max_w;
    ctx->max_h = max_h;
    ctx->max_frames = max_frames;
    ctx->max_npx = (long long)max_w * max_h;
    ctx->max_chunks = (int)((ctx->max_npx + CHUNK - 1) / CHUNK);
    ctx->lay = make_layout(ctx->max_npx, max_frames, rp->hypotheses, ctx->max_chunks);
    auto bail = [&](pm_status s) {
        pm_destroy(ctx);
        return s;
    };
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess)
        e = diffuse_init();
    if (e == cudaSuccess)
        e = score_init();
    if (e != cudaSuccess)
        return bail(fail(PM_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e)));
    e = cudaMalloc(&ctx->arena, ctx->lay.total);
    if (e != cudaSuccess) {
        ctx->arena = nullptr;
        cudaGetLastError();
        return bail(fail(PM_ERR_OOM, "scratch arena of " + std::to_string(ctx->lay.total) +
                                         " bytes: " + cudaGetErrorString(e)));
    }
    // the edge / region passes' scratch and the per-region RANSAC scratch
    // for CREATE_REGIONS regions, so that those calls allocate nothing
    const EdgeLayout EL = edge_layout((size_t)ctx->max_npx);
    const RegionLayout RL = region_layout(CREATE_REGIONS, (size_t)rp->hypotheses);
    e = cudaMalloc(&ctx->eg, EL.total);
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->rg, RL.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PM_ERR_OOM, std::string("edge / region scratch: ") + cudaGetErrorString(e)));
    }
    ctx->rg_cap = RL.total;
    e = cudaMemset(ctx->eg + EL.err, 0, 4);
    if (e == cudaSuccess)
        e = cudaMallocHost(&ctx->h_eg, 2 * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMallocHost(&ctx->h_rg, CREATE_REGIONS * sizeof(pm_region_plane));
    if (e == cudaSuccess) {
        ctx->h_rg_cap = CREATE_REGIONS;
        e = cudaMemset(ctx->arena + ctx->lay.counter, 0, 4 * (1 + MAX_PLANES));
    }
    if (e == cudaSuccess)
        e = cudaMallocHost(&ctx->h_state, max_frames * sizeof(RState));
    if (e == cudaSuccess)
        e = cudaMallocHost(&ctx->h_planes, (size_t)max_frames * MAX_PLANES * sizeof(pm_plane));
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        e = cudaEventCreate(&ctx->ev[i]);
    for (int i = 0; i < 2 * MAX_PLANES && e == cudaSuccess; ++i)
        e = cudaEventCreate(&ctx->kev[i]);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PM_ERR_OOM, std::string("pinned host staging: ") + cudaGetErrorString(e)));
    }
    st = ensure_tables(ctx, 64 * 1024);
    if (st != PM_OK)
        return bail(st);
    *out = ctx;
    return PM_OK;
}

void pm_destroy(pm_ctx *ctx)
{
    if (!ctx)
        return;
    cudaDeviceSynchronize();
    for (GraphEntry &g : ctx->graphs)
        cudaGraphExecDestroy(g.exec);
    if (ctx->rg)
        cudaFree(ctx->rg);
    if (ctx->h_rg)
        cudaFreeHost(ctx->h_rg);
    if (ctx->eg)
        cudaFree(ctx->eg);
    if (ctx->h_eg)
        cudaFreeHost(ctx->h_eg);
    if (ctx->gstream)
        cudaStreamDestroy(ctx->gstream);
    for (int i = 0; i < 2; ++i)
        if (ctx->gev[i])
            cudaEventDestroy(ctx->gev[i]);
    for (int i = 0; i < 4; ++i)
        if (ctx->ev[i])
            cudaEventDestroy(ctx->ev[i]);
    for (int i = 0; i < 2 * MAX_PLANES; ++i)
        if (ctx->kev[i])
            cudaEventDestroy(ctx->kev[i]);
    if (ctx->arena)
        cudaFree(ctx->arena);
    if (ctx->d_tables)
        cudaFree(ctx->d_tables);
    if (ctx->h_tables)
        cudaFreeHost(ctx->h_tables);
    if (ctx->h_state)
        cudaFreeHost(ctx->h_state);
    if (ctx->h_planes)
        cudaFreeHost(ctx->h_planes);
    delete ctx;
}

pm_status pm_diffuse(pm_ctx *ctx, const void *depth, int dtype, int w, int h, int pitch,
                     float *out, void *stream)
{
    Range range_("pm_diffuse");
    if (!ctx || !out)
        return fail(PM_ERR_ARG, "null context or output");
    if (misaligned(out, 4))
        return fail(PM_ERR_ARG, "output pointer not 4-byte aligned");
    pm_status st = check_frame(ctx, depth, dtype, w, h, pitch, nullptr);
    if (st != PM_OK)
        return st;
    // the iterate lives in the context's scratch, which a pending batch still uses
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->dp.iters_per_launch == 1) {
        // one iteration per launch: the streaming kernel, ping-pong in scratch
        const int it = ctx->dp.iters;
        const long long npx = (long long)w * h;
        for (int k = 0; k < (it > 0 ? it : 1); ++k) {
            DiffFrame d{};
            const bool lastk = k == (it > 0 ? it : 1) - 1;
            d.src = depth;
            d.src_dtype = dtype;
            d.src_pitch = pitch;
            d.lo_in = k == 0 ? nullptr : ctx->at<float>(ctx->lay.buf[(k - 1) & 1]);
            d.w = w;
            d.h = h;
            d.dst = lastk ? out : ctx->at<float>(ctx->lay.buf[k & 1]);
            d.dst_lo = lastk ? 0 : 1;
            d.n_iters = it > 0 ? 1 : 0;
            d.scale = ctx->mp.depth_scale;
            (void)npx;
            PM_CK(launch_diffuse_stream(d, ctx->dp.lambda, ctx->dp.K, ctx->dp.mode, s));
        }
        return PM_OK;
    }
    std::vector<FrameJob> jobs(1);
    jobs[0] = FrameJob{depth, dtype, w, h, pitch, 1, 1, 0, 0, 0, ctx->dp.iters, nullptr, out};
    return run_batch(ctx, jobs, false, false, s);
}

pm_status pm_normals(pm_ctx *ctx, const float *depth, int w, int h, const pm_intrinsics *K,
                     float *points, float *normals, unsigned char *valid, void *stream)
{
    Range range_("pm_normals");
    if (!ctx || !K || !points || !normals || !valid)
        return fail(PM_ERR_ARG, "null argument");
    if (misaligned(points, 4) || misaligned(normals, 4))
        return fail(PM_ERR_ARG, "points / normals not 4-byte aligned");
    pm_status st = check_frame(ctx, depth, PM_F32_M, w, h, (long long)w * 4, K);
    if (st != PM_OK)
        return st;
    PM_CK(launch_normals(depth, w, h, (float)K->fx, (float)K->fy, (float)K->cx, (float)K->cy,
                         ctx->mp.normal_stencil, points, normals, valid, (cudaStream_t)stream));
    return PM_OK;
}

pm_status pm_ransac_planes(pm_ctx *ctx, const float *points, const float *normals,
                           const unsigned char *valid, int w, int h, unsigned long long frame_idx,
                           pm_plane *planes, int max_planes, int *n_planes, short *labels,
                           void *stream)
{
    Range range_("pm_ransac_planes");
    if (!ctx || !points || !valid || !planes || !n_planes || max_planes < 0)
        return fail(PM_ERR_ARG, "null argument");
    if (w < 1 || h < 1 || (long long)w * h > ctx->max_npx)
        return fail(PM_ERR_ARG, "image size out of range for this context");
    if (misaligned(points, 4) || misaligned(normals, 4) || misaligned(labels, 2))
        return fail(PM_ERR_ARG, "points / normals / labels not aligned to their element size");
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    cudaStream_t s = (cudaStream_t)stream;
    const Layout &Ly = ctx->lay;
    RFrame r;
    r.P = points;
    r.N = normals;
    r.valid = valid;
    r.labels = labels ? labels : ctx->at<short>(Ly.labels);
    r.w = w;
    r.h = h;
    r.npx = w * h;
    r.frame_idx = frame_idx;
    for (int b = 0; b < 2; ++b) {
        r.cpt[b] = ctx->at<float4>(Ly.cpt[b]);
    }
    r.hyp = ctx->at<float4>(Ly.hyp);
    r.hyp_p0 = ctx->at<float4>(Ly.hyp_p0);
    r.counts = ctx->at<int>(Ly.counts);
    r.kept = ctx->at<int>(Ly.kept);
    r.keepbits = ctx->at<unsigned>(Ly.keepbits);
    r.partial = ctx->at<float>(Ly.partial);
    r.st = ctx->at<RState>(Ly.state);
    r.planes = ctx->at<pm_plane>(Ly.planes);
    std::memcpy(ctx->h_tables, &r, sizeof(RFrame));
    ctx->launches = 0;
    ctx->last_n = 1;
    PM_CK(cudaMemcpyAsync(ctx->d_tables, ctx->h_tables, sizeof(RFrame), cudaMemcpyHostToDevice, s));
    pm_status st = enqueue_ransac(ctx, reinterpret_cast<RFrame *>(ctx->d_tables), 1,
                                  ((long long)w * h + CHUNK - 1) / CHUNK, s);
    if (st != PM_OK)
        return st;
    PM_CK(cudaMemcpyAsync(ctx->h_state, ctx->at<RState>(Ly.state), sizeof(RState),
                          cudaMemcpyDeviceToHost, s));
    PM_CK(cudaMemcpyAsync(ctx->h_planes, ctx->at<pm_plane>(Ly.planes), MAX_PLANES * sizeof(pm_plane),
                          cudaMemcpyDeviceToHost, s));
    PM_CK(cudaStreamSynchronize(s));
    return copy_planes(ctx, 0, planes, max_planes, n_planes);
}

pm_status pm_process_frame(pm_ctx *ctx, const void *depth, int dtype, int w, int h, int pitch,
                           const pm_intrinsics *K, unsigned long long frame_idx, pm_plane *planes,
                           int max_planes, int *n_planes, short *labels, void *stream)
{
    Range range_("pm_process_frame");
    if (!ctx || !K || !planes || !n_planes || max_planes < 0)
        return fail(PM_ERR_ARG, "null argument");
    if (misaligned(labels, 2))
        return fail(PM_ERR_ARG, "labels not 2-byte aligned");
    pm_status st = check_frame(ctx, depth, dtype, w, h, pitch, K);
    if (st != PM_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<FrameJob> jobs(1);
    jobs[0] = FrameJob{depth, dtype, w, h, pitch, (float)K->fx, (float)K->fy, (float)K->cx,
                       (float)K->cy, frame_idx, ctx->dp.iters, labels, nullptr};
    st = run_batch(ctx, jobs, true, true, s);
    if (st != PM_OK)
        return st;
    PM_CK(cudaStreamSynchronize(s));
    st = finish_timing(ctx, true);
    if (st != PM_OK)
        return st;
    return copy_planes(ctx, 0, planes, max_planes, n_planes);
}

pm_status pm_process_frame_host(pm_ctx *ctx, const void *depth_host, int dtype, int w, int h,
                                int pitch, const pm_intrinsics *K, unsigned long long frame_idx,
                                pm_plane *planes, int max_planes, int *n_planes,
                                short *labels_host, void *stream)
{
    Range range_("pm_process_frame_host");
    if (!ctx || !K || !planes || !n_planes || max_planes < 0)
        return fail(PM_ERR_ARG, "null argument");
    pm_status st = check_frame(ctx, depth_host, dtype, w, h, pitch, K);
    if (st != PM_OK)
        return st;
    // the host depth is staged in the context's scratch, which a pending batch still uses
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    cudaStream_t s = (cudaStream_t)stream;
    const int es = elem_size(dtype);
    void *d_in = ctx->at<char>(ctx->lay.input);
    PM_CK(cudaMemcpy2DAsync(d_in, (size_t)w * es, depth_host, pitch, (size_t)w * es, h,
                            cudaMemcpyHostToDevice, s));
    short *d_lab = ctx->at<short>(ctx->lay.labels);
    std::vector<FrameJob> jobs(1);
    jobs[0] = FrameJob{d_in, dtype, w, h, (long long)w * es, (float)K->fx, (float)K->fy,
                       (float)K->cx, (float)K->cy, frame_idx, ctx->dp.iters, d_lab, nullptr};
    st = run_batch(ctx, jobs, true, true, s);
    if (st != PM_OK)
        return st;
    if (labels_host)
        PM_CK(cudaMemcpyAsync(labels_host, d_lab, (size_t)w * h * 2, cudaMemcpyDeviceToHost, s));
    PM_CK(cudaStreamSynchronize(s));
    return copy_planes(ctx, 0, planes, max_planes, n_planes);
}

static pm_status batch_jobs(pm_ctx *ctx, const pm_frame *frames, int n,
                            std::vector<FrameJob> &jobs)
{
    if (!ctx || !frames || n < 1)
        return fail(PM_ERR_ARG, "null context/frames or empty batch");
    if (n > ctx->max_frames)
        return fail(PM_ERR_ARG, "batch larger than the context's max_frames");
    jobs.resize(n);
    for (int f = 0; f < n; ++f) {
        const pm_frame &fr = frames[f];
        pm_status st = check_frame(ctx, fr.depth, fr.dtype, fr.w, fr.h, fr.pitch, &fr.K);
        if (st != PM_OK)
            return fail(st, "frame " + std::to_string(f) + ": " + g_err);
        if (misaligned(fr.labels, 2) || misaligned(fr.depth_out, 4))
            return fail(PM_ERR_ARG, "frame " + std::to_string(f) +
                                        ": labels / depth_out not aligned to their element size");
        const int it = fr.iters < 0 ? ctx->dp.iters : fr.iters;
        if (it > 100000)
            return fail(PM_ERR_ARG, "frame " + std::to_string(f) + ": iters out of range");
        jobs[f] = FrameJob{fr.depth, fr.dtype, fr.w, fr.h, fr.pitch, (float)fr.K.fx, (float)fr.K.fy,
                           (float)fr.K.cx, (float)fr.K.cy, fr.frame_idx, it, fr.labels,
                           fr.depth_out};
    }
    return PM_OK;
}

pm_status pm_process_batch(pm_ctx *ctx, const pm_frame *frames, int n, pm_plane *planes,
                           int *n_planes, int use_graph, void *stream)
{
    Range range_("pm_process_batch");
    if (!planes || !n_planes)
        return fail(PM_ERR_ARG, "null output");
    std::vector<FrameJob> jobs;
    pm_status st = batch_jobs(ctx, frames, n, jobs);
    if (st != PM_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = run_batch(ctx, jobs, true, use_graph != 0, s);
    if (st != PM_OK)
        return st;
    PM_CK(cudaStreamSynchronize(s));
    st = finish_timing(ctx, true);
    if (st != PM_OK)
        return st;
    for (int f = 0; f < n; ++f) {
        st = copy_planes(ctx, f, planes + (size_t)f * ctx->rp.max_planes, ctx->rp.max_planes,
                         n_planes + f);
        if (st != PM_OK)
            return st;
    }
    return PM_OK;
}

pm_status pm_process_batch_async(pm_ctx *ctx, const pm_frame *frames, int n, int use_graph,
                                 void *stream)
{
    Range range_("pm_process_batch_async");
    std::vector<FrameJob> jobs;
    pm_status st = batch_jobs(ctx, frames, n, jobs);
    if (st != PM_OK)
        return st;
    st = run_batch(ctx, jobs, true, use_graph != 0, (cudaStream_t)stream);
    if (st != PM_OK)
        return st;
    ctx->pending_n = n;
    return PM_OK;
}

pm_status pm_process_batch_host_async(pm_ctx *ctx, const pm_frame *frames, int n, int use_graph,
                                      void *stream)
{
    Range range_("pm_process_batch_host_async");
    std::vector<FrameJob> jobs;
    pm_status st = batch_jobs(ctx, frames, n, jobs);
    if (st != PM_OK)
        return st;
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    cudaStream_t s = (cudaStream_t)stream;
    // frame f is staged in input slot f (max_npx * 4 bytes), outside any
    // graph, so the batch's captured launch sequence sees fixed addresses
    for (int f = 0; f < n; ++f) {
        FrameJob &j = jobs[f];
        const size_t row = (size_t)j.w * elem_size(j.dtype);
        char *slot = ctx->at<char>(ctx->lay.input) + (size_t)f * ctx->max_npx * 4;
        PM_CK(cudaMemcpy2DAsync(slot, row, j.src, (size_t)j.pitch, row, j.h,
                                cudaMemcpyHostToDevice, s));
        j.src = slot;
        j.pitch = (long long)row;
    }
    st = run_batch(ctx, jobs, true, use_graph != 0, s);
    if (st != PM_OK)
        return st;
    ctx->pending_n = n;
    return PM_OK;
}

pm_status pm_batch_collect(pm_ctx *ctx, pm_plane *planes, int *n_planes, int n)
{
    if (!ctx || !planes || !n_planes)
        return fail(PM_ERR_ARG, "null argument");
    if (ctx->pending_n == 0 || n != ctx->pending_n)
        return fail(PM_ERR_STATE, "no pending batch of that size");
    ctx->pending_n = 0;
    for (int f = 0; f < n; ++f) {
        pm_status st = copy_planes(ctx, f, planes + (size_t)f * ctx->rp.max_planes,
                                   ctx->rp.max_planes, n_planes + f);
        if (st != PM_OK)
            return st;
    }
    return PM_OK;
}

pm_status pm_frame_geometry(pm_ctx *ctx, int frame, float *points, float *normals,
                            unsigned char *valid, void *stream)
{
    Range range_("pm_frame_geometry");
    if (!ctx)
        return fail(PM_ERR_ARG, "null context");
    if (frame < 0 || 2 * (size_t)frame >= ctx->geom_wh.size())
        return fail(PM_ERR_ARG, "no frame of that index in the last whole-path call");
    if (misaligned(points, 4) || misaligned(normals, 4))
        return fail(PM_ERR_ARG, "points / normals not 4-byte aligned");
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    const size_t npx = (size_t)ctx->geom_wh[2 * frame] * ctx->geom_wh[2 * frame + 1];
    const size_t slot = (size_t)frame * ctx->max_npx;
    cudaStream_t s = (cudaStream_t)stream;
    if (points)
        PM_CK(cudaMemcpyAsync(points, ctx->at<float>(ctx->lay.P) + 3 * slot, 3 * npx * 4,
                              cudaMemcpyDeviceToDevice, s));
    if (normals)
        PM_CK(cudaMemcpyAsync(normals, ctx->at<float>(ctx->lay.N) + 3 * slot, 3 * npx * 4,
                              cudaMemcpyDeviceToDevice, s));
    if (valid)
        PM_CK(cudaMemcpyAsync(valid, ctx->at<unsigned char>(ctx->lay.valid) + slot, npx,
                              cudaMemcpyDeviceToDevice, s));
    return PM_OK;
}

pm_status pm_ransac_regions(pm_ctx *ctx, const float *points, const unsigned char *valid,
                            const int *regions, int w, int h, int n_regions, int hypotheses,
                            unsigned long long frame_idx, pm_region_plane *out, void *stream)
{
    Range range_("pm_ransac_regions");
    if (!ctx || !points || !valid || !regions || !out)
        return fail(PM_ERR_ARG, "null argument");
    if (misaligned(points, 4) || misaligned(regions, 4))
        return fail(PM_ERR_ARG, "points / regions not 4-byte aligned");
    if (w < 1 || h < 1 || (long long)w * h > ctx->max_npx)
        return fail(PM_ERR_ARG, "image size out of range for this context");
    if (n_regions < 1 || n_regions > 65535)
        return fail(PM_ERR_ARG, "n_regions must lie in [1, 65535]");
    if (hypotheses < 1 || hypotheses > MAX_HYP)
        return fail(PM_ERR_ARG, "hypotheses must lie in [1, 2048]");
    if ((long long)n_regions * hypotheses > (1ll << 22))
        return fail(PM_ERR_ARG, "n_regions * hypotheses above 2^22");
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    const size_t R = (size_t)n_regions;
    const RegionLayout RL = region_layout(R, (size_t)hypotheses);
    cudaStream_t s = (cudaStream_t)stream;
    if (RL.total > ctx->rg_cap || n_regions > ctx->h_rg_cap) {
        // more than the scratch pm_create sized: grow it, but never inside a
        // stream capture (an allocation there would fail or break the capture)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        PM_CK(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return fail(PM_ERR_STATE, "region scratch smaller than n_regions x hypotheses while "
                                      "the stream is being captured; make one such call before "
                                      "capturing");
    }
    if (RL.total > ctx->rg_cap) {
        if (ctx->rg)
            cudaFree(ctx->rg);
        ctx->rg = nullptr;
        ctx->rg_cap = 0;
        PM_CK(cudaMalloc(&ctx->rg, RL.total));
        ctx->rg_cap = RL.total;
    }
    if (n_regions > ctx->h_rg_cap) {
        if (ctx->h_rg)
            cudaFreeHost(ctx->h_rg);
        ctx->h_rg = nullptr;
        ctx->h_rg_cap = 0;
        PM_CK(cudaMallocHost(&ctx->h_rg, R * sizeof(pm_region_plane)));
        ctx->h_rg_cap = n_regions;
    }
    char *b = ctx->rg;
    RegionLaunch L;
    L.P = points;
    L.valid = valid;
    L.regions = regions;
    L.w = w;
    L.h = h;
    L.R = n_regions;
    L.H = hypotheses;
    L.frame_idx = frame_idx;
    L.seed = ctx->rp.seed;
    L.thr2 = ctx->rp.thr_m * ctx->rp.thr_m;
    L.cnt = reinterpret_cast<int *>(b + RL.cnt);
    L.box = reinterpret_cast<int *>(b + RL.box);
    L.offset = reinterpret_cast<int *>(b + RL.off);
    L.cursor = reinterpret_cast<int *>(b + RL.cur);
    L.chunk_base = reinterpret_cast<int *>(b + RL.cb);
    L.list = ctx->at<float4>(ctx->lay.cpt[0]);
    L.hyp = reinterpret_cast<float4 *>(b + RL.hyp);
    L.deg = reinterpret_cast<unsigned char *>(b + RL.deg);
    L.err = reinterpret_cast<unsigned long long *>(b + RL.err);
    L.inl = reinterpret_cast<int *>(b + RL.inl);
    L.out = reinterpret_cast<pm_region_plane *>(b + RL.out);
    PM_CK(ransac_regions(L, ctx->sms, s));
    PM_CK(cudaMemcpyAsync(ctx->h_rg, L.out, R * sizeof(pm_region_plane), cudaMemcpyDeviceToHost,
                          s));
    PM_CK(cudaStreamSynchronize(s));
    std::memcpy(out, ctx->h_rg, R * sizeof(pm_region_plane));
    return PM_OK;
}

}  // extern "C"

namespace {

// Scratch of the edge and region passes, carved from one allocation sized
// for the context's largest image.
struct EdgeScratch {
    unsigned char *state, *strong;
    int *L, *size, *pre, *bsum, *err;
};

pm_status edge_scratch(pm_ctx *ctx, EdgeScratch &x)
{
    const EdgeLayout E = edge_layout((size_t)ctx->max_npx);   // allocated by pm_create
    char *b = ctx->eg;
    x.state = reinterpret_cast<unsigned char *>(b + E.state);
    x.strong = reinterpret_cast<unsigned char *>(b + E.strong);
    x.L = reinterpret_cast<int *>(b + E.L);
    x.size = reinterpret_cast<int *>(b + E.size);
    x.pre = reinterpret_cast<int *>(b + E.pre);
    x.bsum = reinterpret_cast<int *>(b + E.bsum);
    x.err = reinterpret_cast<int *>(b + E.err);
    return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_canny(pm_ctx *ctx, const float *normals, const unsigned char *valid, int w, int h,
                   int low, int high, unsigned char *edges, void *stream)
{
    Range range_("pm_canny");
    if (!ctx || !normals || !valid || !edges)
        return fail(PM_ERR_ARG, "null argument");
    if (misaligned(normals, 4))
        return fail(PM_ERR_ARG, "normals not 4-byte aligned");
    if (w < 1 || h < 1 || (long long)w * h > ctx->max_npx)
        return fail(PM_ERR_ARG, "image size out of range for this context");
    if (low < 0 || high < low)
        return fail(PM_ERR_ARG, "thresholds must satisfy 0 <= low <= high");
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    EdgeScratch x;
    const pm_status st = edge_scratch(ctx, x);
    if (st != PM_OK)
        return st;
    EdgeLaunch E;
    E.N = normals;
    E.valid = valid;
    E.w = w;
    E.h = h;
    E.low = low;
    E.high = high;
    E.state = x.state;
    E.strong = x.strong;
    E.edges = edges;
    E.L = x.L;
    E.err = x.err;
    PM_CK(canny_edges(E, (cudaStream_t)stream));
    ctx->launches = 5;
    return PM_OK;
}

pm_status pm_segment(pm_ctx *ctx, const unsigned char *edges, const unsigned char *valid, int w,
                     int h, int gap, int min_pixels, int *labels, int *n_regions, void *stream)
{
    Range range_("pm_segment");
    if (!ctx || !edges || !valid || !labels || !n_regions)
        return fail(PM_ERR_ARG, "null argument");
    if (misaligned(labels, 4))
        return fail(PM_ERR_ARG, "labels not 4-byte aligned");
    if (w < 1 || h < 1 || (long long)w * h > ctx->max_npx)
        return fail(PM_ERR_ARG, "image size out of range for this context");
    if (gap < 0 || gap > 1 || min_pixels < 1)
        return fail(PM_ERR_ARG, "gap must be 0 or 1 and min_pixels >= 1");
    if (ctx->pending_n)
        return fail(PM_ERR_STATE, "an asynchronous batch is still pending on this context");
    EdgeScratch x;
    const pm_status st = edge_scratch(ctx, x);
    if (st != PM_OK)
        return st;
    SegLaunch S;
    S.edges = edges;
    S.valid = valid;
    S.w = w;
    S.h = h;
    S.gap = gap;
    S.min_pixels = min_pixels;
    S.L = x.L;
    S.size = x.size;
    S.pre = x.pre;
    S.bsum = x.bsum;
    S.labels = labels;
    S.err = x.err;
    cudaStream_t s = (cudaStream_t)stream;
    PM_CK(segment_regions(S, s));
    const long long nb = ((long long)w * h + 1023) / 1024;
    PM_CK(cudaMemcpyAsync(ctx->h_eg, x.bsum + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CK(cudaMemcpyAsync(ctx->h_eg + 1, x.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CK(cudaStreamSynchronize(s));
    ctx->launches = 6;
    if (ctx->h_eg[1])
        return fail(PM_ERR_CUDA, "union-find walk exceeded its bound");
    *n_regions = ctx->h_eg[0];
    return PM_OK;
}

pm_status pm_set_tiling(pm_ctx *ctx, int iters_per_launch, int tile_w, int tile_h)
{
    if (!ctx)
        return fail(PM_ERR_ARG, "null context");
    const int T_eff = iters_per_launch > 0 ? iters_per_launch : DT_MAX;
    if (iters_per_launch < 0 || iters_per_launch > DT_MAX || tile_w < 0 || tile_h < 0 ||
        tile_w + 2 * T_eff > TILE_MAX_DX || tile_h + 2 * T_eff > TILE_MAX_DY)
        return fail(PM_ERR_ARG, "tiling out of range");
    ctx->dp.iters_per_launch = iters_per_launch;
    ctx->dp.tile_w = tile_w;
    ctx->dp.tile_h = tile_h;
    return PM_OK;
}

pm_status pm_set_timing(pm_ctx *ctx, int on)
{
    if (!ctx || on < 0 || on > 2)
        return fail(PM_ERR_ARG, "null context or timing mode not in {0, 1, 2}");
    ctx->timing = on;
    return PM_OK;
}

pm_status pm_kernel_stats(pm_ctx *ctx, float *score_ms, long long *score_pairs,
                          long long *evaluated_pairs, int *score_launches, long long *launches)
{
    if (!ctx)
        return fail(PM_ERR_ARG, "null context");
    if (launches)
        *launches = ctx->launches;
    if (ctx->timing != 2)
        return PM_OK;
    float tot = 0.0f;
    long long pairs = 0, evaluated = 0;
    for (int f = 0; f < ctx->last_n; ++f)
        evaluated += (long long)ctx->h_state[f].pairs_eval;
    for (int r = 0; r < ctx->rp.max_planes; ++r) {
        float ms = 0.0f;
        PM_CK(cudaEventElapsedTime(&ms, ctx->kev[2 * r], ctx->kev[2 * r + 1]));
        tot += ms;
        for (int f = 0; f < ctx->last_n; ++f)
            pairs += (long long)ctx->rp.hypotheses * ctx->h_state[f].m_hist[r];
    }
    if (score_ms)
        *score_ms = tot;
    if (score_pairs)
        *score_pairs = pairs;
    if (evaluated_pairs)
        *evaluated_pairs = evaluated;
    if (score_launches)
        *score_launches = ctx->rp.max_planes;
    return PM_OK;
}

pm_status pm_stage_times(pm_ctx *ctx, float ms[3])
{
    if (!ctx || !ms)
        return fail(PM_ERR_ARG, "null argument");
    for (int i = 0; i < 3; ++i)
        ms[i] = ctx->stage_ms[i];
    return PM_OK;
}

pm_status pm_debug_bounds(unsigned long long *status)
{
    if (!status)
        return fail(PM_ERR_ARG, "null argument");
    *status = 0ull;
#ifdef PM_DEBUG_BOUNDS
    unsigned long long v[3] = {0ull, 0ull, 0ull};
    PM_CK(bounds_diffuse(&v[0]));
    PM_CK(bounds_normals(&v[1]));
    PM_CK(bounds_ransac(&v[2]));
    for (unsigned long long x : v)
        if (x && !*status)
            *status = x;
    return PM_OK;
#else
    return fail(PM_ERR_STATE, "not a bounds-checking build (PM_DEBUG_BOUNDS)");
#endif
}

const char *pm_last_error(void) { return g_err.c_str(); }

}  // extern "C"

/*
 * pm.h -- C ABI of libpm, the B300 (sm_103a) implementation of the per-frame
 * hot path of "Real-Time Polygonal Semantic Mapping for Humanoid Robot Stair
 * Climbing" (arXiv 2411.01919):
 *
 *   depth image --(Sec. III-C, Eq. 1, Alg. 1)--> anisotropic diffusion
 *               --(Sec. III-C, Eq. 2, Alg. 1)--> back-projection + normal image
 *               --(Sec. III-D, Eq. 3, Alg. 2)--> sequential multi-plane RANSAC
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Images are row-major, pixel (u, v) = column u, row v, u in [0, w), v in [0, h).
 * - Depth is camera-frame Z in metres.  A depth that is 0, negative or not
 *   finite (u16: the value 0) is a hole.  Holes stay holes: diffusion neither
 *   fills them nor conducts across them, and they yield no points.
 * - "Device" pointers are CUDA device (or managed) memory on the current
 *   device; "host" pointers are ordinary CPU memory.  The caller owns every
 *   buffer it passes; the library owns only the scratch inside a pm_ctx.
 *   Device buffers must be aligned to their element size (2 bytes for u16 /
 *   f16 / int16, 4 for float / int32); a misaligned one returns PM_ERR_ARG.
 * - Every call is asynchronous on `stream` (a cudaStream_t passed as void*,
 *   NULL = the legacy default stream) unless it returns results in host
 *   memory, in which case it synchronises `stream` before returning.
 * - Errors: a bad argument returns PM_ERR_ARG before anything is launched; a
 *   CUDA failure returns PM_ERR_CUDA; nothing aborts the process.  The text
 *   of the last error of the calling thread is pm_last_error().
 * - A pm_ctx is not thread-safe and must not be used from two host threads at
 *   once; use one context per host thread or per stream.
 */
#ifndef PM_H
#define PM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PM_OK = 0,
    PM_ERR_ARG = 1,      /* invalid argument; nothing was launched */
    PM_ERR_OOM = 2,      /* device or pinned-host allocation failed */
    PM_ERR_CUDA = 3,     /* a CUDA call failed; see pm_last_error() */
    PM_ERR_TIMEOUT = 4,  /* a bounded device-side wait expired */
    PM_ERR_STATE = 5     /* call not valid in the context's current state */
} pm_status;

typedef enum {
    PM_U16_MM = 0,       /* uint16 in units of depth_scale metres (sensor millimetres) */
    PM_F16_M = 1,        /* IEEE binary16 metres (FP16 storage; computation is FP32) */
    PM_F32_M = 2         /* IEEE binary32 metres */
} pm_dtype;

/* Pinhole intrinsics K (Alg. 1 and Alg. 2 "camera intrinsic matrix").
 * A pixel (u, v) back-projects to z * ((u - cx)/fx, (v - cy)/fy, 1). */
typedef struct {
    double fx, fy, cx, cy;
} pm_intrinsics;

/* Alg. 1 parameters.  mode 0 (PM4) is the 4-neighbour discretisation of Eq. 1,
 *   I'_p = I_p + lambda * sum_{q in N,S,W,E} g(I_q - I_p) (I_q - I_p),
 *   g(x) = exp(-(x/K)^2);
 * mode 1 (ALG1) is Alg. 1 read literally: one conductance per pixel from the
 *   central-difference gradient magnitude times the 4-neighbour Laplacian.
 * lambda (Alg. 1's gamma) must lie in (0, 0.25] (stability of the explicit
 * scheme); K (Alg. 1's k) is in metres.  iters_per_launch is the temporal
 * blocking depth (iterations fused in one launch, 1..8); tile_w x tile_h is
 * the output tile of one CTA of the fused kernel (tile_w + 2*8 <= 144,
 * tile_h + 2*8 <= 64).  0 lets the library choose any of the three.  None of
 * them changes the result: every choice is bit-identical. */
typedef struct {
    int iters;
    float lambda;
    float K;
    int mode;
    int iters_per_launch;
    int tile_w;
    int tile_h;
} pm_diffusion_params;

/* Alg. 2 parameters (whole-frame sequential form).  Each plane round draws
 * `hypotheses` 3-point samples from Philox4x64-10 (key = (seed, 0), counter =
 * (hypothesis, round, frame_idx, 0)), scores every hypothesis against every
 * candidate point in FP32 (inlier: squared residual below thr_m^2), keeps the
 * hypothesis with the most inliers (ties: lowest index), labels its inliers,
 * refits the plane in FP64 by PCA over the inliers whose normal lies within
 * refit_normal_gate_deg of the hypothesis normal, and repeats on the points
 * not yet labelled.  It stops after max_planes planes or when the best
 * hypothesis has fewer than min_inliers inliers (min_inliers >= 3).
 * hypotheses must lie in [1, 2048]; max_planes in [1, 64].  The gate test
 * is |n_p . n_h| >= cos(gate) in FP32 (n_p the pixel's normal, n_h the
 * hypothesis normal).  Alg. 2's own selection rule (minimum total distance)
 * and 0.9 acceptance ratio are per polygon and belong to pm_ransac_regions. */
typedef struct {
    int hypotheses;
    float thr_m;
    int max_planes;
    int min_inliers;
    unsigned long long seed;
    float refit_normal_gate_deg;
} pm_ransac_params;

/* normal_stencil: 0 = central differences of back-projected points,
 * 1 = the same differences with Sobel (1,2,1) weights (Alg. 1).
 * depth_scale: metres per unit of PM_U16_MM input (0.001 for millimetres). */
typedef struct {
    int normal_stencil;
    float depth_scale;
} pm_misc_params;

/* One extracted plane n . X + d = 0 in the camera frame, |n| = 1, oriented
 * towards the camera (d > 0).  n_inliers: inliers of the winning hypothesis
 * (these pixels carry the plane's label); n_refit: points used by the refit;
 * rms: RMS distance of the refit points to the plane (metres); hyp_index:
 * index of the winning hypothesis in its round. */
typedef struct {
    double n[3];
    double d;
    int n_inliers;
    int n_refit;
    float rms;
    int hyp_index;
} pm_plane;

/* One frame of a batch (pm_process_batch).  depth: device pointer, `pitch`
 * bytes between rows; labels: device int16 [h*w] or NULL (-1 = no plane,
 * k = plane k); depth_out: device float [h*w] receiving the diffused depth, or
 * NULL; iters: diffusion iterations for this frame (< 0: the context's). */
typedef struct {
    const void *depth;
    int dtype;
    int w, h;
    int pitch;
    pm_intrinsics K;
    unsigned long long frame_idx;
    int iters;
    short *labels;
    float *depth_out;
} pm_frame;

typedef struct pm_ctx pm_ctx;

/* Create a context on the current CUDA device whose scratch holds up to
 * `max_frames` frames of at most max_w x max_h pixels each, plus the scratch
 * of the edge and region passes (pm_canny, pm_segment) for one such image and
 * of per-region RANSAC (pm_ransac_regions) for up to 256 regions at
 * rp->hypotheses hypotheses: all of it is allocated here, so no later call
 * allocates device memory except pm_ransac_regions beyond those 256 regions
 * (pm_scratch_bytes gives the total).  The parameters are copied.  Returns
 * PM_ERR_ARG for out-of-range parameters, PM_ERR_OOM if the scratch cannot be
 * allocated.  *out is set only on success. */
pm_status pm_create(const pm_diffusion_params *dp, const pm_ransac_params *rp,
                    const pm_misc_params *mp, int max_w, int max_h, int max_frames,
                    pm_ctx **out);

/* Synchronise the context's work and free its scratch.  NULL is a no-op. */
void pm_destroy(pm_ctx *ctx);

/* Alg. 1, first loop (Eq. 1): decode `depth` (dtype, pitch in bytes, w x h)
 * and run the context's diffusion for dp->iters iterations; write the FP32
 * result (metres, holes = 0, row pitch w) to device `out`. */
pm_status pm_diffuse(pm_ctx *ctx, const void *depth, int dtype, int w, int h, int pitch,
                     float *out, void *stream);

/* Alg. 1, second loop (Eq. 2), and the back-projection of Alg. 2: from FP32 device depth [h*w]
 * compute points P = z K^-1 (u, v, 1) and unit normals (SoA, device float
 * [3][h*w] each; holes get 0) and the validity byte per pixel (device
 * uint8 [h*w]: bit 0 = point valid, bit 1 = normal valid).  Normals point
 * towards the camera; they are invalid on the image border, next to a hole,
 * or where the tangent cross product vanishes. */
pm_status pm_normals(pm_ctx *ctx, const float *depth, int w, int h, const pm_intrinsics *K,
                     float *points, float *normals, unsigned char *valid, void *stream);

/* Alg. 2 (Eq. 3), whole frame: sequential RANSAC over the valid points of
 * `points` (device SoA [3][h*w]) with `valid` (device [h*w], bits as above);
 * `normals` (device SoA, or NULL: no refit gate).  Writes up to
 * min(max_planes, rp->max_planes) planes to host `planes`, their number to
 * host *n_planes, and, if `labels` is not NULL, the per-pixel plane index to
 * device int16 labels [h*w] (-1 = none).  Synchronises `stream`. */
pm_status pm_ransac_planes(pm_ctx *ctx, const float *points, const float *normals,
                           const unsigned char *valid, int w, int h,
                           unsigned long long frame_idx, pm_plane *planes, int max_planes,
                           int *n_planes, short *labels, void *stream);

/* The whole path for one frame on device input: decode, diffusion, normals,
 * RANSAC.  Outputs as in pm_ransac_planes.  Synchronises `stream`.  The launch
 * sequence is captured once per frame shape and replayed as a CUDA graph
 * (on a context-owned stream ordered with the caller's when `stream` is the
 * legacy default stream); if `stream` is being captured by the caller, the
 * kernels are launched directly into that capture instead.  A context keeps
 * the graphs of its 16 most recently captured shapes (frame or batch); a
 * seventeenth shape evicts the oldest. */
pm_status pm_process_frame(pm_ctx *ctx, const void *depth, int dtype, int w, int h, int pitch,
                           const pm_intrinsics *K, unsigned long long frame_idx,
                           pm_plane *planes, int max_planes, int *n_planes, short *labels,
                           void *stream);

/* As pm_process_frame, with the depth and the labels (may be NULL) in HOST
 * memory: the call copies the depth in and the planes and labels out on
 * `stream`.  Synchronises `stream`. */
pm_status pm_process_frame_host(pm_ctx *ctx, const void *depth_host, int dtype, int w, int h,
                                int pitch, const pm_intrinsics *K, unsigned long long frame_idx,
                                pm_plane *planes, int max_planes, int *n_planes,
                                short *labels_host, void *stream);

/* Batched form: the whole path for n frames of mixed sizes and iteration
 * counts in one pass (shared launches; per-frame results identical to
 * pm_process_frame).  planes: host [n * ctx max_planes]; n_planes: host [n].
 * If use_graph is non-zero the launch sequence is captured once per batch
 * shape and replayed as a CUDA graph.  Synchronises `stream`. */
pm_status pm_process_batch(pm_ctx *ctx, const pm_frame *frames, int n, pm_plane *planes,
                           int *n_planes, int use_graph, void *stream);

/* Asynchronous batched form for request loops: enqueue the batch on `stream`
 * and return; the planes land in the context's pinned host staging and are
 * read with pm_batch_collect after `stream` (or the event recorded by the
 * caller after this call) has completed.  A context holds one batch in flight. */
pm_status pm_process_batch_async(pm_ctx *ctx, const pm_frame *frames, int n, int use_graph,
                                 void *stream);
pm_status pm_batch_collect(pm_ctx *ctx, pm_plane *planes, int *n_planes, int n);

/* As pm_process_batch_async, with every frame's depth in HOST memory (pinned
 * memory makes the copies asynchronous; pageable memory is copied before the
 * call returns): the call copies frame f into the context's input staging on
 * `stream` and enqueues the batch after the copies.  labels and depth_out
 * are device pointers or NULL as in pm_frame.  Pinned host buffers must stay
 * unchanged until the batch completes; collect with pm_batch_collect. */
pm_status pm_process_batch_host_async(pm_ctx *ctx, const pm_frame *frames, int n, int use_graph,
                                      void *stream);

/* What the RANSAC stage (Alg. 2) of the context's last whole-path call
 * (pm_process_frame, pm_process_frame_host, pm_process_batch,
 * pm_process_batch_async or pm_process_batch_host_async) consumed for frame `frame` of its batch: the
 * back-projected points and unit normals of Eq. 2 (device float SoA
 * [3][h*w] each) and the validity bytes (device uint8 [h*w]; bits as in
 * pm_normals), w x h being that frame's size.  It lets a caller check each
 * stage of the path on the previous stage's own output.  Any output may be
 * NULL.  Device-to-device copies, asynchronous on `stream`; the data stays
 * valid until the next whole-path call on the context.  PM_ERR_ARG if the
 * last whole-path call had no such frame, PM_ERR_STATE while an asynchronous
 * batch is pending (collect it first). */
pm_status pm_frame_geometry(pm_ctx *ctx, int frame, float *points, float *normals,
                            unsigned char *valid, void *stream);

/* Per-region RANSAC in the literal form of Alg. 2 (Sec. III-D): one plane
 * model per region (e.g. a polygon of the paper's contour step).  For region r
 * (regions[p] == r, device int32 [h*w]; values outside [0, n_regions) and
 * invalid points are ignored), `hypotheses` (1..2048) hypotheses are drawn:
 * each sample is uniform over the region's valid points, by rejection in the
 * region's bounding box (Philox4x64-10, key (seed, 1), counter
 * (hypothesis, region, frame_idx, 64 * sample + attempt), up to 64 attempts;
 * a sample without a hit makes the hypothesis degenerate).  The hypothesis
 * with the minimum total distance sum_i |n . p_i + d| over the region's
 * points wins (each distance, computed in FP32 as the inlier test does, is
 * truncated to a multiple of 2^-32 m and summed in 64-bit integers, so the
 * minimum is exact; ties go to the lowest index); the model is accepted when
 * 10 * inliers > 9 * points (more than 90% inliers, threshold rp->thr_m).
 * out: host [n_regions] (n, d: the winning FP32 hypothesis plane, not refit;
 * hyp_index = -1 when the region has fewer than 3 points or no usable
 * hypothesis).  n_regions in [1, 65535] and n_regions * hypotheses <= 2^22.
 * Uses the context's seed and threshold; synchronises `stream`.  The scratch
 * pm_create allocated covers 256 regions at the context's hypothesis count; a
 * larger call grows it (a device allocation), except while `stream` is being
 * captured, when it returns PM_ERR_STATE: make one call of that size first.
 * This is where the literal selection rule of Alg. 2 (minimum total
 * distance) and its 0.9 inlier-ratio acceptance live; the whole-frame form
 * (pm_ransac_planes) takes the winner by inlier count. */
typedef struct {
    double n[3];
    double d;
    unsigned long long error;   /* sum of distances, units of 2^-32 m */
    int inliers;
    int total;
    int accepted;
    int hyp_index;
} pm_region_plane;

pm_status pm_ransac_regions(pm_ctx *ctx, const float *points, const unsigned char *valid,
                            const int *regions, int w, int h, int n_regions, int hypotheses,
                            unsigned long long frame_idx, pm_region_plane *out, void *stream);

/* Canny edges of the normal image (Sec. III-D: edge detection on the normal
 * vector image).  normals: device FP32 SoA [3][h*w] (pm_normals' layout),
 * valid: device u8 [h*w] (bit 0), edges: device u8 [h*w] out, 1 = edge.
 * Each normal component is coded to 8 bits, q = clamp(floor(fma(n, 127.5,
 * 128)), 0, 255) in FP32 (an invalid pixel codes as the zero vector, 128);
 * per channel the 3x3 Sobel derivatives (borders replicated); per pixel the
 * channel with the largest |gx| + |gy| = m (ties: lowest channel);
 * non-maximum suppression across the 22.5-degree sector of (gx, gy), decided
 * exactly in integers (kept when m > m behind and m >= m ahead, m = 0 outside
 * the image); kept pixels with m > high are strong, with m > low weak, and
 * the edges are the 8-connected components of weak and strong pixels that
 * hold a strong pixel.  No smoothing of its own: the anisotropic diffusion
 * is the smoothing step.  0 <= low <= high.  Asynchronous on `stream`. */
pm_status pm_canny(pm_ctx *ctx, const float *normals, const unsigned char *valid, int w, int h,
                   int low, int high, unsigned char *edges, void *stream);

/* Planar regions bounded by the edges: the 4-connected components of the
 * pixels that are valid, not edges and (gap = 1) have no edge among their 8
 * neighbours, which closes the one-pixel breaks non-maximum suppression
 * leaves where edge lines meet (gap = 0: only the edge pixels themselves are
 * excluded).  labels: device int32 [h*w] out: components of at least
 * min_pixels pixels numbered 0 .. n_regions - 1 in the raster order of their
 * first pixel, -1 elsewhere (the region image pm_ransac_regions takes).
 * *n_regions: host.  Synchronises `stream`. */
pm_status pm_segment(pm_ctx *ctx, const unsigned char *edges, const unsigned char *valid, int w,
                     int h, int gap, int min_pixels, int *labels, int *n_regions, void *stream);

/* ------------------------------------------------------------------------
 * Polygon map manager (Sec. III-E, Eq. 4-10).  Host code; no GPU.
 *
 * Each frame hands over the frame's planar polygons in the camera frame and
 * the camera pose (map <- camera, row-major 4x4 [R t; 0 1], from odometry).
 * Polygons whose plane normal in the map frame is within acos(horizontal_cos)
 * of vertical enter the map as convex footprints in the map's x-y plane with
 * the plane's height at the footprint's area centroid; others are skipped.
 * A new polygon matches the map polygon whose footprint overlaps it by more
 * than min_overlap_m2 and whose height differs from the new height minus the
 * current drift estimate by at most drift_tolerance_m (Eq. 4-5; closest
 * height wins, ties to the older polygon).  The frame's drift measurement is
 * the mean over its matches of (new height - map height); the scalar Kalman
 * filter predicts P += sigma_p every frame and, when the frame matched,
 * updates K = P / (P + sigma_m), x += K (z - x), P = (1 - K) P (Eq. 6-10).
 * New polygons are then lowered by the updated drift x and either merged
 * into their match (the footprint grows to the hull of both; the map
 * polygon keeps its height, the reference the drift is measured against) or
 * added.  Variances in m^2.
 * ------------------------------------------------------------------------ */
typedef struct {
    double drift_tolerance_m;   /* Eq. 5: 0.05 */
    double sigma_p;             /* process variance per frame */
    double sigma_m;             /* measurement variance */
    double initial_variance;    /* P before the first frame */
    double horizontal_cos;      /* cos of the largest tilt of a map polygon, e.g. cos 20 deg */
    double min_overlap_m2;      /* footprint overlap that counts as overlapping */
} pm_map_params;

typedef struct {
    double n[3];                /* plane n . X + d = 0 in the camera frame */
    double d;
    const double *vertices;     /* host [n_vertices][3], camera frame, on or near the plane */
    int n_vertices;             /* >= 3 */
} pm_polygon;

typedef struct {
    int matched, merged, added, skipped;
    double measurement;         /* z_k (0 when nothing matched) */
    double gain;                /* K_k (0 when nothing matched) */
    double drift_prior, drift;  /* x before and after this frame */
    double variance;            /* P after this frame */
} pm_map_step;

typedef struct pm_map pm_map;

pm_status pm_map_create(const pm_map_params *params, pm_map **out);
void pm_map_destroy(pm_map *map);
/* One frame: pose (16 doubles), polygons [n] (n may be 0); step may be NULL. */
pm_status pm_map_integrate(pm_map *map, const double *pose, const pm_polygon *polygons, int n,
                           pm_map_step *step);
int pm_map_size(const pm_map *map);
/* Map polygon i: height, footprint area, observation count, and up to cap
 * footprint vertices (x, y pairs, counter-clockwise) in xy; *n_vertices gets
 * the full count.  Any output but n_vertices may be NULL. */
pm_status pm_map_polygon(const pm_map *map, int i, double *height, double *area,
                         int *observations, double *xy, int cap, int *n_vertices);
pm_status pm_map_drift(const pm_map *map, double *drift, double *variance);

/* Change the diffusion tiling of a context (autotuning): temporal blocking
 * depth iters_per_launch (1..8) and output tile tile_w x tile_h (limits as in
 * pm_diffusion_params; 0 = library choice).  Results are bit-identical for
 * every choice; only speed changes.  PM_ERR_ARG for out-of-range values. */
pm_status pm_set_tiling(pm_ctx *ctx, int iters_per_launch, int tile_w, int tile_h);

/* Device bytes of scratch a context created with these limits allocates. */
long long pm_scratch_bytes(int max_w, int max_h, int max_frames, int hypotheses, int max_planes);

/* Instrumentation.  pm_set_timing(ctx, 1): CUDA events between the stages of
 * each call; pm_stage_times then returns the device time (ms) of the last
 * call's [0] diffusion, [1] normals, [2] RANSAC.  pm_set_timing(ctx, 2):
 * events around every scoring launch (captured into graphs too);
 * pm_kernel_stats then returns the scoring kernels' summed device time (ms),
 * the hypothesis-point pairs they scored (H x candidates per round), the
 * pairs actually evaluated (a box test settled the rest exactly: its
 * 32-candidate segment holds no inlier of the hypothesis, or only inliers)
 * and their launch count.  In every
 * mode pm_kernel_stats returns in *launches the number of kernels the last
 * call launched.  Any output pointer may be NULL. */
pm_status pm_set_timing(pm_ctx *ctx, int on);
pm_status pm_stage_times(pm_ctx *ctx, float ms[3]);
pm_status pm_kernel_stats(pm_ctx *ctx, float *score_ms, long long *score_pairs,
                          long long *evaluated_pairs, int *score_launches, long long *launches);

/* Measured throughput of the two CUDA-core pipes the path's kernels run on,
 * the denominators of their roofline fractions: *fp32_tflops, FP32 fused
 * multiply-adds at 2 FLOP each (the inlier test of Eq. 3 is three FMAs and
 * one squared-threshold FMA per point), and *ex2_tops, the special-function
 * unit's ex2 (the conductance exp(-(x/K)^2) of Eq. 1); *sm_count, the
 * device's multiprocessors.  Each is timed with CUDA events on a kernel that
 * issues only that instruction, in independent chains, on every SM at full
 * occupancy (about 0.15 s in all, synchronising `stream`), at whatever
 * clocks the device runs; no device setting is read or changed.  Any output
 * may be NULL. */
pm_status pm_measure_peaks(double *fp32_tflops, double *ex2_tops, int *sm_count, void *stream);

/* Allocation-free diffusion.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc, e.g. a hard real-time
 * control loop (cudaMalloc and cudaFree can synchronise the whole device and
 * take unbounded time) or a plug-in running inside a host framework whose own
 * allocator owns the device memory.  It needs no pm_ctx and allocates nothing:
 * the caller passes the input and the output, and the library keeps the
 * iterate (the lo parts of the compensated depth; the hi parts are decoded
 * from the input) in a fixed array of device memory that every GPU which
 * loads libpm holds until the process exits (2 x PM_NOALLOC_MAX_PIXELS x 4
 * bytes = 8 MiB).  Same arguments and result as pm_diffuse with
 * iters_per_launch = 1 (dp->iters_per_launch is ignored); w * h above
 * PM_NOALLOC_MAX_PIXELS returns PM_ERR_ARG.  The first call on a device looks
 * up the array's device address (with that device current); make that first
 * call before any stream capture.  The address is kept per device and CUDA
 * context: after cudaDeviceReset (or anything else that replaces the
 * device's context) the next call looks it up again, so that call, too,
 * belongs before any capture.  All calls share the one array: calls whose
 * GPU work overlaps (on different streams, or from different host threads
 * without ordering) race and corrupt each other's results.  Every pixel of
 * the array that a call reads was written earlier in the same call, so no
 * state carries over from one call to the next. */
#define PM_NOALLOC_MAX_PIXELS (1 << 20)
pm_status pm_diffuse_noalloc(const void *depth, int dtype, int w, int h, int pitch,
                             const pm_diffusion_params *dp, float depth_scale, float *out,
                             void *stream);

/* Bounds checks of the bounds-checking build (libpm built with
 * PM_DEBUG_BOUNDS, a stand-in for a memory sanitizer): every instrumented
 * global access of the diffusion, normal and RANSAC kernels checks its index
 * against the extent of its buffer, skips the access when it lies outside
 * and records the first such index in a device status word; nothing traps.
 * This call synchronises the device, returns the first recorded violation in
 * *status (0 if none; otherwise bit 63 set, bits 48-62 the source site -- file
 * id 1 diffusion, 2 normals, 3 RANSAC, times 4096, plus the line -- and bits
 * 0-47 the offending index) and clears the words.  In the release build it
 * returns PM_ERR_STATE and sets *status to 0. */
pm_status pm_debug_bounds(unsigned long long *status);

/* Text of the calling thread's last error ("" if none). */
const char *pm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PM_H */

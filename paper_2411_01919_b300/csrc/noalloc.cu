// noalloc.cu -- pm_diffuse_noalloc: diffusion for callers that cannot
// allocate device memory (see include/pm.h).  The ping-pong iterate lives in
// a file-scope device array, so a call needs no pm_ctx and makes no
// allocation; host code reaches the array through the address that
// cudaGetSymbolAddress returns for the current device.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "pm_internal.cuh"

namespace {

constexpr long long kMaxPixels = PM_NOALLOC_MAX_PIXELS;

// The lo parts of two compensated iterates of up to kMaxPixels pixels each
// (the hi parts are decoded from the input by every launch): 8 MiB, held by
// every device that loads the library until the process exits.
static __device__ __align__(256) float g_iterate[2 * kMaxPixels];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (0 if the driver
// cannot tell), through the driver entry points the runtime hands out, so the
// library needs no link to the driver library.
unsigned long long current_context_id()
{
    typedef int (*get_current_fn)(void **);
    typedef int (*get_id_fn)(void *, unsigned long long *);
    static get_current_fn get_current = nullptr;
    static get_id_fn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault,
                                             &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
                cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<get_current_fn>(a);
            get_id = reinterpret_cast<get_id_fn>(b);
        }
        cudaGetLastError();
        looked_up = true;
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0)
        return id;
    return 0;
}

// Device address of g_iterate in the current context, looked up once per
// device and context, with that device current: a context created after a
// device reset gets a fresh lookup.
pm_status iterate_address(float **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return pm::set_last_error(PM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return pm::set_last_error(PM_ERR_ARG, "device ordinal beyond the supported 64");
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long cid = current_context_id();
    if (!g_addr[dev] || g_ctx_id[dev] != cid) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_iterate);
        if (e != cudaSuccess || !p)
            return pm::set_last_error(PM_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                   : "null symbol address");
        g_addr[dev] = static_cast<float *>(p);
        g_ctx_id[dev] = cid;
    }
    *out = g_addr[dev];
    return PM_OK;
}

pm_status diffuse_noalloc(const void *depth, int dtype, int w, int h, int pitch,
                          const pm_diffusion_params *dp, float depth_scale, float *out,
                          void *stream);

}  // namespace

extern "C" pm_status pm_diffuse_noalloc(const void *depth, int dtype, int w, int h, int pitch,
                                        const pm_diffusion_params *dp, float depth_scale,
                                        float *out, void *stream)
{
    using pm::set_last_error;
    nvtxRangePushA("pm_diffuse_noalloc");
    const pm_status st = diffuse_noalloc(depth, dtype, w, h, pitch, dp, depth_scale, out, stream);
    nvtxRangePop();
    return st;
}

namespace {

pm_status diffuse_noalloc(const void *depth, int dtype, int w, int h, int pitch,
                          const pm_diffusion_params *dp, float depth_scale, float *out,
                          void *stream)
{
    using pm::set_last_error;
    if (!depth || !out || !dp)
        return set_last_error(PM_ERR_ARG, "null depth, output or parameters");
    if (dtype != PM_U16_MM && dtype != PM_F16_M && dtype != PM_F32_M)
        return set_last_error(PM_ERR_ARG, "unknown depth dtype");
    if (w < 1 || h < 1)
        return set_last_error(PM_ERR_ARG, "image size must be at least 1x1");
    if ((long long)w * h > kMaxPixels)
        return set_last_error(PM_ERR_ARG,
                              "image larger than PM_NOALLOC_MAX_PIXELS (1048576 pixels)");
    const int es = dtype == PM_F32_M ? 4 : 2;
    if (((uintptr_t)depth & (es - 1)) != 0 || ((uintptr_t)out & 3) != 0)
        return set_last_error(PM_ERR_ARG, "depth or output pointer not aligned to its element size");
    if (pitch < w * es || pitch % es != 0)
        return set_last_error(PM_ERR_ARG, "pitch smaller than a row or not a multiple of the "
                                          "element size");
    if (dp->iters < 0 || dp->iters > 100000 || !(dp->lambda > 0.0f) || dp->lambda > 0.25f ||
        !(dp->K > 0.0f) || !std::isfinite(dp->K) || (dp->mode != 0 && dp->mode != 1))
        return set_last_error(PM_ERR_ARG, "diffusion parameters out of range");
    if (!(depth_scale > 0.0f) || !std::isfinite(depth_scale))
        return set_last_error(PM_ERR_ARG, "depth_scale must be positive");
    float *it = nullptr;
    pm_status st = iterate_address(&it);
    if (st != PM_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = dp->iters > 0 ? dp->iters : 1;
    for (int k = 0; k < L; ++k) {
        const bool last = k == L - 1;
        pm::DiffFrame d{};
        d.src = depth;
        d.src_dtype = dtype;
        d.src_pitch = pitch;
        d.lo_in = k == 0 ? nullptr : it + ((k - 1) & 1) * kMaxPixels;
        d.w = w;
        d.h = h;
        d.dst = last ? out : it + (k & 1) * kMaxPixels;
        d.dst_lo = last ? 0 : 1;
        d.n_iters = dp->iters > 0 ? 1 : 0;
        d.scale = depth_scale;
        cudaError_t e = pm::launch_diffuse_stream(d, dp->lambda, dp->K, dp->mode, s);
        if (e != cudaSuccess)
            return set_last_error(PM_ERR_CUDA, cudaGetErrorString(e));
    }
    return PM_OK;
}

}  // namespace

// noalloc.cu -- gs_depth_range_noalloc: the robust depth-range estimate for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application whose device memory
// is owned by its own allocator or fixed budget and that hands this library
// only pre-allocated buffers, or code that must not trigger cudaMalloc's
// implicit device synchronisation while other work is in flight.  For them
// this entry point needs no context and no allocation: its scratch (one
// bin-parameter record) is a file-scope static __device__ array that every GPU
// loading the library holds until exit.
#include <cuda.h>  // driver API types only; the functions come from cudaGetDriverEntryPointByVersion

#include <mutex>

#include "internal.cuh"

namespace {

// One record: range, logs and up to GS_MAX_K - 1 split depths (536 bytes).
static __device__ __align__(256) gs::BinParams g_depth_range_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
struct ScratchAddr {
    unsigned long long ctx_id;  // the context the address was resolved in
    void* addr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the calling thread's current context (0 when there is none
// yet or the driver cannot say).  Ids are never reused within a process, so
// a context re-created after a device reset gets a new one.  Called with
// g_scratch_mu held.
unsigned long long current_context_id()
{
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
        if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (g_ctx_get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch on the current device.  The array's name in
// host code is only a host-side stand-in, so the address is resolved with
// that device current: once per device, and again whenever the device's
// current context is a different one (after a device reset the module is
// loaded anew and the old address is stale).
int scratch_for_current_device(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gs_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long id = current_context_id();
    ScratchAddr& s = g_scratch[dev];
    if (!s.addr || id == 0 || s.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_depth_range_scratch);  // makes the primary context current if needed
        if (e != cudaSuccess || !p) return gs_cuda_fail(e, "cudaGetSymbolAddress");
        s.addr = p;
        s.ctx_id = current_context_id();
    }
    *out = s.addr;
    return GS_OK;
}

}  // namespace

extern "C" int gs_depth_range_noalloc(const gs_config* cfg, const void* projected, const float* scales,
                                      int64_t n, const gs_camera* cam, const void* isect, int64_t m_cap,
                                      const int64_t* m_dev, float* zrange, void* stream)
{
    if (gs::check_config(cfg) != GS_OK) return GS_ERR_INVALID_ARG;
    // the scratch holds K - 1 <= GS_MAX_K - 1 splits; the sample buffer lives
    // in shared memory and holds at most 8192 samples
    if (cfg->K > GS_MAX_K || cfg->sample_count > 8192) return GS_ERR_INVALID_ARG;
    if (!cam || cam->width <= 0 || cam->height <= 0 || !(cam->far_plane > cam->near_plane)) return GS_ERR_INVALID_ARG;
    if (n < 0 || m_cap < 0 || m_cap > INT32_MAX - 1 || !m_dev || !zrange) return GS_ERR_INVALID_ARG;
    if ((n > 0 && !projected) || (m_cap > 0 && !isect) || (cfg->near_shift && !scales)) return GS_ERR_INVALID_ARG;
    void* scratch = nullptr;
    int r = scratch_for_current_device(&scratch);
    if (r != GS_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    gs::BinParams* bp = static_cast<gs::BinParams*>(scratch);
    // every field the kernel reads back is rewritten by this call, so nothing
    // left by the previous call needs clearing
    r = gs::launch_depth_range_into(*cfg, gs::proj_view(const_cast<void*>(projected), n), scales,
                                    gs::isect_view(const_cast<void*>(isect), m_cap), m_cap, m_dev, cam, bp, st);
    if (r != GS_OK) return r;
    GS_CUDA_TRY(cudaMemcpyAsync(zrange, &bp->zmin, 2 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return GS_OK;
}

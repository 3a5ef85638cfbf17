// kpp_noalloc.cu -- kpp_seed_noalloc: persistent-form seeding whose scratch
// lives in a fixed array inside the library instead of a caller workspace.
//
// Some callers cannot provide device memory for scratch: code that runs
// under an allocator or memory pool it does not own and may not grow, plugin
// code that only receives its inputs and outputs, and latency-critical paths
// where a cudaMalloc (which can synchronise the whole device) is not allowed.
// For them this entry point needs no workspace and allocates nothing: its
// scratch is the file-scope device array below, which every GPU that loads
// the library holds until the process exits.
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "kpp.h"
#include "kpp_internal.h"

namespace kpp {
namespace {

// The fixed scratch: the persistent form's control block and its two
// buffers of tagged block sums need 256 + 64 * nblocks bytes (rounded up to
// 256), so 16 KiB serves up to 252 CTAs -- one per SM on a GB300 with room
// to spare.
constexpr size_t kNoAllocScratchBytes = 16 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol
// itself is only a host-side stand-in; the device address has to be asked
// for with cudaGetSymbolAddress while that device is current.  The address
// is looked up on the first call on a device and kept together with the
// context it belongs to: if that context is torn down and replaced (e.g. by
// cudaDeviceReset), the module is loaded again at another address, so a
// changed context triggers a fresh lookup.
std::mutex g_mutex;
struct ScratchAddr {
    CUcontext ctx;
    void *ptr;
};
ScratchAddr g_scratch[64] = {};

PFN_cuCtxGetCurrent_v4000 ctx_get_current()
{
    static std::once_flag once;
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    });
    return fn;
}

CUcontext current_context()
{
    auto fn = ctx_get_current();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS)
        return nullptr;
    return c;
}

kpp_status scratch_for_current_device(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return KPP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    const CUcontext ctx = current_context();
    if (!g_scratch[dev].ptr || !ctx || g_scratch[dev].ctx != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return KPP_ERR_CUDA;
        g_scratch[dev].ptr = p;
        g_scratch[dev].ctx = current_context(); // the lookup made the context current
    }
    *out = g_scratch[dev].ptr;
    return KPP_OK;
}

} // namespace
} // namespace kpp

extern "C" kpp_status kpp_seed_noalloc(const void *points, const float *row_scales, int64_t N,
                                       int32_t d, int32_t K, kpp_dtype dtype, uint64_t seed,
                                       uint64_t stream_id, int64_t *indices_out, float *d2_out,
                                       double *phi_out, kpp_stream_t stream,
                                       const kpp_options *opts, int32_t *device_status)
{
    kpp_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts)
        o = *opts;
    o.form = KPP_FORM_PERSISTENT;
    kpp_plan plan;
    const kpp_status st = kpp_describe(N, d, K, dtype, &o, &plan);
    if (st != KPP_OK)
        return st;
    if ((size_t)plan.workspace_bytes > kpp::kNoAllocScratchBytes)
        return KPP_ERR_WORKSPACE; // more scratch than the fixed array holds
    void *scratch = nullptr;
    const kpp_status sst = kpp::scratch_for_current_device(&scratch);
    if (sst != KPP_OK)
        return sst;
    // kpp_seed clears the part of the scratch that must start at zero.
    const kpp_status est = kpp_seed(points, row_scales, N, d, K, dtype, seed, stream_id, nullptr,
                                    0, indices_out, d2_out, phi_out, scratch,
                                    kpp::kNoAllocScratchBytes, stream, &o);
    if (est != KPP_OK || !device_status)
        return est;
    // the device status word is the first word of the scratch
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(device_status, scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return KPP_ERR_CUDA;
    return KPP_OK;
}

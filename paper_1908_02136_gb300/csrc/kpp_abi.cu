// kpp_abi.cu -- the C ABI of libkpp (declared in include/kpp.h): argument
// checks, workspace layout, the choice of form and specialisation, and the
// CUDA-graph cache of the streamed form.  No entry point allocates device
// memory.
#include <cstring>
#include <list>
#include <mutex>

#include "kpp.h"
#include "kpp_internal.h"

namespace kpp {
namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxDim = 4096;
constexpr int kDefaultCtasPerSm = 4;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

int elem_bytes(int dt) { return dt == KPP_F32 ? 4 : dt == KPP_BF16 ? 2 : 1; }

struct Plan {
    int form;
    StreamedKernel sk;
    int grid;       // CTAs per launch
    int64_t chunk;  // rows per CTA
    int nblocks;    // CTAs owning rows (== grid for the streamed form)
    size_t ws_bytes;
};

bool shape_ok(int64_t N, int32_t d, int32_t K, int dt)
{
    return N >= 1 && N < (int64_t(1) << 31) && d >= 1 && d <= kMaxDim && K >= 1 && K <= N &&
           dt >= KPP_F32 && dt <= KPP_FP8_E4M3;
}

kpp_status make_plan(int64_t N, int32_t d, int32_t K, int dt, const kpp_options *opts, Plan *pl)
{
    if (!shape_ok(N, d, K, dt))
        return KPP_ERR_INVALID_ARG;
    kpp_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts)
        o = *opts;
    if (o.form != KPP_FORM_AUTO && o.form != KPP_FORM_STREAMED)
        return KPP_ERR_UNSUPPORTED;
    const int sms = device_sms();
    if (sms <= 0)
        return KPP_ERR_CUDA;
    if (!streamed_lookup(dt, d, o.lanes_per_row, &pl->sk))
        return KPP_ERR_UNSUPPORTED;
    int per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : kDefaultCtasPerSm;
    if (per_sm > 32)
        return KPP_ERR_INVALID_ARG;
    int resident = 0;
    const size_t smem = pl->sk.generic ? sizeof(float) * (size_t)d : 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, pl->sk.fn, streamed_threads(),
                                                      smem) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (resident >= 1 && per_sm > resident)
        per_sm = resident; // one wave: every CTA resident at once
    const int64_t target = (int64_t)sms * per_sm;
    int64_t chunk = (N + target - 1) / target;
    const int64_t a = pl->sk.rows_align;
    chunk = (chunk + a - 1) / a * a;
    pl->form = KPP_FORM_STREAMED;
    pl->chunk = chunk;
    pl->nblocks = (int)((N + chunk - 1) / chunk);
    pl->grid = pl->nblocks;
    pl->ws_bytes = sizeof(Control) + round_up(sizeof(double) * (size_t)pl->nblocks, kAlign);
    return KPP_OK;
}

// ---------------------------------------------------------------------------
// Graph cache of the streamed form: one executable graph per distinct
// argument set (pointers, sizes, seed, specialisation, device).
// ---------------------------------------------------------------------------
struct GraphKey {
    int device;
    int grid;
    const void *fn;
    Problem p;
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
};

std::mutex g_mutex;
std::list<GraphEntry> g_cache; // most recent first
constexpr size_t kCacheMax = 32;
cudaStream_t g_capture_stream[64] = {};

cudaStream_t capture_stream(int dev)
{
    if (dev < 0 || dev >= 64)
        return nullptr;
    if (!g_capture_stream[dev]) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return nullptr;
        g_capture_stream[dev] = s;
    }
    return g_capture_stream[dev];
}

cudaError_t enqueue_streamed(const Plan &pl, const Problem &p, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p.ctl, 0, sizeof(Control), s);
    for (int m = 0; e == cudaSuccess && m < p.K; ++m)
        e = streamed_launch(pl.sk, pl.grid, p, m, s);
    return e;
}

kpp_status run_streamed(const Plan &pl, const Problem &p, cudaStream_t stream, int use_graph)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (stream && cudaStreamIsCapturing(stream, &cs) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (use_graph < 0 || cs != cudaStreamCaptureStatusNone) {
        // plain launches (or the caller is capturing its own graph)
        return enqueue_streamed(pl, p, stream) == cudaSuccess ? KPP_OK : KPP_ERR_LAUNCH;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return KPP_ERR_CUDA;
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.device = dev;
    key.grid = pl.grid;
    key.fn = pl.sk.fn;
    key.p = p;
    std::lock_guard<std::mutex> lock(g_mutex);
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
        if (std::memcmp(&it->key, &key, sizeof(key)) == 0) {
            g_cache.splice(g_cache.begin(), g_cache, it);
            return cudaGraphLaunch(g_cache.front().exec, stream) == cudaSuccess ? KPP_OK
                                                                               : KPP_ERR_LAUNCH;
        }
    }
    cudaStream_t cap = capture_stream(dev);
    if (!cap)
        return KPP_ERR_CUDA;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return KPP_ERR_CUDA;
    cudaError_t e = enqueue_streamed(pl, p, cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
        if (graph)
            cudaGraphDestroy(graph);
        return KPP_ERR_LAUNCH;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return KPP_ERR_LAUNCH;
    g_cache.push_front(GraphEntry{key, exec});
    while (g_cache.size() > kCacheMax) {
        cudaGraphExecDestroy(g_cache.back().exec); // freed once any launch in flight ends
        g_cache.pop_back();
    }
    return cudaGraphLaunch(exec, stream) == cudaSuccess ? KPP_OK : KPP_ERR_LAUNCH;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

} // namespace
} // namespace kpp

using namespace kpp;

extern "C" {

const char *kpp_status_string(kpp_status s)
{
    switch (s) {
    case KPP_OK:
        return "ok";
    case KPP_ERR_INVALID_ARG:
        return "invalid argument";
    case KPP_ERR_CUDA:
        return "CUDA runtime error";
    case KPP_ERR_LAUNCH:
        return "kernel launch failed";
    case KPP_ERR_TIMEOUT:
        return "bounded device wait timed out";
    case KPP_ERR_DEGENERATE:
        return "degenerate data: sum of D^2 is zero before K seeds";
    case KPP_ERR_WORKSPACE:
        return "workspace missing, misaligned or too small";
    case KPP_ERR_UNSUPPORTED:
        return "unsupported option combination";
    }
    return "unknown status";
}

int32_t kpp_version(void) { return 100; }

size_t kpp_workspace_size(int64_t N, int32_t d, int32_t K, kpp_dtype dtype,
                          const kpp_options *opts)
{
    Plan pl;
    if (make_plan(N, d, K, (int)dtype, opts, &pl) != KPP_OK)
        return 0;
    return pl.ws_bytes;
}

kpp_status kpp_seed(const void *points, const float *row_scales, int64_t N, int32_t d,
                    int32_t K, kpp_dtype dtype, uint64_t seed, uint64_t stream_id,
                    const int64_t *forced_prefix, int32_t n_forced, int64_t *indices_out,
                    float *d2_out, double *phi_out, void *workspace, size_t workspace_bytes,
                    kpp_stream_t stream, const kpp_options *opts)
{
    const int dt = (int)dtype;
    if (!points || !aligned(points, 16) || !indices_out || !d2_out || !shape_ok(N, d, K, dt))
        return KPP_ERR_INVALID_ARG;
    if ((dt == KPP_FP8_E4M3) != (row_scales != nullptr))
        return KPP_ERR_INVALID_ARG;
    if (n_forced < 0 || n_forced > K || (n_forced > 0 && !forced_prefix))
        return KPP_ERR_INVALID_ARG;
    Plan pl;
    kpp_status st = make_plan(N, d, K, dt, opts, &pl);
    if (st != KPP_OK)
        return st;
    if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < pl.ws_bytes)
        return KPP_ERR_WORKSPACE;
    Problem p;
    std::memset(&p, 0, sizeof(p));
    p.points = points;
    p.scales = row_scales;
    p.N = N;
    p.d = d;
    p.K = K;
    p.seed = seed;
    p.stream_id = stream_id;
    p.forced = forced_prefix;
    p.n_forced = n_forced;
    p.nblocks = pl.nblocks;
    p.chunk = pl.chunk;
    p.idx = indices_out;
    p.d2 = d2_out;
    p.phi = phi_out;
    p.ctl = reinterpret_cast<Control *>(workspace);
    p.block_sums = reinterpret_cast<double *>(reinterpret_cast<char *>(workspace) + sizeof(Control));
    const int use_graph = opts ? opts->use_graph : 0;
    return run_streamed(pl, p, reinterpret_cast<cudaStream_t>(stream), use_graph);
}

kpp_status kpp_read_status(const void *workspace, kpp_stream_t stream)
{
    if (!workspace)
        return KPP_ERR_WORKSPACE;
    int32_t st = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&st, workspace, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return KPP_ERR_CUDA;
    return (kpp_status)st;
}

kpp_status kpp_seed_host(const void *host_points, const float *host_scales, void *dev_points,
                         float *dev_scales, int64_t N, int32_t d, int32_t K, kpp_dtype dtype,
                         uint64_t seed, uint64_t stream_id, int64_t *host_indices,
                         float *host_d2, double *host_phi, int64_t *dev_indices, float *dev_d2,
                         double *dev_phi, void *workspace, size_t workspace_bytes,
                         kpp_stream_t stream, const kpp_options *opts)
{
    const int dt = (int)dtype;
    if (!host_points || !host_indices || !host_d2 || !shape_ok(N, d, K, dt))
        return KPP_ERR_INVALID_ARG;
    if ((dt == KPP_FP8_E4M3) && (!host_scales || !dev_scales))
        return KPP_ERR_INVALID_ARG;
    if (host_phi && !dev_phi)
        return KPP_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)N * (size_t)d * (size_t)elem_bytes(dt);
    if (!dev_points || cudaMemcpyAsync(dev_points, host_points, bytes, cudaMemcpyHostToDevice, s) !=
                           cudaSuccess)
        return KPP_ERR_INVALID_ARG;
    if (dt == KPP_FP8_E4M3 &&
        cudaMemcpyAsync(dev_scales, host_scales, sizeof(float) * (size_t)N,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    kpp_status st = kpp_seed(dev_points, dt == KPP_FP8_E4M3 ? dev_scales : nullptr, N, d, K, dtype,
                             seed, stream_id, nullptr, 0, dev_indices, dev_d2, dev_phi, workspace,
                             workspace_bytes, stream, opts);
    if (st != KPP_OK)
        return st;
    if (cudaMemcpyAsync(host_indices, dev_indices, sizeof(int64_t) * (size_t)K,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(host_d2, dev_d2, sizeof(float) * (size_t)N, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
        return KPP_ERR_CUDA;
    if (host_phi &&
        cudaMemcpyAsync(host_phi, dev_phi, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    return kpp_read_status(workspace, stream);
}

kpp_status kpp_quantize(const float *x, int64_t N, int32_t d, kpp_dtype to, void *out,
                        float *row_scales, kpp_stream_t stream)
{
    if (!x || !out || N < 1 || d < 1 || !aligned(x, 16) || !aligned(out, 16))
        return KPP_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (to == KPP_BF16) {
        if (row_scales)
            return KPP_ERR_INVALID_ARG;
        e = quantize_bf16(x, N * (int64_t)d, reinterpret_cast<uint16_t *>(out), s);
    } else if (to == KPP_FP8_E4M3) {
        if (!row_scales || d > kMaxDim)
            return KPP_ERR_INVALID_ARG;
        e = quantize_fp8(x, N, d, reinterpret_cast<uint8_t *>(out), row_scales, s);
    } else {
        return KPP_ERR_INVALID_ARG;
    }
    return e == cudaSuccess ? KPP_OK : KPP_ERR_LAUNCH;
}

} // extern "C"

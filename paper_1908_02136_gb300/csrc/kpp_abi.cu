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
    StreamedKernel sk;   // streamed form
    PersistentKernel pk; // persistent form
    const void *pfn;     // persistent kernel chosen (D^2 in smem or ping-pong)
    size_t psmem;        // its dynamic shared memory (also the small form's)
    PersistArgs pargs;
    int grid;      // CTAs per launch (== nblocks)
    int64_t chunk; // rows per CTA
    int nblocks;
    int nseg;   // segments (warps) per block
    int64_t sw; // rows per super-iteration
    // workspace layout (byte offsets after the control block)
    size_t off_bsum, off_seg, off_slots;
    size_t ws_bytes;
};

bool shape_ok(int64_t N, int32_t d, int32_t K, int dt)
{
    return N >= 1 && N < (int64_t(1) << 31) && d >= 1 && d <= kMaxDim && K >= 1 && K <= N &&
           dt >= KPP_F32 && dt <= KPP_FP8_E4M3;
}

void layout(Plan *pl, bool persistent)
{
    size_t off = sizeof(Control);
    pl->off_bsum = pl->off_seg = pl->off_slots = off;
    if (persistent) {
        // two buffers of tagged block sums, one 32-byte slot per block
        off += round_up(2 * sizeof(unsigned long long) * kSlotWords * (size_t)pl->nblocks, kAlign);
    } else {
        off += round_up(sizeof(float2) * (size_t)pl->nblocks, kAlign);
        pl->off_seg = off;
        off += round_up(sizeof(float2) * (size_t)pl->nblocks * pl->nseg, kAlign);
    }
    pl->ws_bytes = off;
}

kpp_status plan_streamed(int64_t N, int32_t d, int dt, const kpp_options &o, int sms, Plan *pl)
{
    if (!streamed_lookup(dt, d, o.lanes_per_row, &pl->sk))
        return KPP_ERR_UNSUPPORTED;
    int per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : kDefaultCtasPerSm;
    if (per_sm > 32)
        return KPP_ERR_INVALID_ARG;
    int resident = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, pl->sk.fn, streamed_threads(),
                                                      streamed_smem(pl->sk, d)) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (resident >= 1 && per_sm > resident)
        per_sm = resident; // one wave: every CTA resident at once
    int64_t target = (int64_t)sms * per_sm;
    if (target > kStage)
        target = kStage; // the draw stages every block sum at once
    const int64_t a = pl->sk.rows_align;
    int64_t chunk = (N + target - 1) / target;
    chunk = (chunk + a - 1) / a * a;
    pl->form = KPP_FORM_STREAMED;
    pl->chunk = chunk;
    pl->nblocks = (int)((N + chunk - 1) / chunk);
    pl->grid = pl->nblocks;
    pl->nseg = streamed_segments();
    pl->sw = a;
    layout(pl, false);
    return KPP_OK;
}

kpp_status plan_persistent_at(int64_t N, int32_t K, const kpp_options &o, int sms, int per_sm,
                              Plan *pl);

// The small form: one CTA, if the points and D^2 fit its shared memory.
kpp_status plan_small(int64_t N, int32_t d, int dt, Plan *pl)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
        return KPP_ERR_CUDA;
    const void *fn = small_lookup(dt, d);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
        return KPP_ERR_CUDA;
    const size_t smem = small_smem(N, d, dt);
    if (smem + fa.sharedSizeBytes > (size_t)optin)
        return KPP_ERR_UNSUPPORTED; // does not fit one SM
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return KPP_ERR_CUDA;
    pl->form = KPP_FORM_SMALL;
    pl->pfn = fn;
    pl->psmem = smem;
    pl->chunk = N;
    pl->nblocks = 1;
    pl->grid = 1;
    pl->nseg = small_threads() / 32;
    pl->sw = 1;
    pl->off_bsum = pl->off_seg = pl->off_slots = sizeof(Control);
    pl->ws_bytes = sizeof(Control);
    return KPP_OK;
}

// The persistent plan at the requested CTAs per SM, or fewer if that many
// cannot be co-resident.
kpp_status plan_persistent(int64_t N, int32_t d, int32_t K, int dt, const kpp_options &o, int sms,
                           Plan *pl)
{
    if (!persistent_lookup(dt, d, o.lanes_per_row, &pl->pk))
        return KPP_ERR_UNSUPPORTED;
    int per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : 1;
    if (per_sm > 4)
        return KPP_ERR_INVALID_ARG;
    kpp_status st = KPP_ERR_UNSUPPORTED;
    for (; per_sm >= 1; --per_sm) {
        st = plan_persistent_at(N, K, o, sms, per_sm, pl);
        if (st != KPP_ERR_UNSUPPORTED)
            return st;
    }
    return st;
}

kpp_status plan_persistent_at(int64_t N, int32_t K, const kpp_options &o, int sms, int per_sm,
                              Plan *pl)
{
    int dev = 0, coop = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
        return KPP_ERR_CUDA;
    if (!coop)
        return KPP_ERR_UNSUPPORTED;
    const int64_t a = pl->pk.rows_align;
    const int64_t min_rows = o.min_rows_per_cta > 0 ? o.min_rows_per_cta : 2048;
    const int64_t target = (int64_t)sms * per_sm;
    int64_t chunk = (N + target - 1) / target;
    if (chunk < min_rows)
        chunk = min_rows;
    chunk = (chunk + a - 1) / a * a;
    const int nblocks = (int)((N + chunk - 1) / chunk);
    if (nblocks > persistent_max_blocks())
        return KPP_ERR_UNSUPPORTED;
    // shared memory: D^2 of the block if it fits, then as many cached rows as fit
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, pl->pk.fn_smem) != cudaSuccess)
        return KPP_ERR_CUDA;
    const int64_t budget = ((int64_t)optin - (int64_t)fa.sharedSizeBytes - 1024) / per_sm;
    int64_t used = 0;
    // D^2 of the block and its 32-row chunk sums
    const int64_t d2_bytes = ((4 * chunk + 15) & ~15ll) + 8 * ((chunk + 31) / 32);
    bool d2_in_smem = d2_bytes <= budget;
    if (d2_in_smem)
        used += d2_bytes;
    // the cache holds the first `supers` super-iterations of every warp's
    // segment (so that all warps read the same share from shared memory)
    const int nseg = persistent_segments();
    const int64_t seg_supers = ((chunk / a) + nseg - 1) / nseg; // longest segment
    const int64_t unit = (int64_t)nseg * a * pl->pk.row_bytes;  // one super per warp
    int64_t supers = 0;
    if (o.smem_cache >= 0) {
        supers = (budget - used) / unit;
        if (supers > seg_supers)
            supers = seg_supers;
        if (o.smem_cache > 0 && supers * nseg * a > o.smem_cache)
            supers = (int64_t)o.smem_cache / (nseg * a);
        if (supers < 0)
            supers = 0;
    }
    pl->pfn = d2_in_smem ? pl->pk.fn_smem : pl->pk.fn_global;
    pl->psmem = (size_t)(supers * unit + (d2_in_smem ? d2_bytes : 0));
    // static + dynamic shared memory above 48 KB needs the opt-in attribute
    if (cudaFuncSetAttribute(pl->pfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pl->psmem) != cudaSuccess)
        return KPP_ERR_CUDA;
    int resident = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, pl->pfn, persistent_threads(),
                                                      pl->psmem) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (resident < 1 || (int64_t)nblocks > (int64_t)resident * sms)
        return KPP_ERR_UNSUPPORTED; // cannot be co-resident
    pl->form = KPP_FORM_PERSISTENT;
    pl->chunk = chunk;
    pl->nblocks = nblocks;
    pl->grid = nblocks;
    pl->nseg = nseg;
    pl->sw = a;
    pl->pargs.cache_supers = supers;
    pl->pargs.reverse = o.alternate >= 0 ? 1 : 0;
    pl->pargs.l2_hint = o.l2_policy == 0 ? 1 : (o.l2_policy == 2 ? 2 : 0);
    pl->pargs.timeout_ns = 1000ull * (o.timeout_us ? o.timeout_us : 2000000u);
    layout(pl, true);
    return KPP_OK;
}

kpp_status make_plan(int64_t N, int32_t d, int32_t K, int dt, const kpp_options *opts, Plan *pl)
{
    if (!shape_ok(N, d, K, dt))
        return KPP_ERR_INVALID_ARG;
    kpp_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts)
        o = *opts;
    kpp_options tuned;
    if (tuned_options(N, d, K, dt, o, &tuned))
        o = tuned; // the autotuner's choice for this shape
    const int sms = device_sms();
    if (sms <= 0)
        return KPP_ERR_CUDA;
    switch (o.form) {
    case KPP_FORM_STREAMED:
        return plan_streamed(N, d, dt, o, sms, pl);
    case KPP_FORM_RECOMPUTE: {
        const kpp_status st = plan_streamed(N, d, dt, o, sms, pl);
        if (st == KPP_OK)
            pl->form = KPP_FORM_RECOMPUTE;
        return st;
    }
    case KPP_FORM_PERSISTENT:
        return plan_persistent(N, d, K, dt, o, sms, pl);
    case KPP_FORM_SMALL:
        return plan_small(N, d, dt, pl);
    case KPP_FORM_AUTO: {
        kpp_status st = plan_small(N, d, dt, pl);
        if (st == KPP_OK || st == KPP_ERR_CUDA)
            return st;
        st = plan_persistent(N, d, K, dt, o, sms, pl);
        if (st == KPP_OK || st == KPP_ERR_INVALID_ARG || st == KPP_ERR_CUDA)
            return st;
        return plan_streamed(N, d, dt, o, sms, pl);
    }
    default:
        return KPP_ERR_UNSUPPORTED;
    }
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

kpp_status run_persistent(const Plan &pl, const Problem &p, cudaStream_t stream)
{
    // the control block and both slot buffers start at zero: a zeroed slot
    // never carries the tag a pass waits for
    if (cudaMemsetAsync(p.ctl, 0, pl.ws_bytes, stream) != cudaSuccess)
        return KPP_ERR_CUDA;
    return persistent_launch(pl.pfn, pl.grid, pl.psmem, p, pl.pargs, stream) == cudaSuccess
               ? KPP_OK
               : KPP_ERR_LAUNCH;
}

// The small kernel clears its own status word: one launch per seeding.
kpp_status run_small(const Plan &pl, const Problem &p, cudaStream_t stream)
{
    return small_launch(pl.pfn, pl.psmem, p, stream) == cudaSuccess ? KPP_OK : KPP_ERR_LAUNCH;
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
    case KPP_ERR_CAPACITY:
        return "more k-means|| candidates than the room given";
    case KPP_ERR_BOUNDS:
        return "debug build: a kernel index was out of bounds (access skipped)";
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

kpp_status kpp_describe(int64_t N, int32_t d, int32_t K, kpp_dtype dtype,
                        const kpp_options *opts, kpp_plan *plan)
{
    if (!plan)
        return KPP_ERR_INVALID_ARG;
    Plan pl;
    std::memset(&pl, 0, sizeof(pl));
    kpp_status st = make_plan(N, d, K, (int)dtype, opts, &pl);
    if (st != KPP_OK)
        return st;
    std::memset(plan, 0, sizeof(*plan));
    plan->form = pl.form;
    plan->grid = pl.grid;
    plan->rows_per_cta = pl.chunk;
    plan->rows_per_segment = (pl.chunk + pl.nseg - 1) / pl.nseg;
    plan->workspace_bytes = (int64_t)pl.ws_bytes;
    if (pl.form == KPP_FORM_SMALL) {
        plan->threads = small_threads();
        plan->launches = 1;
        plan->d2_in_smem = 1;
        plan->cached_rows_per_cta = N;
        plan->smem_bytes = (int64_t)pl.psmem;
    } else if (pl.form == KPP_FORM_PERSISTENT) {
        plan->threads = persistent_threads();
        plan->launches = 1;
        plan->lanes_per_row = pl.pk.lanes;
        plan->d2_in_smem = pl.pfn == pl.pk.fn_smem ? 1 : 0;
        plan->cached_rows_per_cta = pl.pargs.cache_supers * pl.nseg * pl.sw;
        plan->smem_bytes = (int64_t)pl.psmem;
    } else {
        plan->threads = streamed_threads();
        plan->launches = K;
        plan->lanes_per_row = pl.sk.lanes;
        plan->smem_bytes = (int64_t)streamed_smem(pl.sk, d);
    }
    return KPP_OK;
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
    p.nseg = pl.nseg;
    p.sw = pl.sw;
    char *ws = reinterpret_cast<char *>(workspace);
    p.ctl = reinterpret_cast<Control *>(ws);
    if (pl.form == KPP_FORM_PERSISTENT) {
        p.slots = reinterpret_cast<unsigned long long *>(ws + pl.off_slots);
        p.mail = &p.ctl->mail;
    } else {
        p.block_sums = reinterpret_cast<float2 *>(ws + pl.off_bsum);
        p.seg_sums = reinterpret_cast<float2 *>(ws + pl.off_seg);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p.recompute = pl.form == KPP_FORM_RECOMPUTE ? 1 : 0;
    p.exact_draws = (opts && opts->exact_draws) ? 1 : 0;
    if (pl.form == KPP_FORM_PERSISTENT)
        return run_persistent(pl, p, s);
    if (pl.form == KPP_FORM_SMALL)
        return run_small(pl, p, s);
    const int use_graph = opts ? opts->use_graph : 0;
    return run_streamed(pl, p, s, use_graph);
}

// ---------------------------------------------------------------------------
// Point-sharded seeding (one contiguous row range of a problem per process).
// ---------------------------------------------------------------------------
static bool shard_ok(const kpp_shard *s)
{
    return s && s->points && aligned(s->points, 16) && s->indices_out && s->d2_out &&
           s->n_local >= 1 && s->row0 >= 0 && s->n_global < (int64_t(1) << 31) &&
           s->row0 + s->n_local <= s->n_global && s->d >= 1 && s->d <= kMaxDim && s->K >= 1 &&
           s->K <= s->n_global && s->dtype >= KPP_F32 && s->dtype <= KPP_FP8_E4M3 &&
           s->world >= 1 && s->world <= kStage && s->rank >= 0 && s->rank < s->world &&
           ((s->dtype == KPP_FP8_E4M3) == (s->row_scales != nullptr));
}

// The shard's streamed plan and its Problem record.
static kpp_status shard_problem(const kpp_shard *s, const kpp_options *opts, Plan *pl,
                                Problem *p)
{
    if (!shard_ok(s))
        return KPP_ERR_INVALID_ARG;
    kpp_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts)
        o = *opts;
    const int sms = device_sms();
    if (sms <= 0)
        return KPP_ERR_CUDA;
    const kpp_status st = plan_streamed(s->n_local, s->d, s->dtype, o, sms, pl);
    if (st != KPP_OK)
        return st;
    if (!s->workspace || !aligned(s->workspace, kAlign) || s->workspace_bytes < pl->ws_bytes)
        return KPP_ERR_WORKSPACE;
    std::memset(p, 0, sizeof(*p));
    p->points = s->points;
    p->scales = s->row_scales;
    p->N = s->n_local;
    p->d = s->d;
    p->K = s->K;
    p->seed = s->seed;
    p->stream_id = s->stream_id;
    p->nblocks = pl->nblocks;
    p->chunk = pl->chunk;
    p->nseg = pl->nseg;
    p->sw = pl->sw;
    p->idx = s->indices_out;
    p->d2 = s->d2_out;
    char *ws = reinterpret_cast<char *>(s->workspace);
    p->ctl = reinterpret_cast<Control *>(ws);
    p->block_sums = reinterpret_cast<float2 *>(ws + pl->off_bsum);
    p->seg_sums = reinterpret_cast<float2 *>(ws + pl->off_seg);
    p->n_global = s->n_global;
    p->exact_draws = (opts && opts->exact_draws) ? 1 : 0;
    return KPP_OK;
}

int64_t kpp_shard_exchange_words(int32_t d, kpp_dtype dtype)
{
    if (d < 1 || d > kMaxDim || (int)dtype < KPP_F32 || (int)dtype > KPP_FP8_E4M3)
        return 0;
    return xchg_words(d, elem_bytes((int)dtype));
}

size_t kpp_shard_workspace_size(const kpp_shard *s, const kpp_options *opts)
{
    Plan pl;
    kpp_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts)
        o = *opts;
    const int sms = device_sms();
    if (!shard_ok(s) || sms <= 0 || plan_streamed(s->n_local, s->d, s->dtype, o, sms, &pl) != KPP_OK)
        return 0;
    return pl.ws_bytes;
}

kpp_status kpp_shard_first(const kpp_shard *s, int64_t *exchange, kpp_stream_t stream)
{
    Plan pl;
    Problem p;
    const kpp_status st = shard_problem(s, nullptr, &pl, &p);
    if (st != KPP_OK)
        return st;
    if (!exchange || !aligned(exchange, 16))
        return KPP_ERR_INVALID_ARG;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(p.ctl, 0, sizeof(Control), cs) != cudaSuccess)
        return KPP_ERR_CUDA;
    return shard_first_launch(p, s->row0, reinterpret_cast<long long *>(exchange),
                              elem_bytes(s->dtype), cs) == cudaSuccess
               ? KPP_OK
               : KPP_ERR_LAUNCH;
}

kpp_status kpp_shard_pass(const kpp_shard *s, int32_t m, const int64_t *exchange,
                          float *total_out, kpp_stream_t stream, const kpp_options *opts)
{
    Plan pl;
    Problem p;
    const kpp_status st = shard_problem(s, opts, &pl, &p);
    if (st != KPP_OK)
        return st;
    if (!exchange || !aligned(exchange, 16) || !total_out || m < 0 || m >= s->K)
        return KPP_ERR_INVALID_ARG;
    p.xchg = reinterpret_cast<const long long *>(exchange);
    p.shard_total = total_out;
    return streamed_launch(pl.sk, pl.grid, p, m, reinterpret_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? KPP_OK
               : KPP_ERR_LAUNCH;
}

kpp_status kpp_shard_pick(const kpp_shard *s, int32_t m, const float *all_totals,
                          int64_t *exchange, kpp_stream_t stream, const kpp_options *opts)
{
    Plan pl;
    Problem p;
    const kpp_status st = shard_problem(s, opts, &pl, &p);
    if (st != KPP_OK)
        return st;
    if (!exchange || !aligned(exchange, 16) || !all_totals || m < 0 || m >= s->K - 1)
        return KPP_ERR_INVALID_ARG;
    return shard_pick_launch(p, m, s->rank, s->world, all_totals, s->row0,
                             reinterpret_cast<long long *>(exchange), elem_bytes(s->dtype),
                             reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? KPP_OK
               : KPP_ERR_LAUNCH;
}

kpp_status kpp_shard_phi(const float *all_totals, int32_t world, double *phi_out,
                         kpp_stream_t stream)
{
    if (!all_totals || !phi_out || world < 1 || world > kStage)
        return KPP_ERR_INVALID_ARG;
    return shard_phi_launch(all_totals, world, phi_out, reinterpret_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? KPP_OK
               : KPP_ERR_LAUNCH;
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

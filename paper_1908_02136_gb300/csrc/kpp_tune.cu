// kpp_tune.cu -- the autotuner: chooses the form (small, persistent or streamed),
// the lanes per row (points per warp iteration), the row block per CTA and
// the shared-memory cache by timing the candidates on the caller's own data,
// and records the winner for the automatic choice of later calls with the
// same shape.  Host code only; every timed run is an ordinary kpp_seed call.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kpp.h"
#include "kpp_internal.h"

namespace kpp {
namespace {

struct TuneKey {
    int dev, dt, d;
    int64_t N;
    int32_t K;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(dev, dt, d, N, K) < std::tie(o.dev, o.dt, o.d, o.N, o.K);
    }
};

std::mutex g_tune_mutex;
std::map<TuneKey, kpp_options> g_tuned;

// ---------------------------------------------------------------------------
// Optional cache file (environment variable KPP_TUNE_CACHE = a path): every
// winner is appended as one text line keyed by the GPU model (name and SM
// count), dtype, d, N and K, and a process reads the lines of its GPU model
// once, at its first automatic choice on a device, so that later processes
// skip the tuning.  Later lines win over earlier ones for the same shape.
// ---------------------------------------------------------------------------
bool g_cache_read[64] = {};

std::string device_model(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return std::string();
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ' || c == '\t')
            c = '_';
    return name + "/" + std::to_string(prop.multiProcessorCount);
}

// Appends one winner to the cache file (if the environment names one).
void cache_append(int dev, int dt, int d, int64_t N, int32_t K, const kpp_options &o)
{
    const char *path = std::getenv("KPP_TUNE_CACHE");
    if (!path || !*path)
        return;
    const std::string model = device_model(dev);
    if (model.empty())
        return;
    FILE *f = std::fopen(path, "a");
    if (!f)
        return;
    std::fprintf(f, "kpp-tune 1 %s %d %d %lld %d %d %d %d %d %d %d %d\n", model.c_str(), dt, d,
                 (long long)N, K, o.form, o.lanes_per_row, o.ctas_per_sm, o.smem_cache,
                 o.alternate, o.l2_policy, o.min_rows_per_cta);
    std::fclose(f);
}

// Reads the cache file's lines for this device's model into g_tuned (once
// per device and process; the caller holds g_tune_mutex).
void cache_load(int dev)
{
    if (dev < 0 || dev >= 64 || g_cache_read[dev])
        return;
    g_cache_read[dev] = true;
    const char *path = std::getenv("KPP_TUNE_CACHE");
    if (!path || !*path)
        return;
    const std::string model = device_model(dev);
    FILE *f = std::fopen(path, "r");
    if (!f || model.empty()) {
        if (f)
            std::fclose(f);
        return;
    }
    char line[512], m[256];
    while (std::fgets(line, sizeof(line), f)) {
        int ver = 0, dt = 0, d = 0, K = 0;
        long long N = 0;
        kpp_options o;
        std::memset(&o, 0, sizeof(o));
        if (std::sscanf(line, "kpp-tune %d %255s %d %d %lld %d %d %d %d %d %d %d %d", &ver, m, &dt,
                        &d, &N, &K, &o.form, &o.lanes_per_row, &o.ctas_per_sm, &o.smem_cache,
                        &o.alternate, &o.l2_policy, &o.min_rows_per_cta) != 13 ||
            ver != 1 || model != m)
            continue;
        g_tuned[TuneKey{dev, dt, d, (int64_t)N, (int32_t)K}] = o;
    }
    std::fclose(f);
}

// The knobs the tuner sets are all zero: the caller asked for the automatic
// choice.
bool knobs_default(const kpp_options &o)
{
    return o.form == KPP_FORM_AUTO && o.lanes_per_row == 0 && o.ctas_per_sm == 0 &&
           o.smem_cache == 0 && o.alternate == 0 && o.l2_policy == 0 && o.min_rows_per_cta == 0;
}

kpp_options make_opts(int form, int lanes, int ctas_per_sm, int smem_cache, int min_rows)
{
    kpp_options o;
    std::memset(&o, 0, sizeof(o));
    o.form = form;
    o.lanes_per_row = lanes;
    o.ctas_per_sm = ctas_per_sm;
    o.smem_cache = smem_cache;
    o.min_rows_per_cta = min_rows;
    return o;
}

// The candidate grid: the small form (where the problem fits one SM), every
// built lanes-per-row specialisation of the two other forms; for the persistent form with and without the shared-memory point cache and
// three smallest row blocks per CTA, for the streamed form three grid sizes.
std::vector<kpp_options> candidates()
{
    static const int kLanes[] = {0, 1, 2, 4, 8, 16, 32};
    std::vector<kpp_options> c;
    c.push_back(make_opts(KPP_FORM_SMALL, 0, 0, 0, 0));
    for (int lanes : kLanes) {
        for (int cache : {0, -1})
            for (int min_rows : {0, 512, 8192})
                c.push_back(make_opts(KPP_FORM_PERSISTENT, lanes, 0, cache, min_rows));
        for (int cps : {0, 2, 8})
            c.push_back(make_opts(KPP_FORM_STREAMED, lanes, cps, 0, 0));
    }
    return c;
}

// What distinguishes two candidates' launches (equal plans run the same code).
std::tuple<int, int, int, int, int64_t, int64_t, int, int> signature(const kpp_plan &p,
                                                                   const kpp_options &o)
{
    return std::make_tuple(p.form, p.grid, p.lanes_per_row, p.d2_in_smem, p.rows_per_cta,
                           p.cached_rows_per_cta, o.l2_policy, o.alternate);
}

} // namespace

bool tuned_options(int64_t N, int32_t d, int32_t K, int dt, const kpp_options &asked,
                   kpp_options *out)
{
    if (!knobs_default(asked))
        return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return false;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    cache_load(dev);
    auto it = g_tuned.find(TuneKey{dev, dt, d, N, K});
    if (it == g_tuned.end())
        return false;
    *out = it->second;
    out->timeout_us = asked.timeout_us; // the caller's bound and graph choice stand
    out->use_graph = asked.use_graph;
    out->exact_draws = asked.exact_draws;
    return true;
}

} // namespace kpp

using namespace kpp;

extern "C" {

size_t kpp_tune_workspace_size(int64_t N, int32_t d, int32_t K, kpp_dtype dtype)
{
    size_t most = 0;
    for (const kpp_options &o : candidates()) {
        kpp_options v = o;
        for (int l2 : {0, -1, 2}) {
            v.l2_policy = l2;
            most = std::max(most, kpp_workspace_size(N, d, K, dtype, &v));
        }
    }
    return most;
}

void kpp_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned.clear();
    for (bool &r : g_cache_read)
        r = true; // what the cache file held is forgotten too, not read again
}

kpp_status kpp_tune(const void *points, const float *row_scales, int64_t N, int32_t d, int32_t K,
                    kpp_dtype dtype, int64_t *indices_out, float *d2_out, void *workspace,
                    size_t workspace_bytes, kpp_stream_t stream, int32_t passes,
                    kpp_options *best_out, float *best_ms_per_pass)
{
    if (!best_out || passes < 0)
        return KPP_ERR_INVALID_ARG;
    const int32_t Kt = std::min<int32_t>(K, passes > 0 ? passes : 32);
    if (Kt < 1)
        return KPP_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0)
            cudaEventDestroy(e0);
        return KPP_ERR_CUDA;
    }
    kpp_status result = KPP_OK;
    float best_ms = -1.f;
    kpp_options best;
    std::memset(&best, 0, sizeof(best));
    std::vector<std::tuple<int, int, int, int, int64_t, int64_t, int, int>> seen;

    // one candidate: a warm-up run (it also captures a streamed graph), then
    // two timed runs; ms per pass, or < 0 if the candidate does not apply
    auto trial = [&](const kpp_options &o, float *ms) -> kpp_status {
        *ms = -1.f;
        kpp_plan plan;
        if (kpp_describe(N, d, Kt, dtype, &o, &plan) != KPP_OK ||
            (size_t)plan.workspace_bytes > workspace_bytes)
            return KPP_OK;
        const auto sig = signature(plan, o);
        if (std::find(seen.begin(), seen.end(), sig) != seen.end())
            return KPP_OK;
        seen.push_back(sig);
        kpp_status st = kpp_seed(points, row_scales, N, d, Kt, dtype, 1, 0, nullptr, 0,
                                 indices_out, d2_out, nullptr, workspace, workspace_bytes, stream,
                                 &o);
        if (st != KPP_OK)
            return st == KPP_ERR_INVALID_ARG || st == KPP_ERR_WORKSPACE ? st : KPP_OK;
        st = kpp_read_status(workspace, stream);
        if (st == KPP_ERR_DEGENERATE || st == KPP_ERR_CUDA)
            return st; // the data or the device, not the candidate
        if (st != KPP_OK)
            return KPP_OK; // e.g. a bounded wait gave up: not a candidate
        constexpr int kRuns = 2;
        if (cudaEventRecord(e0, s) != cudaSuccess)
            return KPP_ERR_CUDA;
        for (int r = 0; r < kRuns; ++r) {
            st = kpp_seed(points, row_scales, N, d, Kt, dtype, 1, 0, nullptr, 0, indices_out,
                          d2_out, nullptr, workspace, workspace_bytes, stream, &o);
            if (st != KPP_OK)
                return KPP_OK;
        }
        float t = 0.f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return KPP_ERR_CUDA;
        if (kpp_read_status(workspace, stream) != KPP_OK)
            return KPP_OK;
        *ms = t / (kRuns * Kt);
        return KPP_OK;
    };
    auto consider = [&](const kpp_options &o) -> kpp_status {
        float ms;
        const kpp_status st = trial(o, &ms);
        // a later candidate must win by more than 1 %: timing noise alone
        // does not move the choice away from the earlier (default) ones
        if (st == KPP_OK && ms > 0.f && (best_ms < 0.f || ms < 0.99f * best_ms)) {
            best_ms = ms;
            best = o;
        }
        return st;
    };

    for (const kpp_options &o : candidates()) {
        result = consider(o);
        if (result != KPP_OK)
            break;
    }
    // refine the persistent winner's traversal and L2 policy
    if (result == KPP_OK && best_ms > 0.f && best.form == KPP_FORM_PERSISTENT) {
        const kpp_options base = best;
        for (int l2 : {-1, 2}) {
            kpp_options v = base;
            v.l2_policy = l2;
            if ((result = consider(v)) != KPP_OK)
                break;
        }
        if (result == KPP_OK) {
            kpp_options v = best;
            v.alternate = -1;
            result = consider(v);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != KPP_OK)
        return result;
    if (best_ms < 0.f)
        return KPP_ERR_UNSUPPORTED; // no candidate ran (workspace too small?)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return KPP_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[TuneKey{dev, (int)dtype, d, N, K}] = best;
        cache_append(dev, (int)dtype, d, N, K, best);
    }
    *best_out = best;
    if (best_ms_per_pass)
        *best_ms_per_pass = best_ms;
    return KPP_OK;
}

} // extern "C"

// kpp_batched.cu -- host side of the batching form: problems grouped into
// waves by d; per wave, team sizes from cost, the static list schedule of
// the team jobs (longest first, each on the CTAs free earliest) and the queue
// of single-CTA jobs; the workspace and the launches.  Kernel in
// kpp_batched.cuh.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kpp_batched.cuh"

namespace kpp {

namespace {

BatchFn batched_fn(int dt, int d)
{
    switch (dt) {
    case KPP_F32:
        return batched_kernel_f32(d);
    case KPP_BF16:
        return batched_kernel_bf16(d);
    default:
        return batched_kernel_fp8(d);
    }
}

template <int DT>
int batch_sw_of(int d)
{
    switch (d) {
    case 2:
        return BatchGeom<DT, 2>::SW;
    case 4:
        return BatchGeom<DT, 4>::SW;
    case 8:
        return BatchGeom<DT, 8>::SW;
    case 16:
        return BatchGeom<DT, 16>::SW;
    case 32:
        return BatchGeom<DT, 32>::SW;
    case 64:
        return BatchGeom<DT, 64>::SW;
    case 128:
        return BatchGeom<DT, 128>::SW;
    default:
        return 0; // no batched specialisation for this d
    }
}

// rows per super-iteration of the batched specialisation, 0 if none
int batch_rows_per_super(int dt, int d)
{
    if (dt == KPP_F32)
        return batch_sw_of<KPP_F32>(d);
    if (dt == KPP_BF16)
        return batch_sw_of<KPP_BF16>(d);
    return batch_sw_of<KPP_FP8_E4M3>(d);
}

constexpr size_t kAlign = 256;
size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The problems of one d and their schedule on the grid.
struct Wave {
    int d;
    BatchFn fn;
    std::vector<std::vector<BatchEntry>> lists; // team jobs per CTA, in schedule order
    std::vector<int32_t> queue;                  // single-CTA jobs, longest first
    size_t nentries;
    size_t off_entries, off_first, off_queue, off_counter; // workspace offsets
};

struct BatchPlan {
    int grid;
    std::vector<int> team;    // team size of each problem (by problem index)
    std::vector<int> nblocks; // CTAs that own rows (<= team)
    std::vector<int64_t> chunk;
    std::vector<Wave> waves; // launched in this order
    // workspace layout
    size_t off_jobs, off_ctls, off_slots, bytes;
    std::vector<size_t> slot_off; // per problem, relative to off_slots
};

int elem_bytes(int dt) { return dt == KPP_F32 ? 4 : dt == KPP_BF16 ? 2 : 1; }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

kpp_status check_problems(const kpp_problem *pr, int32_t n, int dt)
{
    if (!pr || n < 1 || dt < KPP_F32 || dt > KPP_FP8_E4M3)
        return KPP_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const kpp_problem &q = pr[i];
        if (!q.points || !aligned16(q.points) || !q.indices_out || !q.d2_out || q.N < 1 ||
            q.N >= (int64_t(1) << 31) || q.K < 1 || q.K > q.N)
            return KPP_ERR_INVALID_ARG;
        if ((dt == KPP_FP8_E4M3) != (q.row_scales != nullptr))
            return KPP_ERR_INVALID_ARG;
        if (batch_rows_per_super(dt, q.d) == 0)
            return KPP_ERR_UNSUPPORTED;
    }
    return KPP_OK;
}

kpp_status make_batch_plan(const kpp_problem *pr, int32_t n, int dt, const kpp_options *opts,
                           BatchPlan *bp)
{
    kpp_status st = check_problems(pr, n, dt);
    if (st != KPP_OK)
        return st;
    int dev = 0, sms = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (!coop)
        return KPP_ERR_UNSUPPORTED;
    const int grid = sms; // one CTA per SM
    const int64_t min_rows = (opts && opts->min_rows_per_cta > 0) ? opts->min_rows_per_cta : 2048;
    const double eb = elem_bytes(dt);
    // Cost model, in bytes-equivalents: the points read per pass, D^2 read and
    // written per pass, and a fixed per-pass cost of the exchange.
    auto cost_of = [&](int i, int t) {
        const double rows = (double)pr[i].N / t;
        return (double)pr[i].K * (rows * (pr[i].d * eb + 8.0) + (t > 1 ? 256.0e3 : 64.0e3));
    };
    std::vector<double> c1(n);
    for (int i = 0; i < n; ++i)
        c1[i] = cost_of(i, 1);
    bp->grid = grid;
    bp->team.assign(n, 1);
    bp->nblocks.assign(n, 1);
    bp->chunk.assign(n, 0);
    bp->waves.clear();
    static const int kDims[] = {2, 4, 8, 16, 32, 64, 128};
    std::vector<int> order;
    std::vector<double> avail(grid);
    std::vector<int> cta(grid);
    for (int d : kDims) {
        order.clear();
        double total = 0;
        for (int i = 0; i < n; ++i)
            if (pr[i].d == d) {
                order.push_back(i);
                total += c1[i];
            }
        if (order.empty())
            continue;
        Wave w;
        w.d = d;
        w.fn = batched_fn(dt, d);
        int resident = 0;
        if (!w.fn ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, (const void *)w.fn,
                                                          kPersistThreads, 0) != cudaSuccess)
            return KPP_ERR_CUDA;
        if (resident < 1)
            return KPP_ERR_UNSUPPORTED;
        const double share = total / grid;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return c1[x] > c1[y]; });
        w.lists.assign(grid, {});
        // list scheduling: each team problem, longest first, takes the t CTAs
        // that are free earliest; all of them start it when the last of them
        // is free
        std::fill(avail.begin(), avail.end(), 0.0);
        for (int i : order) {
            int t = (int)std::ceil(c1[i] / share);
            const int64_t tmax = (pr[i].N + min_rows - 1) / min_rows;
            if (t > tmax)
                t = (int)tmax;
            if (t < 1)
                t = 1;
            if (t > grid)
                t = grid;
            const int64_t sw = batch_rows_per_super(dt, d);
            int64_t chunk = (pr[i].N + t - 1) / t;
            chunk = (chunk + sw - 1) / sw * sw;
            const int nb = (int)((pr[i].N + chunk - 1) / chunk);
            bp->team[i] = t;
            bp->nblocks[i] = nb;
            bp->chunk[i] = chunk;
            if (nb == 1) { // served by the queue
                w.queue.push_back(i);
                continue;
            }
            for (int c = 0; c < grid; ++c)
                cta[c] = c;
            std::partial_sort(cta.begin(), cta.begin() + nb, cta.end(), [&](int x, int y) {
                return avail[x] < avail[y] || (avail[x] == avail[y] && x < y);
            });
            double start = 0;
            for (int r = 0; r < nb; ++r)
                start = std::max(start, avail[cta[r]]);
            const double fin = start + cost_of(i, nb);
            for (int r = 0; r < nb; ++r) {
                avail[cta[r]] = fin;
                w.lists[cta[r]].push_back(BatchEntry{i, r});
            }
        }
        w.nentries = 0;
        for (auto &l : w.lists)
            w.nentries += l.size();
        bp->waves.push_back(std::move(w));
    }
    // workspace: batch control | job table | job control blocks |
    //            per wave: entries, list offsets, queue, queue counter |
    //            every problem's slots
    size_t off = sizeof(Control);
    bp->off_jobs = off;
    off += round_up(sizeof(BatchJob) * (size_t)n, kAlign);
    bp->off_ctls = off;
    off += round_up(sizeof(Control) * (size_t)n, kAlign);
    for (Wave &w : bp->waves) {
        w.off_entries = off;
        off += round_up(sizeof(BatchEntry) * w.nentries, kAlign);
        w.off_first = off;
        off += round_up(sizeof(int32_t) * (size_t)(grid + 1), kAlign);
        w.off_queue = off;
        off += round_up(sizeof(int32_t) * (w.queue.size() + 1), kAlign);
        w.off_counter = off;
        off += kAlign;
    }
    bp->off_slots = off;
    bp->slot_off.assign(n, 0);
    size_t soff = 0;
    for (int i = 0; i < n; ++i) {
        bp->slot_off[i] = soff;
        soff += round_up(8 * 2 * kSlotWords * (size_t)bp->nblocks[i], 64);
    }
    off += round_up(soff, kAlign);
    bp->bytes = off;
    return KPP_OK;
}

} // namespace
} // namespace kpp

using namespace kpp;

extern "C" {

size_t kpp_batch_workspace_size(const kpp_problem *problems, int32_t n, kpp_dtype dtype,
                                const kpp_options *opts)
{
    BatchPlan bp;
    if (make_batch_plan(problems, n, (int)dtype, opts, &bp) != KPP_OK)
        return 0;
    return bp.bytes;
}

kpp_status kpp_seed_batched(const kpp_problem *problems, int32_t n, kpp_dtype dtype,
                            void *workspace, size_t workspace_bytes, kpp_stream_t stream,
                            const kpp_options *opts)
{
    const int dt = (int)dtype;
    BatchPlan bp;
    kpp_status st = make_batch_plan(problems, n, dt, opts, &bp);
    if (st != KPP_OK)
        return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 ||
        workspace_bytes < bp.bytes)
        return KPP_ERR_WORKSPACE;
    char *ws = reinterpret_cast<char *>(workspace);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // host image of the job table and the work lists
    std::vector<BatchJob> jobs(n);
    Control *ctls = reinterpret_cast<Control *>(ws + bp.off_ctls);
    for (int i = 0; i < n; ++i) {
        const kpp_problem &q = problems[i];
        BatchJob &b = jobs[i];
        std::memset(&b, 0, sizeof(b));
        Problem &p = b.p;
        p.points = q.points;
        p.scales = q.row_scales;
        p.N = q.N;
        p.d = q.d;
        p.K = q.K;
        p.seed = q.seed;
        p.stream_id = q.stream_id;
        p.idx = q.indices_out;
        p.d2 = q.d2_out;
        p.phi = q.phi_out;
        p.ctl = ctls + i;
        p.mail = &p.ctl->mail;
        p.nseg = kPersistWarps;
        p.sw = batch_rows_per_super(dt, q.d);
        p.chunk = bp.chunk[i];
        p.nblocks = bp.nblocks[i];
        p.slots = reinterpret_cast<unsigned long long *>(ws + bp.off_slots + bp.slot_off[i]);
        p.exact_draws = (opts && opts->exact_draws) ? 1 : 0;
        b.d = q.d;
    }
    if (cudaMemsetAsync(ws, 0, bp.bytes, s) != cudaSuccess ||
        cudaMemcpyAsync(ws + bp.off_jobs, jobs.data(), sizeof(BatchJob) * (size_t)n,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    // the lists and queues of every wave, in one staging image
    const size_t lo = bp.waves.empty() ? bp.off_slots : bp.waves.front().off_entries;
    std::vector<char> image(bp.off_slots - lo, 0);
    for (const Wave &w : bp.waves) {
        BatchEntry *ent = reinterpret_cast<BatchEntry *>(image.data() + (w.off_entries - lo));
        int32_t *first = reinterpret_cast<int32_t *>(image.data() + (w.off_first - lo));
        int32_t k = 0;
        for (int c = 0; c < bp.grid; ++c) {
            first[c] = k;
            for (const BatchEntry &e : w.lists[c])
                ent[k++] = e;
        }
        first[bp.grid] = k;
        if (!w.queue.empty())
            std::memcpy(image.data() + (w.off_queue - lo), w.queue.data(),
                        sizeof(int32_t) * w.queue.size());
    }
    // (a copy from pageable memory has read its source when it returns)
    if (!image.empty() && cudaMemcpyAsync(ws + lo, image.data(), image.size(),
                                          cudaMemcpyHostToDevice, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    PersistArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.cache_supers = 0;
    pa.reverse = (opts && opts->alternate < 0) ? 0 : 1;
    pa.l2_hint = (opts && opts->l2_policy == -1) ? 0 : ((opts && opts->l2_policy == 2) ? 2 : 1);
    pa.timeout_ns = 1000ull * ((opts && opts->timeout_us) ? opts->timeout_us : 2000000u);
    for (const Wave &w : bp.waves) {
        BatchArgs a;
        std::memset(&a, 0, sizeof(a));
        a.jobs = reinterpret_cast<const BatchJob *>(ws + bp.off_jobs);
        a.entries = reinterpret_cast<const BatchEntry *>(ws + w.off_entries);
        a.first = reinterpret_cast<const int32_t *>(ws + w.off_first);
        a.queue_jobs = reinterpret_cast<const int32_t *>(ws + w.off_queue);
        a.nqueue = (int32_t)w.queue.size();
        a.queue = reinterpret_cast<unsigned int *>(ws + w.off_counter);
        a.ctl = reinterpret_cast<Control *>(ws);
        a.pa = pa;
        void *args[] = {&a};
        if (cudaLaunchCooperativeKernel((const void *)w.fn, dim3(bp.grid), dim3(kPersistThreads),
                                        args, 0, s) != cudaSuccess)
            return KPP_ERR_LAUNCH;
    }
    return KPP_OK;
}

} // extern "C"

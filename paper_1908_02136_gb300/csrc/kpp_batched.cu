// kpp_batched.cu -- host side of the batching form: the schedule (teams for
// the costly problems, an LPT queue for the rest), the workspace and the
// launch.  Kernel in kpp_batched.cuh.
//
// The host sorts the problems by cost (K * N * d * bytes) and splits them in
// two classes.  A problem costing more than one SM's fair share of the whole
// batch gets a team of CTAs sized in proportion to its cost; the team runs it
// exactly like the persistent form (seed_blocks: per-warp segments, tagged
// block-sum slots and mailbox local to the team).  Every other problem is
// seeded by a single CTA: CTAs outside the teams -- and team members once
// their team's problem is done -- take the next problem from an atomic queue
// in decreasing order of cost (longest processing time first).  D^2 stays in
// each problem's output array; every problem has its own control block, so
// one problem's degenerate data does not stop the others.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kpp_batched.cuh"

namespace kpp {

namespace {

BatchFn batched_fn(int dt)
{
    switch (dt) {
    case KPP_F32:
        return batched_kernel_f32();
    case KPP_BF16:
        return batched_kernel_bf16();
    default:
        return batched_kernel_fp8();
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

struct BatchPlan {
    int grid;
    std::vector<int> order;     // problem index of job j
    std::vector<int> team_size; // for big jobs
    std::vector<int> team_first;
    int nbig;
    // workspace layout
    size_t off_jobs, off_ctls, off_cta_job, off_team_slots, off_solo_slots, bytes;
    std::vector<size_t> team_slot_off; // per big job, relative to off_team_slots
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
    int resident = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, (const void *)batched_fn(dt),
                                                      kPersistThreads, 0) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (resident < 1)
        return KPP_ERR_UNSUPPORTED;
    const int grid = sms; // one CTA per SM
    const int64_t min_rows = (opts && opts->min_rows_per_cta > 0) ? opts->min_rows_per_cta : 2048;
    const double eb = elem_bytes(dt);
    // cost in bytes read, plus a per-pass cost for the exchange of a team
    std::vector<double> cost(n);
    double total = 0;
    for (int i = 0; i < n; ++i) {
        cost[i] = (double)pr[i].K * ((double)pr[i].N * pr[i].d * eb + 256.0 * 1024.0);
        total += cost[i];
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i)
        idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    const double share = total / grid;
    bp->grid = grid;
    bp->order.clear();
    bp->team_size.clear();
    bp->team_first.clear();
    int used = 0;
    std::vector<int> small;
    for (int i : idx) {
        int t = (int)std::lround(cost[i] / share);
        const int64_t tmax = (pr[i].N + min_rows - 1) / min_rows;
        if (t > tmax)
            t = (int)tmax;
        if (t >= 2 && used + t <= grid) {
            bp->order.push_back(i);
            bp->team_size.push_back(t);
            bp->team_first.push_back(used);
            used += t;
        } else {
            small.push_back(i);
        }
    }
    bp->nbig = (int)bp->order.size();
    for (int i : small)
        bp->order.push_back(i);
    // workspace: batch control | job table | job control blocks | cta_job |
    //            team slots (+ team mailbox word) | solo slots
    size_t off = sizeof(Control);
    bp->off_jobs = off;
    off += round_up(sizeof(BatchJob) * (size_t)n, kAlign);
    bp->off_ctls = off;
    off += round_up(sizeof(Control) * (size_t)n, kAlign);
    bp->off_cta_job = off;
    off += round_up(sizeof(int32_t) * (size_t)grid, kAlign);
    bp->off_team_slots = off;
    bp->team_slot_off.clear();
    size_t toff = 0;
    for (int j = 0; j < bp->nbig; ++j) {
        bp->team_slot_off.push_back(toff);
        toff += round_up(8 * (2 * kSlotWords * (size_t)bp->team_size[j]), kAlign);
    }
    off += toff;
    bp->off_solo_slots = off;
    off += round_up(8 * 2 * kSlotWords * (size_t)grid, kAlign);
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
    // host image of the job table and the CTA map
    std::vector<BatchJob> jobs(n);
    std::vector<int32_t> cta_job(bp.grid, -1);
    Control *ctls = reinterpret_cast<Control *>(ws + bp.off_ctls);
    for (int j = 0; j < n; ++j) {
        const kpp_problem &q = problems[bp.order[j]];
        BatchJob &b = jobs[j];
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
        p.ctl = ctls + j;
        p.nseg = kPersistWarps;
        p.sw = batch_rows_per_super(dt, q.d);
        b.d = q.d;
        const int t = j < bp.nbig ? bp.team_size[j] : 1;
        int64_t chunk = (q.N + t - 1) / t;
        chunk = (chunk + p.sw - 1) / p.sw * p.sw;
        p.chunk = chunk;
        p.nblocks = (int)((q.N + chunk - 1) / chunk);
        p.mail = &p.ctl->mail;
        if (j < bp.nbig) {
            b.team_first = bp.team_first[j];
            p.slots = reinterpret_cast<unsigned long long *>(ws + bp.off_team_slots +
                                                               bp.team_slot_off[j]);
            for (int r = 0; r < p.nblocks; ++r)
                cta_job[b.team_first + r] = j;
        } else {
            b.team_first = -1;
            p.slots = nullptr; // set per CTA on the device
        }
    }
    if (cudaMemsetAsync(ws, 0, bp.bytes, s) != cudaSuccess ||
        cudaMemcpyAsync(ws + bp.off_jobs, jobs.data(), sizeof(BatchJob) * (size_t)n,
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ws + bp.off_cta_job, cta_job.data(), sizeof(int32_t) * (size_t)bp.grid,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.jobs = reinterpret_cast<const BatchJob *>(ws + bp.off_jobs);
    a.njobs = n;
    a.nbig = bp.nbig;
    a.cta_job = reinterpret_cast<const int32_t *>(ws + bp.off_cta_job);
    a.ctl = reinterpret_cast<Control *>(ws);
    a.queue = &a.ctl->ticket;
    a.solo_slots = reinterpret_cast<unsigned long long *>(ws + bp.off_solo_slots);
    a.pa.cache_supers = 0;
    a.pa.reverse = (opts && opts->alternate < 0) ? 0 : 1;
    a.pa.l2_hint = (opts && opts->l2_policy == -1) ? 0 : ((opts && opts->l2_policy == 2) ? 2 : 1);
    a.pa.timeout_ns = 1000ull * ((opts && opts->timeout_us) ? opts->timeout_us : 2000000u);
    void *args[] = {&a};
    if (cudaLaunchCooperativeKernel((const void *)batched_fn(dt), dim3(bp.grid),
                                    dim3(kPersistThreads), args, 0, s) != cudaSuccess)
        return KPP_ERR_LAUNCH;
    return KPP_OK;
}

} // extern "C"

// kpp_batched.cuh -- batching form: many independent seeding problems of
// uneven N, d and K, one cooperative launch (one CTA per SM) per distinct d
// -- a wave -- on the caller's stream.  The kernel; the host-side scheduling
// is in kpp_batched.cu, the instantiations in kpp_batched_{f32,bf16,fp8}.cu.
//
// Each wave's kernel is specialised for its d alone: one kernel body holding
// every d's specialisation would need more registers than a 512-thread CTA
// may have and spill in the streaming loop.
//
// Within a wave the host gives every problem a team size from its cost: one
// CTA for most, several for the costly ones.  Team jobs get a static list
// schedule -- longest first, each on the CTAs that become free earliest --
// and the single-CTA jobs a dynamic queue, longest first, which every CTA
// serves once its list is done.  A team runs its problem exactly like the
// persistent form (seed_blocks: per-warp segments, tagged block-sum slots
// and mailbox local to the problem).  D^2 stays in each problem's output
// array; every problem has its own control block, so one problem's
// degenerate data does not stop the others.
#pragma once

#include "kpp_persistent.cuh"

namespace kpp {


// lanes per row of the batched specialisation of (dtype, d)
template <int DT, int D>
struct BatchGeom {
    static constexpr int VPR = Geom<DT, D, 1>::WIDE ? Geom<DT, D, 1>::VPR : 1;
    static constexpr int L = VPR >= 8 ? 8 : VPR; // lanes per row
    static constexpr int SW = Geom<DT, D, L>::SW;
};

struct BatchJob {
    Problem p; // nblocks, chunk, sw, nseg, slots, mail and ctl set by the host
    int32_t d;
    int32_t pad_;
};

// One entry of a CTA's work list: run job `job` as team member `rank`.
struct BatchEntry {
    int32_t job;
    int32_t rank;
};

// The work of one wave.
struct BatchArgs {
    const BatchJob *jobs;      // every problem of the batch
    const BatchEntry *entries; // every CTA's list of team jobs, back to back
    const int32_t *first;      // [grid + 1]: CTA c's list is entries[first[c], first[c+1])
    const int32_t *queue_jobs; // single-CTA jobs, longest first
    int32_t nqueue;
    unsigned int *queue;       // next entry of queue_jobs (zero at launch)
    Control *ctl;              // batch status (first error of any job)
    PersistArgs pa;
};

// After a job: its rank-0 CTA reports a non-OK status to the batch status.
__device__ __forceinline__ void report(const Problem &p, const BatchArgs &a, int rank)
{
    if (rank == 0 && threadIdx.x == 0) {
        const int32_t st = *(volatile int32_t *)&p.ctl->status;
        if (st != KPP_OK)
            atomicCAS(&a.ctl->status, KPP_OK, st);
    }
}

// Every CTA first runs its list of team jobs in order -- the host orders all
// lists by one global schedule (each team job has a single start time, the
// same in every member's list), so a member only ever waits for CTAs busy
// with earlier jobs and no cycle of waits can form -- then takes single-CTA
// jobs from the queue, longest first, until it is empty.  A batch status of
// TIMEOUT or INVALID_ARG (a wait gave up, or bad input) stops the wave.
template <int DT, int D>
__global__ void __launch_bounds__(kPersistThreads, 1) batched_kernel(BatchArgs a)
{
    __shared__ BlockShared sh;
    __shared__ int job_sh, rank_sh;
    const int list0 = a.first[blockIdx.x];
    const int n_list = a.first[blockIdx.x + 1] - list0;
    for (int e = 0;; ++e) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int32_t st = *(volatile int32_t *)&a.ctl->status;
            int job = -1, rank = 0;
            if (st == KPP_ERR_TIMEOUT || st == KPP_ERR_INVALID_ARG) {
                // stop
            } else if (e < n_list) {
                const BatchEntry en = a.entries[list0 + e];
                job = en.job;
                rank = en.rank;
            } else {
                const int q = (int)atomicAdd(a.queue, 1u);
                if (q < a.nqueue)
                    job = a.queue_jobs[q];
            }
            job_sh = job;
            rank_sh = rank;
        }
        __syncthreads();
        const int j = job_sh, rank = rank_sh;
        if (j < 0)
            break;
        const Problem &p = a.jobs[j].p;
        seed_blocks<DT, D, BatchGeom<DT, D>::L, D2_INPLACE>(p, a.pa, rank, nullptr, sh);
        report(p, a, rank);
    }
}

using BatchFn = void (*)(BatchArgs);

// The wave kernel of (dtype, d), or null when d has no specialisation.
BatchFn batched_kernel_f32(int d);
BatchFn batched_kernel_bf16(int d);
BatchFn batched_kernel_fp8(int d);

template <int DT>
BatchFn batched_kernel_of(int d)
{
    switch (d) {
    case 2:
        return &batched_kernel<DT, 2>;
    case 4:
        return &batched_kernel<DT, 4>;
    case 8:
        return &batched_kernel<DT, 8>;
    case 16:
        return &batched_kernel<DT, 16>;
    case 32:
        return &batched_kernel<DT, 32>;
    case 64:
        return &batched_kernel<DT, 64>;
    case 128:
        return &batched_kernel<DT, 128>;
    default:
        return nullptr;
    }
}

} // namespace kpp

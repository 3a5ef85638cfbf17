// kpp_batched.cuh -- batching form: many independent seeding problems of
// uneven N, d and K in one cooperative launch (one CTA per SM).  The kernel;
// the host-side scheduling is in kpp_batched.cu, the instantiations in
// kpp_batched_{f32,bf16,fp8}.cu.
//
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
    Problem p;          // nblocks, chunk, sw, nseg, slots, mail and ctl set by the host
    int32_t d;
    int32_t team_first; // first CTA of the team, or -1 for a queued problem
};

struct BatchArgs {
    const BatchJob *jobs;
    int32_t njobs;
    int32_t nbig;                   // jobs [0, nbig) have teams; [nbig, njobs) are queued
    const int32_t *cta_job;         // team job of each CTA, or -1
    unsigned int *queue;            // next queued job (offset from nbig)
    Control *ctl;                   // batch status (first error of any job)
    unsigned long long *solo_slots; // [grid][2 * kSlotWords]: a lone CTA's slots
    PersistArgs pa;
};

template <int DT, int D>
__device__ __forceinline__ void run_as(const Problem &p, const PersistArgs &pa, int rank,
                                       BlockShared &sh)
{
    seed_blocks<DT, D, BatchGeom<DT, D>::L, D2_INPLACE>(p, pa, rank, nullptr, sh);
}

template <int DT>
__device__ void run_job(const Problem &p, int d, const PersistArgs &pa, int rank, BlockShared &sh)
{
    switch (d) {
    case 2:
        run_as<DT, 2>(p, pa, rank, sh);
        break;
    case 4:
        run_as<DT, 4>(p, pa, rank, sh);
        break;
    case 8:
        run_as<DT, 8>(p, pa, rank, sh);
        break;
    case 16:
        run_as<DT, 16>(p, pa, rank, sh);
        break;
    case 32:
        run_as<DT, 32>(p, pa, rank, sh);
        break;
    case 64:
        run_as<DT, 64>(p, pa, rank, sh);
        break;
    default:
        run_as<DT, 128>(p, pa, rank, sh);
        break;
    }
}

// After a job: its rank-0 CTA reports a non-OK status to the batch status.
__device__ __forceinline__ void report(const Problem &p, const BatchArgs &a, int rank)
{
    if (rank == 0 && threadIdx.x == 0) {
        const int32_t st = *(volatile int32_t *)&p.ctl->status;
        if (st != KPP_OK)
            atomicCAS(&a.ctl->status, KPP_OK, st);
    }
}

template <int DT>
__global__ void __launch_bounds__(kPersistThreads, 1) batched_kernel(BatchArgs a)
{
    __shared__ BlockShared sh;
    __shared__ int job_sh;
    const int j = a.cta_job[blockIdx.x];
    if (j >= 0) {
        const BatchJob &job = a.jobs[j];
        const int rank = (int)blockIdx.x - job.team_first;
        run_job<DT>(job.p, job.d, a.pa, rank, sh);
        report(job.p, a, rank);
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int32_t st = *(volatile int32_t *)&a.ctl->status;
            job_sh = (st == KPP_ERR_TIMEOUT || st == KPP_ERR_INVALID_ARG)
                         ? -1
                         : a.nbig + (int)atomicAdd(a.queue, 1u);
        }
        __syncthreads();
        const int q = job_sh;
        if (q < 0 || q >= a.njobs)
            break;
        Problem p = a.jobs[q].p;
        p.slots = a.solo_slots + (size_t)blockIdx.x * 2 * kSlotWords;
        run_job<DT>(p, a.jobs[q].d, a.pa, 0, sh);
        report(p, a, 0);
    }
}

using BatchFn = void (*)(BatchArgs);

BatchFn batched_kernel_f32();
BatchFn batched_kernel_bf16();
BatchFn batched_kernel_fp8();

} // namespace kpp

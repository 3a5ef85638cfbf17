// kpp_persistent.cuh -- persistent form: one cooperative launch runs all K
// passes of Algorithm 1's loop over seeds.
//
// Every CTA owns one contiguous block of rows for the whole seeding and walks
// it with one contiguous segment per warp.  D^2 of the block lives in shared
// memory when it fits (D2_SMEM; copied to the output in the last pass), else
// in the output array itself (D2_INPLACE).  The first `cache_supers`
// super-iterations of every warp's segment are copied into shared memory in
// pass 0 and read from there afterwards; the rest are streamed from HBM/L2
// each pass, in alternating directions and with an L2 evict-last policy so
// that what the previous pass left in L2 is read first.
//
// Between passes there is no counter barrier.  Each CTA publishes its block
// sum as one tagged 64-bit word; waiting for all nblocks words of the pass is
// the grid-wide synchronisation and stages the draw's first level in the same
// round trip.  Every CTA then finds the block holding t = u * T (the same
// pair arithmetic on the same words gives the same answer everywhere); only
// that block's CTA, the owner, resolves the segment and the point from its
// own shared memory and publishes the index in a tagged mailbox word, which
// the other CTAs wait for.  Words carry their pass tag, so no fence orders
// them, and slots alternate between two buffers by pass parity (no CTA can be
// more than one pass ahead of another).  Every wait is bounded.
#pragma once

#include "kpp_internal.h"
#include "kpp_pass.cuh"

namespace kpp {

constexpr int kPersistThreads = 512;
constexpr int kPersistWarps = kPersistThreads / 32;
constexpr int kMaxBlocks = 640;    // grid limit of the persistent form
constexpr int kMaxChunks = 1024;   // 32-row chunks per block searched directly

struct DrawShared {
    float2 stage_pairs[kMaxBlocks]; // level 1: block sums of the pass
    Pair before;                    // prefix before the owner block
    Thresh th[2];                   // thresholds of the draws, by parity
    Thresh th_draw;                 // the threshold of this pass's draw, with T
    double T;
    int64_t owner; // winning block, or -1 (degenerate: T == 0)
    int64_t pick;
    int ok;
    // the owner's search through a warp segment: its rows, the prefix before
    // it, the threshold, and the sums of its kPersistWarps sub-slices
    int64_t seg_first, seg_last;
    Pair seg_before;
    Thresh seg_th;
    float2 subsum[kPersistWarps];
};

// Static shared state of one CTA running seed_blocks.
struct BlockShared {
    float2 segsum[kPersistWarps];
    DrawShared ds;
};

// The seeding of problem p by a team of p.nblocks co-resident CTAs, this CTA
// being member b: p.slots and p.mail are the team's own exchange words.
// `smem` is the CTA's dynamic shared memory (point cache, D^2, chunk sums;
// unused when a.cache_supers == 0 and MODE == D2_INPLACE).  Returns when the
// seeding is done, or early -- the same way on every member -- on an error
// recorded in the status word.
template <int DT, int D, int L, int MODE>
__device__ __forceinline__ void seed_blocks(const Problem &p, const PersistArgs &a, const int b,
                                            char *smem, BlockShared &sh)
{
    using G = Geom<DT, D, L>;
    float2 *segsum = sh.segsum;
    DrawShared &ds = sh.ds;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)b * p.chunk;
    const int64_t r1 = (r0 + p.chunk) < p.N ? (r0 + p.chunk) : p.N;
    // dynamic shared memory: [point cache][D^2 of the block][32-row chunk sums]
    char *cache = a.cache_supers > 0 ? smem : nullptr;
    const int64_t cache_bytes = a.cache_supers * (int64_t)kPersistWarps * G::SW * G::RB;
    float *d2s = reinterpret_cast<float *>(smem + cache_bytes);
    float2 *chunk_sums = reinterpret_cast<float2 *>(smem + cache_bytes + ((4 * p.chunk + 15) & ~15ll));
    const int nchunks = (int)((r1 - r0 + 31) / 32);
    const bool chunk_path = (MODE == D2_SMEM) && (p.chunk + 31) / 32 <= kMaxChunks;
    const uint64_t policy =
        a.l2_hint == 1 ? policy_evict_last() : (a.l2_hint == 2 ? policy_evict_first() : 0ull);

    // the plan's limits: this block exists, the level-1 stage and the chunk
    // sums hold what the draw will put there (every CTA sees the same values)
    if (!kpp_check(p.ctl,
                   b >= 0 && b < p.nblocks && p.nblocks <= kMaxBlocks && r0 < r1 &&
                       (!chunk_path || nchunks <= kMaxChunks),
                   201))
        return;
    int64_t ci = first_seed(p);
    if (ci < 0 || ci >= p.N) {
        if (b == 0 && threadIdx.x == 0)
            atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_INVALID_ARG);
        return; // every CTA takes this branch: nobody is left waiting
    }
    if (threadIdx.x == 0) {
        if (b == 0)
            p.idx[0] = ci;
        if (p.K > 1)
            ds.th[1] = thresh_for_u(philox_uniform(p.seed, p.stream_id, 1), p.exact_draws);
    }

    for (int m = 0; m < p.K; ++m) {
        const bool last = (m == p.K - 1);
        const int next = m + 1;
        CentreRegs<DT, D, L> cr;
        cr.load(p.points, p.scales, ci);

        PassIO io{};
        io.ctl = p.ctl;
        io.r0 = r0;
        io.r1 = r1;
        io.first = (m == 0);
        io.reverse = a.reverse && (m & 1);
        io.gpts = reinterpret_cast<const char *>(p.points);
        io.scales = p.scales;
        io.cache = cache;
        io.cache_supers = a.cache_supers;
        io.fill_cache = (m == 0);
        io.d2 = p.d2;
        io.d2_out = last ? p.d2 : nullptr;
        io.d2s = d2s;
        io.segs = segsum;
        io.policy = policy;
        pass_rows<DT, D, L, MODE>(io, cr);
        __syncthreads();

        // publish this block's pair sum (segments in warp order)
        unsigned long long *slots = p.slots + (size_t)(m & 1) * p.nblocks * kSlotWords;
        if (threadIdx.x == 0) {
            Pair bs{};
            for (int w = 0; w < kPersistWarps; ++w)
                bs.add(Pair{segsum[w].x, segsum[w].y});
            st_relaxed_u64(slots + (size_t)b * kSlotWords, pack_slot(bs, m));
            if (p.nblocks == 1) // alone: this block's sum is level 1
                ds.stage_pairs[0] = make_float2(bs.hi, bs.lo);
        }
        if (last && b != 0)
            return; // only block 0 waits, to sum phi
        const bool forced = !last && next < p.n_forced;

        if (warp == 0) {
            // wait for every block's sum of this pass (the grid-wide sync),
            // then the draw's first level: the block holding t = u * T
            bool ok = true;
            for (int k0 = 0; ok && p.nblocks > 1 && k0 < p.nblocks; k0 += 256) {
                const int n = (p.nblocks - k0) < 256 ? (p.nblocks - k0) : 256;
                ok = warp_wait_slots(slots + (size_t)k0 * kSlotWords, n, m, p.ctl, a.timeout_ns,
                                     ds.stage_pairs + k0);
            }
            __syncwarp();
            if (ok && last) { // block 0: phi = the ordered sum of the final block sums
                const PFind r = warp_pfind(
                    p.nblocks,
                    [&](int k) { return Pair{ds.stage_pairs[k].x, ds.stage_pairs[k].y}; },
                    Pair{}, thresh_inf(), false);
                if (lane == 0 && p.phi)
                    p.phi[0] = (double)r.total.hi + (double)r.total.lo;
            } else if (ok && !forced) {
                const PFind r = warp_pfind(
                    p.nblocks,
                    [&](int k) { return Pair{ds.stage_pairs[k].x, ds.stage_pairs[k].y}; },
                    Pair{}, ds.th[next & 1], true);
                if (lane == 0) {
                    ds.th_draw = r.th;
                    if (!(r.total.hi > 0.f)) {
                        ds.owner = -1;
                        ds.T = 0.0;
                    } else if (r.index >= 0) {
                        ds.owner = r.index;
                        ds.before = r.before;
                    } else { // rounding left no block above t: the last with weight
                        ds.owner = r.last_positive;
                        ds.before = Pair{};
                        ds.th_draw.inf = 1;
                    }
                }
            }
            if (lane == 0)
                ds.ok = ok ? 1 : 0;
        } else if (!last) {
            // meanwhile: the uniform of the draw after next, and this block's
            // 32-row chunk sums (for the owner's search below)
            if (threadIdx.x == 32 && next + 1 < p.K)
                ds.th[(next + 1) & 1] =
                    thresh_for_u(philox_uniform(p.seed, p.stream_id, (uint64_t)(next + 1)),
                                 p.exact_draws);
            if (chunk_path && !forced) {
                for (int c = threadIdx.x - 32; c < nchunks; c += blockDim.x - 32) {
                    const int64_t rb = r0 + 32ll * c;
                    const int n = (int)((r1 - rb) < 32 ? (r1 - rb) : 32);
                    Pair cs{};
                    if (kpp_check(p.ctl, rb - r0 + n <= p.chunk, 202))
                        for (int k = 0; k < n; ++k)
                            cs.add(d2s[rb - r0 + k]);
                    chunk_sums[c] = make_float2(cs.hi, cs.lo);
                }
            }
        }
        __syncthreads();
        if (!ds.ok || last)
            return;
        if (forced) {
            ci = p.forced[next];
            if (ci < 0 || ci >= p.N) {
                if (b == 0 && threadIdx.x == 0)
                    atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_INVALID_ARG);
                return; // the same forced index on every CTA
            }
            if (b == 0 && threadIdx.x == 0)
                p.idx[next] = ci;
            continue;
        }
        const int64_t owner = ds.owner;
        if (owner < 0) {
            // sum D^2 == 0: fewer distinct points than K.  This pass's D^2 is
            // the result.
            if (MODE == D2_SMEM)
                for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
                    p.d2[r] = d2s[r - r0];
            if (b == 0 && threadIdx.x == 0) {
                for (int k = next; k < p.K; ++k)
                    p.idx[k] = -1;
                if (p.phi)
                    p.phi[0] = 0.0;
                atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_DEGENERATE);
            }
            return;
        }

        if (owner == b) {
            // the point within this block; then publish the index
            auto d2_at = [&](int64_t row) {
                if (!kpp_check(p.ctl, row >= r0 && row < r1, 203))
                    return 0.f;
                return MODE == D2_SMEM ? d2s[row - r0] : p.d2[row];
            };
            int64_t pick = -1;
            if (chunk_path) {
                // from the 32-row chunk sums made during the wait, by warp 0
                if (warp == 0) {
                    const Pair base = ds.before;
                    Thresh t = ds.th_draw;
                    const PFind r = warp_pfind(
                        nchunks, [&](int k) { return Pair{chunk_sums[k].x, chunk_sums[k].y}; },
                        base, t, false);
                    int c;
                    Pair before = r.before;
                    if (r.index >= 0) {
                        c = (int)r.index;
                    } else {
                        c = r.last_positive >= 0 ? (int)r.last_positive : 0;
                        t.inf = 1;
                    }
                    const int64_t rb = r0 + 32ll * c;
                    const int n = (int)((r1 - rb) < 32 ? (r1 - rb) : 32);
                    const float v =
                        (lane < n && kpp_check(p.ctl, rb - r0 + lane < p.chunk && c < nchunks, 204))
                            ? d2s[rb - r0 + lane]
                            : 0.f;
                    const Find32 f = warp_find32(n, Pair{v, 0.f}, before, t);
                    pick = rb + (f.index >= 0 ? f.index : 0);
                }
            } else {
                // the warp segment (warp 0); the sums of its sub-slices of
                // whole 32-row chunks, one per warp; the sub-slice and the
                // row in it (warp 0)
                if (warp == 0) {
                    Thresh t = ds.th_draw;
                    const PFind r = warp_pfind(
                        kPersistWarps, [&](int k) { return Pair{segsum[k].x, segsum[k].y}; },
                        ds.before, t, false);
                    Pair sbase = ds.before;
                    int seg;
                    if (r.index >= 0) {
                        seg = (int)r.index;
                        sbase = r.before;
                    } else { // rounding: the last segment with weight
                        seg = r.last_positive >= 0 ? (int)r.last_positive : 0;
                        t.inf = 1;
                    }
                    if (lane == 0) {
                        segment_rows(r0, r1 - r0, G::SW, kPersistWarps, seg, &ds.seg_first,
                                     &ds.seg_last);
                        ds.seg_before = sbase;
                        ds.seg_th = t;
                    }
                }
                __syncthreads();
                const int64_t sf = ds.seg_first, sl = ds.seg_last;
                const int64_t per = 32 * (((sl - sf + 31) / 32 + kPersistWarps - 1) / kPersistWarps);
                {
                    const int64_t wb = sf + per * warp;
                    const int64_t we = (wb + per) < sl ? (wb + per) : sl;
                    Pair acc{};
#pragma unroll 4
                    for (int64_t row = wb + lane; row < we; row += 32)
                        acc.add(d2_at(row));
                    const Pair ws = warp_pair_sum(acc);
                    if (lane == 0)
                        ds.subsum[warp] = make_float2(ws.hi, ws.lo);
                }
                __syncthreads();
                if (warp == 0) {
                    Thresh t = ds.seg_th;
                    const PFind r = warp_pfind(
                        kPersistWarps, [&](int k) { return Pair{ds.subsum[k].x, ds.subsum[k].y}; },
                        ds.seg_before, t, false);
                    Pair wbase = ds.seg_before;
                    int w;
                    if (r.index >= 0) {
                        w = (int)r.index;
                        wbase = r.before;
                    } else { // rounding: the last sub-slice with weight
                        w = r.last_positive >= 0 ? (int)r.last_positive : 0;
                        t.inf = 1;
                    }
                    const int64_t wb = sf + per * w;
                    const int64_t we = (wb + per) < sl ? (wb + per) : sl;
                    pick = warp_rows_find(wb < sl ? wb : sf, we, d2_at, wbase, t);
                }
            }
            if (threadIdx.x == 0) {
                kpp_check(p.ctl, pick >= r0 && pick < r1, 205);
                p.idx[next] = pick;
                st_relaxed_u64(p.mail,
                               ((unsigned long long)pick << 32) | (unsigned long long)(uint32_t)next);
                ds.pick = pick;
            }
        } else if (threadIdx.x == 0) {
            ds.pick = wait_mail(p.mail, p.ctl, m, a.timeout_ns);
        }
        __syncthreads();
        ci = ds.pick;
        if (ci < 0)
            return; // a wait gave up: the status word says why
    }
}

template <int DT, int D, int L, int MODE>
__global__ void __launch_bounds__(kPersistThreads, 1)
    persistent_kernel(Problem p, PersistArgs a)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ BlockShared sh;
    seed_blocks<DT, D, L, MODE>(p, a, blockIdx.x, smem, sh);
}

// One specialisation of the persistent kernel, as listed by the per-dtype
// translation units.
using PersistFn = void (*)(Problem, PersistArgs);

struct PSpec {
    int dt, d, lanes, sw, rb;
    PersistFn fn_smem, fn_global;
};

template <int DT, int D, int L>
constexpr PSpec make_pspec()
{
    return PSpec{DT,
                 D,
                 Geom<DT, D, L>::L,
                 Geom<DT, D, L>::SW,
                 Geom<DT, D, L>::RB,
                 &persistent_kernel<DT, D, L, D2_SMEM>,
                 &persistent_kernel<DT, D, L, D2_INPLACE>};
}

// The specialisations built for each stored type (one translation unit each,
// compiled in parallel).
const PSpec *persistent_specs_f32(int *n);
const PSpec *persistent_specs_bf16(int *n);
const PSpec *persistent_specs_fp8(int *n);

} // namespace kpp

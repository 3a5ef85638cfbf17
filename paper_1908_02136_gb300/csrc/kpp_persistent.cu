// kpp_persistent.cu -- persistent form: one cooperative launch runs all K
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
#include "kpp_internal.h"
#include "kpp_pass.cuh"

namespace kpp {

constexpr int kPersistThreads = 512;
constexpr int kPersistWarps = kPersistThreads / 32;

struct DrawShared {
    float2 stage_pairs[kStage]; // level 1: block sums of the pass
    float stage_rows[kStage];   // level 3: D^2 of the owner's segment
    RowsShared rows;
    Pair before;   // prefix before the owner block / segment
    double u;      // draw of the next seed
    double t;      // threshold u * T
    double T;
    int64_t owner; // winning block, or -1 (degenerate: T == 0)
    int64_t seg;
    int64_t pick;
    int ok;
};

template <int DT, int D, int L, int MODE>
__global__ void __launch_bounds__(kPersistThreads, 1)
    persistent_kernel(Problem p, PersistArgs a)
{
    using G = Geom<DT, D, L>;
    extern __shared__ __align__(16) char smem[];
    __shared__ float2 segsum[kPersistWarps];
    __shared__ DrawShared ds;

    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)b * p.chunk;
    const int64_t r1 = (r0 + p.chunk) < p.N ? (r0 + p.chunk) : p.N;
    char *cache = a.cache_supers > 0 ? smem : nullptr;
    const int64_t cache_bytes = a.cache_supers * (int64_t)kPersistWarps * G::SW * G::RB;
    float *d2s = reinterpret_cast<float *>(smem + cache_bytes);
    const uint64_t policy =
        a.l2_hint == 1 ? policy_evict_last() : (a.l2_hint == 2 ? policy_evict_first() : 0ull);

    int64_t ci = first_seed(p);
    if (ci < 0 || ci >= p.N) {
        if (b == 0 && threadIdx.x == 0)
            atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_INVALID_ARG);
        return; // every CTA takes this branch: nobody is left waiting
    }
    if (b == 0 && threadIdx.x == 0)
        p.idx[0] = ci;

    for (int m = 0; m < p.K; ++m) {
        const bool last = (m == p.K - 1);
        const int next = m + 1;
        CentreRegs<DT, D, L> cr;
        cr.load(p.points, p.scales, ci);
        // the next draw's uniform, by a thread that has time to spare
        if (threadIdx.x == blockDim.x - 1 && !last)
            ds.u = philox_uniform(p.seed, p.stream_id, (uint64_t)next);

        PassIO io{};
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
            ds.ok = 1;
        }
        if (last && b != 0)
            return; // only block 0 waits, to sum phi
        __syncthreads();

        // wait for every block's sum of this pass (the grid-wide sync)
        for (int k = threadIdx.x; k < p.nblocks; k += blockDim.x) {
            Pair v;
            if (wait_slot(slots + (size_t)k * kSlotWords, m, p.ctl, a.timeout_ns, &v))
                ds.stage_pairs[k] = make_float2(v.hi, v.lo);
            else
                ds.ok = 0;
        }
        __syncthreads();
        if (!ds.ok)
            return;

        if (last) { // block 0: phi = the ordered sum of the final block sums
            if (warp == 0) {
                const PFind r = warp_pfind(
                    p.nblocks,
                    [&](int k) { return Pair{ds.stage_pairs[k].x, ds.stage_pairs[k].y}; },
                    Pair{}, INFINITY, false);
                if (lane == 0 && p.phi)
                    p.phi[0] = (double)r.total.hi + (double)r.total.lo;
            }
            return;
        }
        if (next < p.n_forced) {
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

        // level 1, on every CTA: the block holding t = u * T
        if (warp == 0) {
            const PFind r = warp_pfind(
                p.nblocks,
                [&](int k) { return Pair{ds.stage_pairs[k].x, ds.stage_pairs[k].y}; }, Pair{},
                ds.u, true);
            if (lane == 0) {
                ds.T = (double)r.total.hi + (double)r.total.lo;
                ds.t = r.t;
                if (!(ds.T > 0.0)) {
                    ds.owner = -1;
                } else if (r.index >= 0) {
                    ds.owner = r.index;
                    ds.before = r.before;
                } else { // rounding left no block above t: the last with weight
                    ds.owner = r.last_positive;
                    ds.before = Pair{};
                    ds.t = INFINITY;
                }
            }
        }
        __syncthreads();
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
                    p.phi[0] = ds.T;
                atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_DEGENERATE);
            }
            return;
        }

        if (owner == b) {
            // levels 2 and 3 from this CTA's own memory: the segment, then the row
            if (warp == 0) {
                const PFind r = warp_pfind(
                    kPersistWarps, [&](int k) { return Pair{segsum[k].x, segsum[k].y}; },
                    ds.before, ds.t, false);
                if (lane == 0) {
                    if (r.index >= 0) {
                        ds.seg = r.index;
                        ds.before = r.before;
                    } else {
                        ds.seg = r.last_positive >= 0 ? r.last_positive : 0;
                        ds.t = INFINITY;
                    }
                }
            }
            __syncthreads();
            int64_t first, lastr;
            segment_rows(r0, r1 - r0, G::SW, kPersistWarps, (int)ds.seg, &first, &lastr);
            const Pair base = ds.before;
            const double t = ds.t;
            int64_t pick;
            if (MODE == D2_SMEM)
                pick = block_rows_find(
                    first, lastr, [&](int64_t row) { return d2s[row - r0]; }, base, t,
                    ds.stage_rows, &ds.rows);
            else
                pick = block_rows_find(
                    first, lastr, [&](int64_t row) { return p.d2[row]; }, base, t,
                    ds.stage_rows, &ds.rows);
            if (threadIdx.x == 0) {
                p.idx[next] = pick;
                st_relaxed_u64(&p.ctl->mail, ((unsigned long long)pick << 32) |
                                                 (unsigned long long)(uint32_t)next);
                ds.pick = pick;
            }
        } else if (threadIdx.x == 0) {
            ds.pick = wait_mail(p.ctl, m, a.timeout_ns);
        }
        __syncthreads();
        ci = ds.pick;
        if (ci < 0)
            return; // a wait gave up: the status word says why
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

using PFn = void (*)(Problem, PersistArgs);

struct PSpec {
    int dt, d, lanes, sw, rb;
    PFn fn_smem, fn_global;
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

const PSpec kPSpecs[] = {
    make_pspec<KPP_F32, 2, 1>(),       make_pspec<KPP_F32, 4, 1>(),
    make_pspec<KPP_F32, 8, 2>(),       make_pspec<KPP_F32, 16, 4>(),
    make_pspec<KPP_F32, 32, 4>(),      make_pspec<KPP_F32, 32, 8>(),
    make_pspec<KPP_F32, 64, 8>(),      make_pspec<KPP_F32, 128, 8>(),
    make_pspec<KPP_BF16, 2, 1>(),      make_pspec<KPP_BF16, 4, 1>(),
    make_pspec<KPP_BF16, 8, 1>(),      make_pspec<KPP_BF16, 16, 2>(),
    make_pspec<KPP_BF16, 32, 4>(),     make_pspec<KPP_BF16, 64, 8>(),
    make_pspec<KPP_BF16, 128, 8>(),    make_pspec<KPP_FP8_E4M3, 2, 1>(),
    make_pspec<KPP_FP8_E4M3, 4, 1>(),  make_pspec<KPP_FP8_E4M3, 8, 1>(),
    make_pspec<KPP_FP8_E4M3, 16, 1>(), make_pspec<KPP_FP8_E4M3, 32, 2>(),
    make_pspec<KPP_FP8_E4M3, 64, 4>(), make_pspec<KPP_FP8_E4M3, 128, 8>(),
};

} // namespace

bool persistent_lookup(int dt, int d, int lanes, PersistentKernel *out)
{
    const PSpec *best = nullptr;
    for (const PSpec &s : kPSpecs) {
        if (s.dt != dt || s.d != d)
            continue;
        if (lanes > 0 && s.lanes != lanes)
            continue;
        if (!best || (s.lanes <= 8 && s.lanes > best->lanes))
            best = &s;
    }
    if (!best)
        return false;
    out->fn_smem = reinterpret_cast<const void *>(best->fn_smem);
    out->fn_global = reinterpret_cast<const void *>(best->fn_global);
    out->rows_align = best->sw;
    out->row_bytes = best->rb;
    out->lanes = best->lanes;
    return true;
}

int persistent_threads() { return kPersistThreads; }
int persistent_segments() { return kPersistWarps; }

cudaError_t persistent_launch(const void *fn, int grid, size_t smem, const Problem &p,
                              const PersistArgs &a, cudaStream_t stream)
{
    Problem pp = p;
    PersistArgs aa = a;
    void *args[] = {&pp, &aa};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPersistThreads), args, smem, stream);
}

} // namespace kpp

// kpp_streamed.cu -- streamed form: one kernel launch per seeding pass.
//
// Launch m (m = 0..K-1) reads the centre index idx[m], streams every point
// once (Algorithm 2: the per-point loop in parallel over contiguous per-CTA
// partitions N_1..N_l), updates D^2 in HBM, and writes per-warp-segment and
// per-CTA D^2 sums.  The last CTA to finish (atomic ticket) draws seed m+1 --
// block, then segment, then point -- and writes idx[m+1] (the sum the
// paper takes with a double-precision Thrust reduction, Section II, fused
// into the pass).  The host captures the K launches into one CUDA graph.
#include "kpp_internal.h"
#include "kpp_pass.cuh"

namespace kpp {

constexpr int kStreamThreads = 256;

// Returns the centre of pass m, or -1 if the kernel must stop.  A sharded
// pass takes it from the exchange buffer (a global index) and records it.
__device__ __forceinline__ int64_t pass_centre(const Problem &p, int m)
{
    if (*(volatile int32_t *)&p.ctl->status != KPP_OK)
        return -1;
    if (p.xchg) {
        const int64_t ci = (int64_t)__ldcg(p.xchg);
        if (ci < 0 || ci >= p.n_global) {
            if (threadIdx.x == 0 && blockIdx.x == 0)
                atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_INVALID_ARG);
            return -1;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0)
            p.idx[m] = ci;
        return ci;
    }
    int64_t ci = (m == 0) ? first_seed(p) : __ldcg(p.idx + m);
    if (ci < 0 || ci >= p.N) {
        if (threadIdx.x == 0 && blockIdx.x == 0)
            atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_INVALID_ARG);
        return -1;
    }
    if (m == 0 && blockIdx.x == 0 && threadIdx.x == 0)
        p.idx[0] = ci;
    return ci;
}

// Block sum, ticket, and -- in the CTA that finishes last -- the draw of
// seed m+1 (or phi after the final pass): the block holding t = u * T from
// the block sums, the segment within it, then the point.
__device__ __forceinline__ void finish_pass(const Problem &p, int m, const Pair &wseg)
{
    __shared__ float2 segsum[kStreamThreads / 32];
    __shared__ float2 stage_pairs[kStage];
    __shared__ int is_last;
    __shared__ int64_t blk_sh, seg_sh;
    __shared__ Pair before_sh;
    __shared__ Thresh th_sh;
    __shared__ double T_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        segsum[warp] = make_float2(wseg.hi, wseg.lo);
    __syncthreads();
    if (threadIdx.x == 0) {
        Pair bs{};
        for (int w = 0; w < kStreamThreads / 32; ++w)
            bs.add(Pair{segsum[w].x, segsum[w].y});
        p.block_sums[blockIdx.x] = make_float2(bs.hi, bs.lo);
        __threadfence(); // this CTA's D^2, segment and block sums before the ticket
        const unsigned prev = atomicAdd(&p.ctl->ticket, 1u);
        is_last = (prev == (unsigned)p.nblocks - 1u);
    }
    __syncthreads();
    if (!is_last)
        return;
    __threadfence();
    if (!kpp_check(p.ctl, p.nblocks <= kStage && (int)blockIdx.x < p.nblocks, 301))
        return;
    for (int k = threadIdx.x; k < p.nblocks; k += blockDim.x)
        stage_pairs[k] = __ldcg(p.block_sums + k);
    __syncthreads();
    if (p.shard_total) { // sharded pass: the shard's total, no draw here
        if (warp == 0) {
            const PFind r = warp_pfind(
                p.nblocks, [&](int k) { return Pair{stage_pairs[k].x, stage_pairs[k].y}; },
                Pair{}, thresh_inf(), false);
            if (lane == 0) {
                p.shard_total[0] = r.total.hi;
                p.shard_total[1] = r.total.lo;
                p.ctl->ticket = 0u;
            }
        }
        return;
    }
    const bool final_pass = (m == p.K - 1);
    const int next = m + 1;
    const bool forced = !final_pass && next < p.n_forced;
    if (warp == 0) {
        const double u = (final_pass || forced) ? 0.0
                                                : philox_uniform(p.seed, p.stream_id, (uint64_t)next);
        const PFind r = warp_pfind(
            p.nblocks, [&](int k) { return Pair{stage_pairs[k].x, stage_pairs[k].y}; }, Pair{},
            thresh_for_u(u, p.exact_draws), true);
        if (lane == 0) {
            T_sh = (double)r.total.hi + (double)r.total.lo;
            th_sh = r.th;
            blk_sh = r.index;
            before_sh = r.before;
            if (r.index < 0) { // rounding left no block above t: the last with weight
                blk_sh = r.last_positive;
                before_sh = Pair{};
                th_sh.inf = 1;
            }
        }
    }
    __syncthreads();
    if (final_pass || forced || !(T_sh > 0.0)) {
        if (threadIdx.x == 0) {
            if (final_pass) {
                if (p.phi)
                    p.phi[0] = T_sh;
            } else if (forced) {
                p.idx[next] = p.forced[next];
            } else { // sum D^2 == 0: fewer distinct points than K
                for (int k = next; k < p.K; ++k)
                    p.idx[k] = -1;
                if (p.phi)
                    p.phi[0] = T_sh;
                atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_DEGENERATE);
            }
            p.ctl->ticket = 0u;
        }
        return;
    }
    const int64_t blk = blk_sh;
    const int64_t row0 = blk * p.chunk;
    const int64_t rows_blk = (p.N - row0) < p.chunk ? (p.N - row0) : p.chunk;
    if (warp == 0) {
        const float2 *segs = p.seg_sums + blk * (int64_t)p.nseg;
        const PFind r = warp_pfind(
            p.nseg,
            [&](int k) {
                const float2 v = __ldcg(segs + k);
                return Pair{v.x, v.y};
            },
            before_sh, th_sh, false);
        if (lane == 0) {
            if (r.index >= 0) {
                seg_sh = r.index;
                before_sh = r.before;
            } else {
                seg_sh = r.last_positive >= 0 ? r.last_positive : 0;
                th_sh.inf = 1;
            }
        }
    }
    __syncthreads();
    if (warp != 0)
        return;
    int64_t first, last;
    segment_rows(row0, rows_blk, p.sw, p.nseg, (int)seg_sh, &first, &last);
    const int64_t pick = warp_rows_find(
        first, last,
        [&](int64_t row) {
            return kpp_check(p.ctl, row >= 0 && row < p.N, 302) ? __ldcg(p.d2 + row) : 0.f;
        },
        before_sh, th_sh);
    if (threadIdx.x == 0) {
        kpp_check(p.ctl, blk < p.nblocks && pick >= row0 && pick < row0 + rows_blk, 303);
        p.idx[next] = pick;
        p.ctl->ticket = 0u; // ready for the next launch
    }
}

template <int DT, int D, int L>
__global__ void __launch_bounds__(kStreamThreads)
    streamed_pass_kernel(Problem p, int m)
{
    const int64_t ci = pass_centre(p, m);
    if (ci < 0)
        return;
    PassIO io{};
    io.ctl = p.ctl;
    io.r0 = (int64_t)blockIdx.x * p.chunk;
    io.r1 = (io.r0 + p.chunk) < p.N ? (io.r0 + p.chunk) : p.N;
    io.gpts = reinterpret_cast<const char *>(p.points);
    io.scales = p.scales;
    io.d2 = p.d2;
    io.segs = p.seg_sums + (int64_t)blockIdx.x * p.nseg;
    // The paper's own step (Section II) recomputes every point's distance to
    // all seeds chosen so far; the incremental form takes only the newest.
    // Both keep the minimum of the same FP32 distances, so D^2 is identical.
    Pair w{};
    for (int j = p.recompute ? 0 : m; j <= m; ++j) {
        const int64_t cj = (j == m) ? ci : __ldcg(p.idx + j);
        CentreRegs<DT, D, L> cr;
        if (p.xchg) // the centre row as the exchange buffer carries it
            cr.load(p.xchg + 2, reinterpret_cast<const float *>(p.xchg + 1), 0);
        else
            cr.load(p.points, p.scales, cj);
        io.first = (j == 0);
        w = pass_rows<DT, D, L, D2_INPLACE>(io, cr);
    }
    finish_pass(p, m, w);
}

template <int DT>
__global__ void __launch_bounds__(kStreamThreads)
    streamed_pass_generic_kernel(Problem p, int m)
{
    extern __shared__ float c_sh[];
    const int64_t ci = pass_centre(p, m);
    if (ci < 0)
        return;
    PassIO io{};
    io.ctl = p.ctl;
    io.r0 = (int64_t)blockIdx.x * p.chunk;
    io.r1 = (io.r0 + p.chunk) < p.N ? (io.r0 + p.chunk) : p.N;
    io.gpts = reinterpret_cast<const char *>(p.points);
    io.scales = p.scales;
    io.d2 = p.d2;
    io.segs = p.seg_sums + (int64_t)blockIdx.x * p.nseg;
    Pair w{};
    for (int j = p.recompute ? 0 : m; j <= m; ++j) {
        const int64_t cj = (j == m) ? ci : __ldcg(p.idx + j);
        __syncthreads(); // the previous centre is no longer read
        if (p.xchg)
            load_centre_smem<DT>(p.xchg + 2, reinterpret_cast<const float *>(p.xchg + 1), 0, p.d,
                                 c_sh);
        else
            load_centre_smem<DT>(p.points, p.scales, cj, p.d, c_sh);
        __syncthreads();
        io.first = (j == 0);
        w = pass_rows_generic<DT>(io, p.d, c_sh);
    }
    finish_pass(p, m, w);
}

// ---------------------------------------------------------------------------
// Point-sharded seeding: one problem's rows split into contiguous ranges,
// one per process (Algorithm 2's partition N_1..N_l across GPUs).  A process
// holds rows [row0, row0 + p.N) of the n_global rows; between its passes the
// processes gather their D^2 totals and sum their exchange buffers.
// ---------------------------------------------------------------------------

// Copies local row `r` (stored bytes and FP8 scale) of the shard into the
// exchange buffer under global index `gidx`; all threads of the CTA take part.
__device__ __forceinline__ void shard_put_row(const Problem &p, int64_t r, int64_t gidx,
                                              long long *xchg, int eb)
{
    const int64_t rb = (int64_t)p.d * eb;
    if (!kpp_check(p.ctl, r >= 0 && r < p.N, 603))
        return;
    const unsigned char *src = reinterpret_cast<const unsigned char *>(p.points) + r * rb;
    unsigned char *dst = reinterpret_cast<unsigned char *>(xchg + 2);
    for (int64_t k = threadIdx.x; k < rb; k += blockDim.x)
        dst[k] = src[k];
    if (threadIdx.x == 0) {
        xchg[0] = (long long)gidx;
        xchg[1] = p.scales ? (long long)__float_as_uint(p.scales[r]) : 0ll;
    }
}

__device__ __forceinline__ void zero_words(long long *w, int64_t n)
{
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x)
        w[k] = 0;
}

// The first seed, min(floor(u_0 * n_global), n_global - 1): the process
// holding it writes its row, every other one zeros.
__global__ void __launch_bounds__(kStreamThreads)
    shard_first_kernel(Problem p, int64_t row0, long long *xchg, int64_t words, int eb)
{
    zero_words(xchg, words);
    __syncthreads();
    const double u = philox_uniform(p.seed, p.stream_id, 0);
    int64_t i0 = (int64_t)floor(u * (double)p.n_global);
    i0 = i0 < p.n_global - 1 ? i0 : p.n_global - 1;
    if (i0 >= row0 && i0 < row0 + p.N)
        shard_put_row(p, i0 - row0, i0, xchg, eb);
}

// The draw of seed m + 1 after pass m, given every process's D^2 total
// (`totals`, world FP32 pairs in rank order, the same on every process):
// every process finds the owner rank whose running total passes
// t = u_{m+1} * T; the owner narrows it to a block, a warp segment and a row
// of its own D^2 exactly as the single-GPU streamed form does, and writes the
// row into the exchange buffer; the others write zeros.  T = 0 (fewer
// distinct points than K) stops the seeding on every process alike.
__global__ void __launch_bounds__(kStreamThreads)
    shard_pick_kernel(Problem p, int m, int rank, int world, const float *totals, int64_t row0,
                      long long *xchg, int64_t words, int eb)
{
    __shared__ Thresh th_sh;
    __shared__ Pair before_sh;
    __shared__ int64_t sel_sh, pick_sh;
    __shared__ int degenerate_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (*(volatile int32_t *)&p.ctl->status != KPP_OK)
        return;
    zero_words(xchg, words);
    if (warp == 0) {
        const double u = philox_uniform(p.seed, p.stream_id, (uint64_t)(m + 1));
        const PFind r = warp_pfind(
            world, [&](int k) { return Pair{totals[2 * k], totals[2 * k + 1]}; }, Pair{},
            thresh_for_u(u, p.exact_draws), true);
        if (lane == 0) {
            degenerate_sh = !(r.total.hi > 0.f);
            th_sh = r.th;
            before_sh = r.before;
            sel_sh = r.index;
            if (r.index < 0) { // rounding left no rank above t: the last with weight
                sel_sh = r.last_positive;
                before_sh = Pair{};
                th_sh.inf = 1;
            }
        }
    }
    __syncthreads();
    if (degenerate_sh) {
        if (threadIdx.x == 0) {
            for (int k = m + 1; k < p.K; ++k)
                p.idx[k] = -1;
            atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_DEGENERATE);
        }
        return;
    }
    if (sel_sh != rank)
        return;
    if (warp == 0) {
        // block, segment, row -- as the streamed form's own draw
        Thresh th = th_sh;
        PFind r = warp_pfind(
            p.nblocks,
            [&](int k) {
                const float2 v = __ldcg(p.block_sums + k);
                return Pair{v.x, v.y};
            },
            before_sh, th, false);
        int64_t blk = r.index;
        Pair before = r.before;
        if (blk < 0) {
            blk = r.last_positive >= 0 ? r.last_positive : 0;
            before = before_sh;
            th.inf = 1;
        }
        const float2 *segs = p.seg_sums + blk * (int64_t)p.nseg;
        r = warp_pfind(
            p.nseg,
            [&](int k) {
                const float2 v = __ldcg(segs + k);
                return Pair{v.x, v.y};
            },
            before, th, false);
        int64_t seg = r.index;
        if (seg >= 0) {
            before = r.before;
        } else {
            seg = r.last_positive >= 0 ? r.last_positive : 0;
            th.inf = 1;
        }
        const int64_t rb0 = blk * p.chunk;
        const int64_t rows_blk = (p.N - rb0) < p.chunk ? (p.N - rb0) : p.chunk;
        int64_t first, last;
        segment_rows(rb0, rows_blk, p.sw, p.nseg, (int)seg, &first, &last);
        const int64_t pick = warp_rows_find(
            first, last,
            [&](int64_t row) {
                return kpp_check(p.ctl, row >= 0 && row < p.N, 601) ? __ldcg(p.d2 + row) : 0.f;
            },
            before, th);
        if (lane == 0)
            pick_sh = kpp_check(p.ctl, blk < p.nblocks && pick >= 0 && pick < p.N, 602) ? pick : 0;
    }
    __syncthreads();
    shard_put_row(p, pick_sh, row0 + pick_sh, xchg, eb);
}

// phi = the processes' final D^2 totals added in rank order (FP64 result).
__global__ void shard_phi_kernel(const float *totals, int world, double *phi)
{
    const PFind r = warp_pfind(
        world, [&](int k) { return Pair{totals[2 * k], totals[2 * k + 1]}; }, Pair{},
        thresh_inf(), false);
    if (threadIdx.x == 0)
        phi[0] = (double)r.total.hi + (double)r.total.lo;
}

// ---------------------------------------------------------------------------
// Host side: specialisation table and launch.
// ---------------------------------------------------------------------------
namespace {

using PassFn = void (*)(Problem, int);

struct Spec {
    int dt, d, lanes, sw; // sw: rows per warp super-iteration
    PassFn fn;
};

template <int DT, int D, int L>
constexpr Spec make_spec()
{
    return Spec{DT, D, Geom<DT, D, L>::L, Geom<DT, D, L>::SW, &streamed_pass_kernel<DT, D, L>};
}

// Only combinations whose lanes divide the row's 16-byte vectors are valid.
const Spec kSpecs[] = {
    // FP32: rows of 8 .. 512 bytes
    make_spec<KPP_F32, 2, 1>(), make_spec<KPP_F32, 4, 1>(), make_spec<KPP_F32, 8, 1>(),
    make_spec<KPP_F32, 8, 2>(), make_spec<KPP_F32, 16, 2>(), make_spec<KPP_F32, 16, 4>(),
    make_spec<KPP_F32, 32, 2>(), make_spec<KPP_F32, 32, 4>(), make_spec<KPP_F32, 32, 8>(),
    make_spec<KPP_F32, 64, 4>(), make_spec<KPP_F32, 64, 8>(), make_spec<KPP_F32, 64, 16>(),
    make_spec<KPP_F32, 128, 8>(), make_spec<KPP_F32, 128, 16>(), make_spec<KPP_F32, 128, 32>(),
    // BF16: rows of 4 .. 256 bytes
    make_spec<KPP_BF16, 2, 1>(), make_spec<KPP_BF16, 4, 1>(), make_spec<KPP_BF16, 8, 1>(),
    make_spec<KPP_BF16, 16, 1>(), make_spec<KPP_BF16, 16, 2>(), make_spec<KPP_BF16, 32, 2>(),
    make_spec<KPP_BF16, 32, 4>(), make_spec<KPP_BF16, 64, 4>(), make_spec<KPP_BF16, 64, 8>(),
    make_spec<KPP_BF16, 128, 4>(), make_spec<KPP_BF16, 128, 8>(), make_spec<KPP_BF16, 128, 16>(),
    // FP8: rows of 2 .. 128 bytes
    make_spec<KPP_FP8_E4M3, 2, 1>(), make_spec<KPP_FP8_E4M3, 4, 1>(),
    make_spec<KPP_FP8_E4M3, 8, 1>(), make_spec<KPP_FP8_E4M3, 16, 1>(),
    make_spec<KPP_FP8_E4M3, 32, 1>(), make_spec<KPP_FP8_E4M3, 32, 2>(),
    make_spec<KPP_FP8_E4M3, 64, 2>(), make_spec<KPP_FP8_E4M3, 64, 4>(),
    make_spec<KPP_FP8_E4M3, 128, 4>(), make_spec<KPP_FP8_E4M3, 128, 8>(),
};

PassFn generic_fn(int dt)
{
    switch (dt) {
    case KPP_F32:
        return &streamed_pass_generic_kernel<KPP_F32>;
    case KPP_BF16:
        return &streamed_pass_generic_kernel<KPP_BF16>;
    default:
        return &streamed_pass_generic_kernel<KPP_FP8_E4M3>;
    }
}

} // namespace

// Picks the specialisation: the requested lanes if built, else the default
// (8 lanes, or the widest built below that); the generic kernel otherwise.
bool streamed_lookup(int dt, int d, int lanes, StreamedKernel *out)
{
    const Spec *best = nullptr;
    for (const Spec &s : kSpecs) {
        if (s.dt != dt || s.d != d)
            continue;
        if (lanes > 0) {
            if (s.lanes == lanes)
                best = &s;
        } else if (s.lanes <= 8 && (!best || s.lanes > best->lanes)) {
            best = &s;
        }
    }
    if (!best) {
        out->fn = reinterpret_cast<const void *>(generic_fn(dt));
        out->rows_align = 32;
        out->lanes = 0;
        out->generic = true;
        return lanes <= 0;
    }
    out->fn = reinterpret_cast<const void *>(best->fn);
    out->rows_align = best->sw;
    out->lanes = best->lanes;
    out->generic = false;
    return true;
}

int streamed_threads() { return kStreamThreads; }
int streamed_segments() { return kStreamThreads / 32; }

size_t streamed_smem(const StreamedKernel &k, int d)
{
    return k.generic ? 2 * sizeof(float) * (size_t)d : 0;
}

cudaError_t streamed_launch(const StreamedKernel &k, int grid, const Problem &p, int m,
                            cudaStream_t stream)
{
    Problem pp = p;
    int mm = m;
    void *args[] = {&pp, &mm};
    return cudaLaunchKernel(k.fn, dim3(grid), dim3(kStreamThreads), args, streamed_smem(k, p.d),
                            stream);
}

cudaError_t shard_first_launch(const Problem &p, int64_t row0, long long *xchg, int eb,
                               cudaStream_t stream)
{
    shard_first_kernel<<<1, kStreamThreads, 0, stream>>>(p, row0, xchg, xchg_words(p.d, eb), eb);
    return cudaGetLastError();
}

cudaError_t shard_pick_launch(const Problem &p, int m, int rank, int world, const float *totals,
                              int64_t row0, long long *xchg, int eb, cudaStream_t stream)
{
    shard_pick_kernel<<<1, kStreamThreads, 0, stream>>>(p, m, rank, world, totals, row0, xchg,
                                                        xchg_words(p.d, eb), eb);
    return cudaGetLastError();
}

cudaError_t shard_phi_launch(const float *totals, int world, double *phi, cudaStream_t stream)
{
    shard_phi_kernel<<<1, 32, 0, stream>>>(totals, world, phi);
    return cudaGetLastError();
}

} // namespace kpp

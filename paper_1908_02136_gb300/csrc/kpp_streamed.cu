// kpp_streamed.cu -- streamed form: one kernel launch per seeding pass.
//
// Launch m (m = 0..K-1) reads the centre index idx[m], streams every point
// once (Algorithm 2: the per-point loop "in parallel", the points
// partitioned into contiguous per-CTA ranges N_1..N_l), updates D^2 in HBM
// and writes the CTA's FP64 D^2 sum.  The last CTA to finish (atomic
// ticket) draws seed m+1 from the block sums and a rescan of the winning
// block (the sum the paper takes with a double-precision Thrust reduction,
// Section II, fused into the pass), and writes idx[m+1].  The K launches are
// captured once into a CUDA graph by the host code.
#include "kpp_internal.h"
#include "kpp_pass.cuh"

namespace kpp {

constexpr int kStreamThreads = 256;

// Work after the pass, by the CTA that finishes last: the draw of seed m+1,
// or phi after the final pass.
__device__ __forceinline__ void last_cta_epilogue(const Problem &p, int m, double *shd,
                                                  int64_t *shi)
{
    if (m == p.K - 1) { // phi: the ordered FP64 sum of the block sums
        double total = block_ordered_total<kStreamThreads>(
            p.nblocks, [&](int64_t k) { return ld_cg(p.block_sums + k); }, shd);
        if (threadIdx.x == 0 && p.phi)
            p.phi[0] = total;
        return;
    }
    const int next = m + 1;
    if (next < p.n_forced) {
        if (threadIdx.x == 0)
            p.idx[next] = p.forced[next];
        return;
    }
    const double u = philox_uniform(p.seed, p.stream_id, (uint64_t)next);
    double T;
    int64_t pick = hierarchical_draw<kStreamThreads>(p.block_sums, p.nblocks, p.d2, p.N, p.chunk,
                                                     u, shd, shi, &T);
    if (threadIdx.x == 0) {
        if (pick < 0) { // sum D^2 == 0: fewer distinct points than K
            for (int k = next; k < p.K; ++k)
                p.idx[k] = -1;
            if (p.phi)
                p.phi[0] = T;
            p.ctl->status = KPP_ERR_DEGENERATE;
        } else {
            p.idx[next] = pick;
        }
    }
}

// Returns the centre of pass m, or -1 if the kernel must stop.
__device__ __forceinline__ int64_t pass_centre(const Problem &p, int m)
{
    if (*(volatile int32_t *)&p.ctl->status != KPP_OK)
        return -1;
    int64_t ci = (m == 0) ? first_seed(p) : __ldcg(p.idx + m);
    if (ci < 0 || ci >= p.N) {
        if (threadIdx.x == 0 && blockIdx.x == 0)
            p.ctl->status = KPP_ERR_INVALID_ARG;
        return -1;
    }
    if (m == 0 && blockIdx.x == 0 && threadIdx.x == 0)
        p.idx[0] = ci;
    return ci;
}

// Block sum, ticket, and the last CTA's epilogue.
__device__ __forceinline__ void finish_pass(const Problem &p, int m, const Acc2 &acc)
{
    __shared__ double shd[kStreamThreads / 32 + 1];
    __shared__ int64_t shi[kStreamThreads / 32];
    __shared__ int is_last;
    __threadfence(); // this thread's D^2 stores before the ticket
    double s = block_sum<kStreamThreads>(acc.value(), shd);
    if (threadIdx.x == 0) {
        p.block_sums[blockIdx.x] = s;
        __threadfence();
        unsigned prev = atomicAdd(&p.ctl->ticket, 1u);
        is_last = (prev == (unsigned)p.nblocks - 1u);
    }
    __syncthreads();
    if (!is_last)
        return;
    __threadfence();
    last_cta_epilogue(p, m, shd, shi);
    if (threadIdx.x == 0)
        p.ctl->ticket = 0u; // ready for the next launch
}

template <int DT, int D, int L>
__global__ void __launch_bounds__(kStreamThreads)
    streamed_pass_kernel(Problem p, int m)
{
    const int64_t ci = pass_centre(p, m);
    if (ci < 0)
        return;
    CentreRegs<DT, D, L> cr;
    cr.load(p.points, p.scales, ci);
    const int64_t r0 = (int64_t)blockIdx.x * p.chunk;
    const int64_t r1 = (r0 + p.chunk) < p.N ? (r0 + p.chunk) : p.N;
    Acc2 acc = pass_rows<DT, D, L>(p.points, p.scales, p.d2, r0, r1, m == 0, cr);
    finish_pass(p, m, acc);
}

template <int DT>
__global__ void __launch_bounds__(kStreamThreads)
    streamed_pass_generic_kernel(Problem p, int m)
{
    extern __shared__ float c_sh[];
    const int64_t ci = pass_centre(p, m);
    if (ci < 0)
        return;
    load_centre_smem<DT>(p.points, p.scales, ci, p.d, c_sh);
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * p.chunk;
    const int64_t r1 = (r0 + p.chunk) < p.N ? (r0 + p.chunk) : p.N;
    Acc2 acc = pass_rows_generic<DT>(p.points, p.scales, p.d2, r0, r1, p.d, m == 0, c_sh);
    finish_pass(p, m, acc);
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

// Only combinations whose lanes divide the row's vectors are valid; the
// table below lists, per dtype, the ones that compile for that dtype.
const Spec kSpecs[] = {
    // FP32: rows of 8, 16, 32, 64, 128, 256, 512 bytes
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

// Picks the specialisation: requested lanes if built, else the default
// (8 lanes, or the widest built below that).
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

cudaError_t streamed_launch(const StreamedKernel &k, int grid, const Problem &p, int m,
                            cudaStream_t stream)
{
    Problem pp = p;
    int mm = m;
    void *args[] = {&pp, &mm};
    size_t smem = k.generic ? sizeof(float) * (size_t)p.d : 0;
    return cudaLaunchKernel(k.fn, dim3(grid), dim3(kStreamThreads), args, smem, stream);
}

} // namespace kpp

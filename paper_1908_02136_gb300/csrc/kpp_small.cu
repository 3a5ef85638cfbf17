// kpp_small.cu -- small form: the whole seeding of a problem that fits in
// one SM's shared memory, by one CTA of 1024 threads.
//
// The points (decoded to FP32; FP8 keeps the E4M3 values and the row
// scales), D^2 and the draws of the next 1024 passes live in shared memory
// for all K passes, so a pass touches no global memory and synchronises
// with two CTA barriers only -- no grid-wide exchange, whose latency bounds
// the persistent form on small problems.  Thread t owns the contiguous rows
// [t*P, (t+1)*P) (P = ceil(N / 1024)), so index order is warp-major, then
// lane, then row, and the draw's inverse CDF (Algorithm 1's probability
// line) is hierarchical in the same order:
//   pass m: every thread takes the distance of its rows to the newest
//   centre (difference form, FP32), min-updates their D^2 and sums it as an
//   FP32 two-sum pair; each warp scans its lanes' sums; barrier; every warp
//   scans the 32 warp totals (the same arithmetic everywhere, so all agree
//   on T and on the warp holding t = u * T); that warp finds the lane, the
//   lane walks its rows; barrier.
#include "kpp_internal.h"
#include "kpp_pass.cuh"

namespace kpp {
namespace {

constexpr int kSmallThreads = 1024;
constexpr int kSmallDraws = 1024; // draws computed ahead, one per thread

struct SmallShared {
    float2 wsum[kSmallThreads / 32];
    double u[kSmallDraws];   // the draws of the next passes
    float2 usp[kSmallDraws]; // their float splits (u ~ x + y), off the pass's critical path
    int64_t pick;
};

// min-update of row r's D^2 in shared memory; returns the new value
__device__ __forceinline__ float small_update(float *D2, int r, float v, bool first)
{
    if (first) {
        D2[r] = v;
        return v;
    }
    const float o = D2[r];
    if (v < o) {
        D2[r] = v;
        return v;
    }
    return o;
}

template <int DT, int D>
__global__ void __launch_bounds__(kSmallThreads, 1) small_kernel(Problem p)
{
    extern __shared__ __align__(16) float smem_f[];
    __shared__ SmallShared sh;
    const int d = D > 0 ? D : p.d;
    const int N = (int)p.N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) { // the status block starts clean (no memset launch before this one)
        p.ctl->status = KPP_OK;
        p.ctl->bounds_site = 0;
    }
    __syncthreads();
    float *X = smem_f;                                  // [N x d] stored values (FP8: E4M3 value)
    float *S = X + (int64_t)N * d;                      // [N] FP8 row scales
    float *D2 = S + (DT == KPP_FP8_E4M3 ? N : 0);       // [N]
    {
        // stage the stored points: 16-byte vectors, several in flight per
        // thread, decoded into shared memory; then the elements past the
        // last whole vector, and the FP8 row scales
        constexpr int EPV = Fmt<DT>::per16, U = 4;
        const int64_t nel = (int64_t)N * d;
        const int64_t nv = nel / EPV;
        const uint4 *src = reinterpret_cast<const uint4 *>(p.points);
        for (int64_t v0 = tid; v0 < nv; v0 += U * kSmallThreads) {
            uint4 buf[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (v0 + (int64_t)u * kSmallThreads < nv)
                    buf[u] = ld_stream16(src + v0 + (int64_t)u * kSmallThreads);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t v = v0 + (int64_t)u * kSmallThreads;
                if (v < nv) {
                    float f[EPV];
                    decode16<DT>(buf[u], f);
#pragma unroll
                    for (int e = 0; e < EPV; ++e)
                        X[v * EPV + e] = f[e];
                }
            }
        }
        for (int64_t k = nv * EPV + tid; k < nel; k += kSmallThreads)
            X[k] = decode1<DT>(p.points, k);
        if (DT == KPP_FP8_E4M3) {
            for (int r0_ = tid; r0_ < N; r0_ += U * kSmallThreads) {
                float sv[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    sv[u] = (r0_ + u * kSmallThreads < N) ? __ldg(p.scales + r0_ + u * kSmallThreads)
                                                         : 0.f;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (r0_ + u * kSmallThreads < N)
                        S[r0_ + u * kSmallThreads] = sv[u];
            }
        }
    }
    const int P = (N + kSmallThreads - 1) / kSmallThreads;
    const int r0 = tid * P < N ? tid * P : N;
    const int r1 = r0 + P < N ? r0 + P : N;
    if (!kpp_check(p.ctl, r0 >= 0 && r1 <= N && r0 <= r1, 401))
        return;

    int64_t ci = first_seed(p);
    if (ci < 0 || ci >= N) { // a forced first index out of range (same on every thread)
        if (tid == 0)
            atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_INVALID_ARG);
        return;
    }
    if (tid == 0)
        p.idx[0] = ci;

    for (int m = 0; m < p.K; ++m) {
        const bool last = (m == p.K - 1);
        const int next = m + 1;
        const bool forced = !last && next < p.n_forced;
        if (m % kSmallDraws == 0) {
            // the draws of the next 1024 passes, one per thread; the barrier
            // also orders the first pass after the loads above
            const int64_t k = (int64_t)m + 1 + tid;
            const double u = k < p.K ? philox_uniform(p.seed, p.stream_id, (uint64_t)k) : 0.0;
            const float uh = (float)u;
            sh.u[tid] = u;
            sh.usp[tid] = make_float2(uh, (float)(u - (double)uh));
            __syncthreads();
        }
        // the centre, decoded as the other forms decode it (FP8: c = s * q
        // as an exact pair), then the distance, min-update and pair sum of
        // this thread's rows
        if (!kpp_check(p.ctl, ci >= 0 && ci < N, 403))
            ci = 0;
        const float cs = (DT == KPP_FP8_E4M3) ? S[ci] : 1.f;
        const float *crow = X + ci * d;
        Pair acc{};
        if constexpr (D > 0) {
            float c[D], cl[D];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                if constexpr (DT == KPP_FP8_E4M3)
                    split_fp8_centre(cs, crow[j], c[j], cl[j]);
                else
                    c[j] = crow[j];
            }
            for (int r = r0; r < r1; ++r) {
                const float *x = X + (int64_t)r * D;
                const float sr = (DT == KPP_FP8_E4M3) ? S[r] : 1.f;
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int j = 0; j < D; j += 2) {
                    float t0, t1;
                    if constexpr (DT == KPP_FP8_E4M3) {
                        t0 = diff_fp8(sr, x[j], c[j], cl[j]);
                        t1 = diff_fp8(sr, x[j + 1], c[j + 1], cl[j + 1]);
                    } else {
                        t0 = __fsub_rn(x[j], c[j]);
                        t1 = __fsub_rn(x[j + 1], c[j + 1]);
                    }
                    a0 = __fmaf_rn(t0, t0, a0);
                    a1 = __fmaf_rn(t1, t1, a1);
                }
                acc.add(small_update(D2, r, __fadd_rn(a0, a1), m == 0));
            }
        } else {
            for (int r = r0; r < r1; ++r) {
                const float *x = X + (int64_t)r * d;
                const float sr = (DT == KPP_FP8_E4M3) ? S[r] : 1.f;
                float a0 = 0.f, a1 = 0.f;
                for (int j = 0; j < d; ++j) {
                    float t;
                    if constexpr (DT == KPP_FP8_E4M3) {
                        float h, l;
                        split_fp8_centre(cs, crow[j], h, l);
                        t = diff_fp8(sr, x[j], h, l);
                    } else {
                        t = __fsub_rn(x[j], crow[j]);
                    }
                    if (j & 1)
                        a1 = __fmaf_rn(t, t, a1);
                    else
                        a0 = __fmaf_rn(t, t, a0);
                }
                acc.add(small_update(D2, r, __fadd_rn(a0, a1), m == 0));
            }
        }
        // lanes' prefixes within the warp; the warp totals
        Pair lex;
        const Pair lin = warp_pair_scan(acc, lex);
        if (lane == 31)
            sh.wsum[warp] = make_float2(lin.hi, lin.lo);
        __syncthreads();
        // every warp scans the warp totals (identically)
        const Pair wv{sh.wsum[lane].x, sh.wsum[lane].y};
        Pair wex;
        const Pair win = warp_pair_scan(wv, wex);
        const Pair T = shfl_pair(win, 31);
        if (last) {
            if (tid == 0 && p.phi)
                p.phi[0] = (double)T.hi + (double)T.lo;
            break;
        }
        if (forced) {
            const int64_t f = p.forced[next];
            if (f < 0 || f >= N) {
                if (tid == 0)
                    atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_INVALID_ARG);
                return; // the same forced index on every thread
            }
            if (tid == 0) {
                p.idx[next] = f;
                sh.pick = f;
            }
        } else if (!(T.hi > 0.f)) { // sum D^2 == 0: fewer distinct points than K
            if (tid == 0) {
                for (int k = next; k < p.K; ++k)
                    p.idx[k] = -1;
                if (p.phi)
                    p.phi[0] = 0.0;
                atomicCAS(&p.ctl->status, KPP_OK, KPP_ERR_DEGENERATE);
            }
            break;
        } else {
            const int du = m % kSmallDraws;
            Thresh th = thresh_for_split(sh.u[du], sh.usp[du].x, sh.usp[du].y, p.exact_draws);
            thresh_set_total(th, T);
            // the warp holding t: the first whose inclusive prefix passes it
            const unsigned wcross = __ballot_sync(0xffffffffu, th.gt(win));
            int ws;
            if (wcross) {
                ws = __ffs(wcross) - 1;
            } else { // rounding left no warp above t: the last warp with weight
                const unsigned pos = __ballot_sync(0xffffffffu, wv.hi > 0.f);
                ws = 31 - __clz(pos);
                th.inf = 1;
            }
            const Pair wbase = shfl_pair(wex, ws);
            if (warp == ws) {
                // the lane, then the row
                const unsigned lcross =
                    __ballot_sync(0xffffffffu, r0 < r1 && th.gt(pair_sum(wbase, lin)));
                int ls;
                if (lcross) {
                    ls = __ffs(lcross) - 1;
                } else {
                    const unsigned pos = __ballot_sync(0xffffffffu, acc.hi > 0.f);
                    ls = pos ? 31 - __clz(pos) : 0;
                    th.inf = 1;
                }
                const Pair lbase = pair_sum(wbase, shfl_pair(lex, ls));
                if (lane == ls) {
                    Pair run = lbase;
                    int pick = -1, lastpos = -1;
                    for (int r = r0; r < r1; ++r) {
                        const float v = D2[r];
                        const Pair nx = pair_sum(run, Pair{v, 0.f});
                        if (v > 0.f) {
                            if (th.gt(nx)) {
                                pick = r;
                                break;
                            }
                            lastpos = r;
                        }
                        run = nx;
                    }
                    if (pick < 0)
                        pick = lastpos >= 0 ? lastpos : r0;
                    if (!kpp_check(p.ctl, pick >= 0 && pick < N, 402))
                        pick = 0;
                    sh.pick = pick;
                    p.idx[next] = pick;
                }
            }
        }
        // the pick to every thread; also orders this pass's reads of sh
        // before the next pass's writes
        __syncthreads();
        ci = sh.pick;
    }
    __syncthreads();
    for (int r = tid; r < N; r += kSmallThreads)
        p.d2[r] = D2[r];
}

using SmallFn = void (*)(Problem);

template <int DT>
SmallFn small_fn(int d)
{
    switch (d) {
    case 2:
        return &small_kernel<DT, 2>;
    case 4:
        return &small_kernel<DT, 4>;
    case 8:
        return &small_kernel<DT, 8>;
    case 16:
        return &small_kernel<DT, 16>;
    default:
        return &small_kernel<DT, 0>;
    }
}

} // namespace

const void *small_lookup(int dt, int d)
{
    switch (dt) {
    case KPP_F32:
        return reinterpret_cast<const void *>(small_fn<KPP_F32>(d));
    case KPP_BF16:
        return reinterpret_cast<const void *>(small_fn<KPP_BF16>(d));
    default:
        return reinterpret_cast<const void *>(small_fn<KPP_FP8_E4M3>(d));
    }
}

int small_threads() { return kSmallThreads; }

size_t small_smem(int64_t N, int d, int dt)
{
    return sizeof(float) * (size_t)N * ((size_t)d + 1 + (dt == KPP_FP8_E4M3 ? 1 : 0));
}

cudaError_t small_launch(const void *fn, size_t smem, const Problem &p, cudaStream_t stream)
{
    Problem pp = p;
    void *args[] = {&pp};
    return cudaLaunchKernel(fn, dim3(1), dim3(kSmallThreads), args, smem, stream);
}

} // namespace kpp

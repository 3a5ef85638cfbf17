// kpp_kmpar.cu -- k-means|| on the GPU: the oversampling initialisation of
// Bahmani et al., which the paper's introduction cites beside k-means++.
//
//   * c_0 is the first k-means++ seed; D^2 is the FP32 difference-form
//     distance to it (the seeding pass's arithmetic), phi its sum.
//   * Each round draws one Bernoulli per point, u_{r,i} < ell D^2_i / phi in
//     FP64, and appends the chosen points in increasing index (per-CTA
//     counts, one scan, an ordered compaction).  The points' nearest new
//     candidate is an N x (new candidates) x d contraction, so it runs on
//     the tensor-core assignment kernel of kpp_lloyd_assign; the exact FP32
//     difference-form distance to the candidate it picked then replaces D^2
//     when it is smaller.
//   * Every point keeps the position of its nearest candidate through the
//     rounds (a later candidate replaces it only when strictly nearer, or at
//     an equal distance with an earlier position), so the weights are one
//     histogram at the end.
//   * The weighted k-means++ recluster over the candidates is sequential in
//     K and small (a few thousand candidates): one thread-block cluster of up
//     to 16 CTAs, each holding a slice of the candidates in shared memory,
//     FP32 distances, values w_c D^2_c as FP32 two-sum pairs, a cluster-wide
//     prefix through distributed shared memory for the inverse CDF.
//
// Per-CTA sums are FP32 two-sum pairs over a fixed partition of the points,
// combined in CTA order, so a run is deterministic; FP64 appears only in the
// Bernoulli test near its boundary and in the draw decisions near a tie.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "kpp.h"
#include "kpp_device.cuh"
#include "kpp_internal.h"

namespace kpp {
namespace {

constexpr int kThreads = 256;      // per-point kernels
constexpr int kGrid = 1024;        // their CTAs; each owns a contiguous range of points
constexpr int kChunk = 4096;       // candidates per tensor-core assignment (its K limit)
constexpr int kMaxD = 128;
constexpr int kRecThreads = 1024;  // most threads per recluster CTA
// rows a warp loads before reducing, by features per lane (VEC = ceil(d/32)):
// 32 rows of one register, 16 of two, 8 of four (<= 32: lane q owns row q)
template <int VEC> __host__ __device__ constexpr int rows_in_flight()
{
    return VEC == 1 ? 32 : VEC == 2 ? 16 : 8;
}
constexpr size_t kAlign = 256;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Round state on the device (the rounds run without host round trips).
struct Scalars {
    double phi;
    long long count;   // new candidates of the current round (0 after a stop)
    long long nc;      // candidates so far
    long long base;    // position of the current round's first candidate
    long long max_new; // largest round drawn
    int32_t n_chunk;   // min(count, candidates per assignment launch)
    int32_t stop;      // the candidates outgrew their room: no further rounds
    long long pad_[26];
};
static_assert(sizeof(Scalars) == 256, "round state is 256 bytes");

struct Layout {
    int64_t range; // points per CTA
    int64_t cap;   // candidates the workspace holds
    size_t off_scal, off_d2, off_lab, off_tmp, off_flags, off_bcnt, off_boff, off_part, off_cbuf,
        off_w, off_ct, off_lloyd, lloyd_bytes, bytes;
    int64_t ldc; // leading dimension of the feature-major candidate copy
};

bool shape_ok(int64_t N, int32_t d, int64_t cap)
{
    return N >= 1 && N < (int64_t(1) << 31) && d >= 1 && d <= kMaxD && cap >= 1;
}

int lloyd_k(int64_t N) { return (int)(N < kChunk ? N : kChunk); }

Layout layout(int64_t N, int32_t d, int64_t cand_cap)
{
    Layout L;
    L.range = (N + kGrid - 1) / kGrid;
    L.cap = cand_cap < N ? cand_cap : N;
    size_t off = sizeof(Control);
    L.off_scal = off = round_up(off, kAlign);
    off += sizeof(Scalars);
    L.off_d2 = off = round_up(off, kAlign);
    off += (size_t)N * 4;
    L.off_lab = off = round_up(off, kAlign);
    off += (size_t)N * 4;
    L.off_tmp = off = round_up(off, kAlign);
    off += (size_t)N * 4;
    L.off_flags = off = round_up(off, kAlign);
    off += (size_t)N;
    L.off_bcnt = off = round_up(off, kAlign);
    off += (size_t)kGrid * 8;
    L.off_boff = off = round_up(off, kAlign);
    off += (size_t)kGrid * 8;
    L.off_part = off = round_up(off, kAlign);
    off += (size_t)kGrid * 8;
    L.off_cbuf = off = round_up(off, kAlign);
    off += (size_t)L.cap * d * 4;
    L.off_w = off = round_up(off, kAlign);
    off += (size_t)L.cap * 8;
    L.ldc = (L.cap + 31) / 32 * 32;
    L.off_ct = off = round_up(off, kAlign);
    off += (size_t)L.ldc * d * 4;
    L.off_lloyd = off = round_up(off, kAlign);
    L.lloyd_bytes = kpp_lloyd_workspace_size(N, d, lloyd_k(N));
    off += L.lloyd_bytes;
    L.bytes = round_up(off, kAlign);
    return L;
}

// ---------------------------------------------------------------------------
// Distances: a warp per row, lane j holding features j, j+32, j+64, j+96; the
// lane partials are combined by an xor butterfly, so every lane ends with
// the same FP32 value.
// ---------------------------------------------------------------------------
template <int VEC>
__device__ __forceinline__ float lane_sq(const float (&xv)[VEC], const float *c, int d, int lane)
{
    float s = 0.f;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        const int j = lane + 32 * v;
        if (j < d) {
            const float t = xv[v] - c[j];
            s = fmaf(t, t, s);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

template <int VEC>
__device__ __forceinline__ void load_row(const float *x, int64_t row, int d, int lane, bool ok,
                                         float (&xv)[VEC])
{
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        const int j = lane + 32 * v;
        xv[v] = (ok && j < d) ? __ldcs(x + row * d + j) : 0.f;
    }
}

// The CTA's sum of per-warp pair partials, combined in warp order (valid in
// thread 0).  Every lane of a warp holds the same partial.
__device__ __forceinline__ Pair cta_sum_ordered(const Pair &v, Pair *sh)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        sh[warp] = v;
    __syncthreads();
    Pair s{};
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            s.add(sh[w]);
    return s;
}

// ---------------------------------------------------------------------------
// Step 1: c_0, D^2 to it, labels 0.
// ---------------------------------------------------------------------------
template <int VEC>
__global__ void __launch_bounds__(kThreads) kmpar_init_kernel(const float *x, int64_t N, int d,
                                                              int64_t range, uint64_t seed,
                                                              uint64_t stream, float *D2,
                                                              int32_t *lab, int64_t *cand,
                                                              float *cbuf, Pair *part,
                                                              Scalars *sc)
{
    __shared__ float c[kMaxD];
    __shared__ Pair sh[kThreads / 32];
    const double u0 = philox_uniform(seed, stream, 0);
    int64_t c0 = (int64_t)floor(u0 * (double)N);
    c0 = c0 < N - 1 ? c0 : N - 1;
    for (int j = threadIdx.x; j < d; j += blockDim.x)
        c[j] = x[c0 * d + j];
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            cand[0] = c0;
            sc->nc = 1;
        }
        for (int j = threadIdx.x; j < d; j += blockDim.x)
            cbuf[j] = x[c0 * d + j];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t lo = blockIdx.x * range, hi = lo + range < N ? lo + range : N;
    constexpr int kRowsInFlight = rows_in_flight<VEC>();
    // a warp takes kRowsInFlight rows at a time; lane q keeps row q's
    // result, so the D^2 and label stores of a batch are one coalesced store
    Pair acc{};
    for (int64_t r0 = lo + (int64_t)warp * kRowsInFlight; r0 < hi; r0 += (int64_t)nw * kRowsInFlight) {
        float xv[kRowsInFlight][VEC];
#pragma unroll
        for (int q = 0; q < kRowsInFlight; ++q)
            load_row(x, r0 + q, d, lane, r0 + q < hi, xv[q]);
        float mine = 0.f;
#pragma unroll
        for (int q = 0; q < kRowsInFlight; ++q) {
            const float sq = lane_sq(xv[q], c, d, lane);
            mine = lane == q ? sq : mine;
        }
        const int64_t row = r0 + lane;
        if (lane < kRowsInFlight && row < hi) {
            D2[row] = mine;
            lab[row] = 0;
            acc.add(mine);
        }
    }
    acc = warp_pair_sum(acc);
    const Pair t = cta_sum_ordered(acc, sh);
    if (threadIdx.x == 0)
        part[blockIdx.x] = t;
}

// phi = sum of the CTA partials (one warp: lane l adds partials l*per ..
// in order, then a butterfly), FP64 only for the final hi + lo.
__global__ void kmpar_phi_kernel(const Pair *part, int n, Scalars *sc)
{
    const int lane = threadIdx.x & 31;
    const int per = (n + 31) / 32;
    Pair s{};
    for (int b = lane * per; b < n && b < (lane + 1) * per; ++b)
        s.add(part[b]);
    s = warp_pair_sum(s);
    if (lane == 0)
        sc->phi = s.value();
}

// ---------------------------------------------------------------------------
// Step 2a: round r's Bernoulli decisions and per-CTA counts.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
    kmpar_sample_kernel(const float *D2, int64_t N, int64_t range, const Scalars *sc, double ell,
                        uint64_t seed, uint64_t stream, int r, uint8_t *flags, long long *bcnt)
{
    __shared__ int wc[kThreads / 32];
    const double phi = sc->phi;
    // FP32 estimate of p = ell D^2 / phi, within a few ulps; the FP64
    // decision is taken only when u is within 2^-20 (relative, plus 2^-100
    // absolute for tiny p) of it -- GB300's FP64 divide is slow.
    const float scale = phi > 0.0 ? (float)(ell / phi) : 0.f;
    const bool fast = phi > 0.0 && scale < 1e30f && scale > 1e-30f;
    const int64_t lo = blockIdx.x * range, hi = lo + range < N ? lo + range : N;
    int n = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float d2 = D2[i];
        uint8_t f = 0;
        if (phi > 0.0 && d2 > 0.f) {
            const double u = philox_uniform_ctr(seed, stream, (uint64_t)i, (uint64_t)r + 1, 0, 0);
            const float pf = scale * d2;
            const float uf = (float)u;
            if (fast && pf < 1e30f && uf < pf * (1.f - 0x1.0p-20f) - 0x1.0p-100f)
                f = 1;
            else if (fast && pf < 1e30f && uf > pf * (1.f + 0x1.0p-20f) + 0x1.0p-100f)
                f = 0;
            else
                f = u < ell * (double)d2 / phi ? 1 : 0;
        }
        flags[i] = f;
        n += f;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1)
        n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0)
        wc[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            t += wc[w];
        bcnt[blockIdx.x] = t;
    }
}

// Step 2b: exclusive scan of the per-CTA counts (one CTA of kGrid threads).
// Also advances the round state: the round's count and first position, the
// candidates so far, and the stop (status KPP_ERR_CAPACITY) if they would
// outgrow `cap`.
__global__ void __launch_bounds__(kGrid) kmpar_scan_kernel(const long long *bcnt, long long *boff,
                                                           Scalars *sc, long long cap, int kl,
                                                           Control *ctl)
{
    __shared__ long long ws[kGrid / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long v = bcnt[t];
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += y;
    }
    if (lane == 31)
        ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long w = ws[lane];
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += y;
        }
        ws[lane] = wi - w;
        if (lane == 31) {
            long long cnt = sc->stop ? 0 : wi;
            if (cnt > 0 && sc->nc + cnt > cap) {
                sc->stop = 1;
                cnt = 0;
                atomicCAS(&ctl->status, KPP_OK, KPP_ERR_CAPACITY);
            }
            sc->count = cnt;
            sc->base = sc->nc;
            sc->nc += cnt;
            sc->n_chunk = (int32_t)(cnt < kl ? cnt : kl);
            if (wi > sc->max_new)
                sc->max_new = wi;
        }
    }
    __syncthreads();
    boff[t] = ws[warp] + inc - v;
}

// Step 2c: ordered compaction.  The round's candidates go to positions
// base + (chosen points before them) (base and count from the round state);
// each takes D^2 = 0 and its own position as nearest candidate (a point is
// at distance 0 from itself).
__global__ void __launch_bounds__(kThreads)
    kmpar_compact_kernel(const float *x, int64_t N, int d, int64_t range, const uint8_t *flags,
                         const long long *boff, const Scalars *sc, int64_t *cand, float *cbuf,
                         float *D2, int32_t *lab)
{
    __shared__ int wc[kThreads / 32 + 1];
    if (sc->count == 0)
        return;
    const int64_t base = sc->base;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const int64_t lo = blockIdx.x * range, hi = lo + range < N ? lo + range : N;
    int64_t pos0 = base + boff[blockIdx.x];
    for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int64_t i = t0 + t;
        const bool f = i < hi && flags[i];
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0)
            wc[warp] = __popc(m);
        __syncthreads();
        if (t == 0) {
            int s = 0;
            for (int w = 0; w < nw; ++w) {
                const int c = wc[w];
                wc[w] = s;
                s += c;
            }
            wc[nw] = s;
        }
        __syncthreads();
        if (f) {
            const int64_t pos = pos0 + wc[warp] + __popc(m & ((1u << lane) - 1u));
            cand[pos] = i;
            for (int j = 0; j < d; ++j)
                cbuf[pos * d + j] = x[i * d + j];
            D2[i] = 0.f;
            lab[i] = (int32_t)pos;
        }
        pos0 += wc[nw];
        __syncthreads();
    }
}

// Step 2d: D^2 = min(D^2, exact distance to the candidate the tensor-core
// assignment picked among cbuf[base .. base + n)); a tie goes to the earlier
// position.  Writes the CTA's sum of the resulting D^2 (an FP32 pair).
template <int VEC>
__global__ void __launch_bounds__(kThreads)
    kmpar_min_update_kernel(const float *x, int64_t N, int d, int64_t range, const float *cbuf,
                            const Scalars *sc, int64_t c0, int kl, const int32_t *pick, float *D2,
                            int32_t *lab, Pair *part)
{
    __shared__ Pair sh[kThreads / 32];
    // chunk c0 of the round: candidates base + c0 .. base + c0 + n - 1
    const long long left = sc->count - c0;
    const int32_t n = (int32_t)(left < kl ? left : kl);
    if (n <= 0)
        return; // D^2 unchanged: the CTA partials of the last update stand
    const int64_t base = sc->base + c0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t lo = blockIdx.x * range, hi = lo + range < N ? lo + range : N;
    constexpr int kRowsInFlight = rows_in_flight<VEC>();
    Pair acc{};
    for (int64_t r0 = lo + (int64_t)warp * kRowsInFlight; r0 < hi; r0 += (int64_t)nw * kRowsInFlight) {
        // lane q < kRowsInFlight loads row q's label, D^2 and nearest so far
        const int64_t row = r0 + lane;
        const bool own = lane < kRowsInFlight && row < hi;
        // (a label outside the chunk -- only possible if the assignment gave
        // up on a timeout, which the host reports -- reads position base)
        int32_t pk = own ? pick[row] : 0;
        pk = (unsigned)pk < (unsigned)n ? pk : 0;
        float cur = own ? D2[row] : 0.f;
        const int32_t l = own ? lab[row] : 0;
        float xv[kRowsInFlight][VEC];
#pragma unroll
        for (int q = 0; q < kRowsInFlight; ++q)
            load_row(x, r0 + q, d, lane, r0 + q < hi, xv[q]);
        float mine = 0.f;
#pragma unroll
        for (int q = 0; q < kRowsInFlight; ++q) {
            const int32_t pq = __shfl_sync(0xffffffffu, pk, q);
            const float sq = lane_sq(xv[q], cbuf + (base + pq) * d, d, lane);
            mine = lane == q ? sq : mine;
        }
        if (own) {
            const int64_t pos = base + pk;
            if (mine < cur || (mine == cur && pos < l)) {
                cur = mine;
                D2[row] = mine;
                lab[row] = (int32_t)pos;
            }
            acc.add(cur);
        }
    }
    acc = warp_pair_sum(acc);
    const Pair t = cta_sum_ordered(acc, sh);
    if (threadIdx.x == 0)
        part[blockIdx.x] = t;
}

// Step 3: weights = histogram of the nearest-candidate positions.
__global__ void kmpar_weights_kernel(const int32_t *lab, int64_t N, unsigned long long *w)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&w[lab[i]], 1ull);
}

__global__ void kmpar_weights_out_kernel(const unsigned long long *w, int64_t n, int64_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)w[i];
}

// ---------------------------------------------------------------------------
// Step 4: weighted k-means++ over the nc candidates, on one thread-block
// cluster (up to 16 CTAs, one per SM, so the per-step work spreads over that
// many SMs).  CTA r owns the contiguous slice [r S, r S + S) of the
// candidate list, thread t of it the contiguous run [t R, t R + R) of the
// slice; coordinates (feature-major), D^2 and the weights of the slice stay
// in shared memory.  Per centre m:
//   1. every thread updates D^2 of its run to the last centre (FP32
//      difference form, features in order), forms v = w D^2 as an FP32
//      two-sum pair (w split into two floats, products with their exact
//      FMA error terms), sums its run in order and publishes the sum; each
//      warp publishes its total;
//   2. after a cluster barrier, warp c of every CTA sums CTA c's warp totals
//      read from distributed shared memory, and warp 0 prefixes the CTA
//      totals in rank order; every CTA does the same arithmetic on the same
//      values, so all agree on T, on the threshold t = v_m T and on the CTA
//      whose prefix first exceeds t;
//   3. warp 0 of that CTA narrows the crossing to a warp, a thread and an
//      element of its run (decisions in FP32 pairs, exactly in FP64 when
//      within 2^-40 t; at any level where rounding leaves no crossing, the
//      last element with a positive value -- the clamp of the inverse CDF)
//      and writes the new centre's coordinates into every CTA's shared
//      memory; a second cluster barrier completes the step.
// A step synchronises at two cluster barriers and one CTA barrier.  The draws are computed
// 32 at a time, one per lane of warp 0, ahead of the steps that use them.
// T = 0 at a draw (fewer than K candidates carry weight) is a degenerate
// stop: the remaining indices are -1.
// ---------------------------------------------------------------------------
constexpr int kRecMaxCluster = 16;
constexpr int kRecPerCta = 512; // target candidates per CTA

struct RecArgs {
    const float *cT; // [d][ldc] candidate coordinates, feature-major
    int64_t ldc;
    const float *cbuf; // [nc][d]
    int64_t nc;
    int32_t d;
    int32_t K;
    int64_t slice;  // candidates per CTA
    int64_t run;    // candidates per thread
    int32_t staged; // the slice's coordinates are copied to shared memory
    const unsigned long long *w;
    uint64_t seed, stream;
    const int64_t *cand;
    int64_t *idx_out;
    Control *ctl;
};

// w * r as a pair: w = whi + wlo (two floats, exact for w < 2^48), each
// product with its exact FMA error term.
__device__ __forceinline__ Pair weighted(float whi, float wlo, float r)
{
    const float p1 = __fmul_rn(whi, r);
    const float e1 = __fmaf_rn(whi, r, -p1);
    const float p2 = __fmul_rn(wlo, r);
    const float e2 = __fmaf_rn(wlo, r, -p2);
    Pair v{p1, e1};
    v.add(p2);
    v.lo = __fadd_rn(v.lo, e2);
    return v;
}

// Over n <= 32 lanes holding values v (lanes at or past n hold zero): the
// first lane whose running prefix base + v_0 + .. + v_l exceeds the threshold
// (-1 if none), the last lane with a positive value (-1 if none), and the
// prefix before the lane taken (the first, else the last).  Every lane
// returns the same.
__device__ __forceinline__ void lane_cross(const Pair &v, const Pair &base, const Thresh &th,
                                           int &first, int &last, Pair &before)
{
    Pair ex;
    const Pair inc = warp_pair_scan(v, ex);
    Pair P = base;
    P.add(inc);
    const bool pos = v.hi > 0.f;
    const unsigned cm = __ballot_sync(0xffffffffu, pos && th.gt(P));
    const unsigned pm = __ballot_sync(0xffffffffu, pos);
    first = cm ? __ffs(cm) - 1 : -1;
    last = pm ? 31 - __clz(pm) : -1;
    const int sel = first >= 0 ? first : (last >= 0 ? last : 0);
    Pair B = base;
    B.add(ex);
    before = shfl_pair(B, sel);
}

__global__ void __launch_bounds__(kRecThreads, 1) kmpar_recluster_kernel(RecArgs a)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int C = (int)cl.num_blocks();
    // [slice] D^2, [slice] w hi, [slice] w lo, then (staged) [d][slice]
    // coordinates
    extern __shared__ float rsm[];
    float *s_rd2 = rsm, *s_whi = rsm + a.slice, *s_wlo = rsm + 2 * a.slice;
    float *s_x = rsm + 3 * a.slice;
    __shared__ float cen[kMaxD];
    __shared__ Pair s_seg[kRecThreads];     // each thread's run sum
    __shared__ Pair s_wt[kRecThreads / 32]; // each warp's total
    __shared__ Pair s_ct[kRecMaxCluster];   // each CTA's total
    __shared__ int s_stop;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const int64_t lo = (int64_t)rank * a.slice;
    const int64_t hi = lo + a.slice < a.nc ? lo + a.slice : a.nc;
    const int64_t r0 = lo + (int64_t)t * a.run < hi ? lo + (int64_t)t * a.run : hi;
    const int64_t r1 = r0 + a.run < hi ? r0 + a.run : hi;
    for (int64_t c = lo + t; c < hi; c += blockDim.x) {
        const unsigned long long wv = a.w[c];
        const float wh = __ull2float_rn(wv);
        s_whi[c - lo] = wh;
        s_wlo[c - lo] = (float)((long long)wv - (long long)wh);
    }
    if (a.staged)
        for (int j = 0; j < a.d; ++j)
            for (int64_t c = lo + t; c < hi; c += blockDim.x)
                s_x[(int64_t)j * a.slice + (c - lo)] = a.cT[(int64_t)j * a.ldc + c];
    if (t == 0)
        s_stop = 0;
    __syncthreads();
    double udraw = 0.0; // warp 0: lane l holds the draw of step 32 q + l
    for (int m = 0; m < a.K; ++m) {
        if (warp == 0 && (m & 31) == 0)
            udraw = m + lane < a.K
                        ? philox_uniform_ctr(a.seed, a.stream, (uint64_t)(m + lane), 0, 1, 0)
                        : 0.0;
        // 1. this thread's run: D^2 to the last centre, values, their sum
        Pair seg{};
        for (int64_t c = r0; c < r1; ++c) {
            const int li = (int)(c - lo);
            Pair v;
            if (m == 0) {
                s_rd2[li] = __int_as_float(0x7f800000);
                v = Pair{s_whi[li], s_wlo[li]};
            } else {
                float s = 0.f;
                if (a.staged) {
#pragma unroll 8
                    for (int j = 0; j < a.d; ++j) {
                        const float q = s_x[(int64_t)j * a.slice + li] - cen[j];
                        s = fmaf(q, q, s);
                    }
                } else {
#pragma unroll 8
                    for (int j = 0; j < a.d; ++j) {
                        const float q = __ldg(a.cT + (int64_t)j * a.ldc + c) - cen[j];
                        s = fmaf(q, q, s);
                    }
                }
                float r = s_rd2[li];
                if (s < r) {
                    r = s;
                    s_rd2[li] = s;
                }
                v = weighted(s_whi[li], s_wlo[li], r);
            }
            seg.add(v);
        }
        s_seg[t] = seg;
        const Pair wtot = warp_pair_sum(seg);
        if (lane == 0)
            s_wt[warp] = wtot;
        cl.sync(); // every thread's and warp's sum is published
        // 2. warp c sums CTA c's warp totals (one remote load per lane); warp
        // 0 then prefixes the CTA totals in rank order
        for (int c = warp; c < C; c += nw) {
            const Pair *rw = cl.map_shared_rank(s_wt, (unsigned)c);
            const Pair v = warp_pair_sum(lane < nw ? rw[lane] : Pair{});
            if (lane == 0)
                s_ct[c] = v;
        }
        __syncthreads();
        if (warp == 0) {
            const Pair ct = lane < C ? s_ct[lane] : Pair{};
            Pair cex;
            const Pair cinc = warp_pair_scan(ct, cex);
            const Pair T = shfl_pair(cinc, 31);
            Thresh th = thresh_for_u(__shfl_sync(0xffffffffu, udraw, m & 31));
            thresh_set_total(th, T);
            if (!(T.hi > 0.f)) {
                // degenerate stop
                if (rank == 0) {
                    if (lane == 0)
                        atomicCAS(&a.ctl->status, KPP_OK, KPP_ERR_DEGENERATE);
                    for (int k = m + lane; k < a.K; k += 32)
                        a.idx_out[k] = -1;
                }
                if (lane == 0)
                    s_stop = 1;
            } else {
                const unsigned cm = __ballot_sync(0xffffffffu, ct.hi > 0.f && th.gt(cinc));
                const unsigned pm = __ballot_sync(0xffffffffu, ct.hi > 0.f);
                const int des = cm ? __ffs(cm) - 1 : 31 - __clz(pm);
                bool clamp = cm == 0;
                if (rank == des) {
                    // 3. narrow the crossing to a warp, a thread, an element
                    const Pair base = shfl_pair(cex, des);
                    int f, l;
                    Pair before;
                    lane_cross(lane < nw ? s_wt[lane] : Pair{}, base, th, f, l, before);
                    const int ws = !clamp && f >= 0 ? f : l;
                    clamp = clamp || f < 0;
                    lane_cross(s_seg[ws * 32 + lane], before, th, f, l, before);
                    const int tt = ws * 32 + (!clamp && f >= 0 ? f : l);
                    clamp = clamp || f < 0;
                    const int64_t e0 = lo + (int64_t)tt * a.run < hi ? lo + (int64_t)tt * a.run : hi;
                    const int64_t e1 = e0 + a.run < hi ? e0 + a.run : hi;
                    long long pick = -1;
                    if (lane == 0) {
                        Pair P = before;
                        long long lastp = -1;
                        for (int64_t c = e0; c < e1; ++c) {
                            const int li = (int)(c - lo);
                            const Pair v = m == 0 ? Pair{s_whi[li], s_wlo[li]}
                                                  : weighted(s_whi[li], s_wlo[li], s_rd2[li]);
                            if (!(v.hi > 0.f))
                                continue;
                            lastp = c;
                            P.add(v);
                            if (!clamp && th.gt(P)) {
                                pick = c;
                                break;
                            }
                        }
                        if (pick < 0)
                            pick = lastp;
                    }
                    pick = __shfl_sync(0xffffffffu, pick, 0);
                    // 4. the new centre into every CTA's shared memory
                    for (int j = lane; j < a.d; j += 32) {
                        const float v = a.staged ? s_x[(int64_t)j * a.slice + (pick - lo)]
                                                 : a.cbuf[pick * a.d + j];
                        for (int r = 0; r < C; ++r)
                            *cl.map_shared_rank(&cen[j], (unsigned)r) = v;
                    }
                    if (lane == 0)
                        a.idx_out[m] = a.cand[pick];
                }
            }
        }
        cl.sync(); // the new centre is in place everywhere
        if (s_stop)
            break;
    }
    cl.sync(); // no CTA leaves while another may still read its shared memory
}

// cT[j][c] = cbuf[c][j]
__global__ void kmpar_transpose_kernel(const float *cbuf, int64_t nc, int d, int64_t ldc, float *cT)
{
    const int64_t n = nc * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / d;
        const int j = (int)(e - c * d);
        cT[(int64_t)j * ldc + c] = cbuf[e];
    }
}

// Cluster shape of the recluster: C CTAs of T threads, S candidates per CTA,
// R per thread; false if the candidates do not fit.
struct RecShape {
    int C, T;
    int64_t S, R;
    bool staged;
    size_t smem;
};

bool rec_shape(int64_t nc, int d, int max_cluster, RecShape *out)
{
    RecShape r;
    r.C = (int)((nc + kRecPerCta - 1) / kRecPerCta);
    r.C = r.C < 1 ? 1 : (r.C > max_cluster ? max_cluster : r.C);
    r.S = (nc + r.C - 1) / r.C;
    r.T = (int)((r.S + 31) / 32 * 32);
    r.T = r.T > kRecThreads ? kRecThreads : r.T;
    r.R = (r.S + r.T - 1) / r.T;
    r.staged = (size_t)r.S * (12 + 4 * (size_t)d) <= 200 * 1024;
    r.smem = (size_t)r.S * (r.staged ? 12 + 4 * (size_t)d : 12);
    *out = r;
    return r.smem <= 200 * 1024;
}

// Largest cluster (16 if the device schedules it, else 8) for this kernel.
int rec_max_cluster()
{
    static int cached = 0;
    if (cached)
        return cached;
    int best = 8;
    if (cudaFuncSetAttribute(kmpar_recluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) == cudaSuccess &&
        cudaFuncSetAttribute(kmpar_recluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kRecMaxCluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(kRecMaxCluster);
        cfg.blockDim = dim3(kRecThreads);
        cfg.dynamicSmemBytes = 200 * 1024;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kmpar_recluster_kernel, &cfg) == cudaSuccess &&
            n >= 1)
            best = kRecMaxCluster;
    }
    cudaGetLastError();
    cached = best;
    return best;
}

cudaError_t rec_launch(const RecShape &r, const RecArgs &a, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(kmpar_recluster_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r.smem);
    if (e != cudaSuccess)
        return e;
    if (r.C > 8 && (e = cudaFuncSetAttribute(kmpar_recluster_kernel,
                                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                       cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)r.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)r.C);
    cfg.blockDim = dim3((unsigned)r.T);
    cfg.dynamicSmemBytes = r.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kmpar_recluster_kernel, a);
}

int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

} // namespace
} // namespace kpp

using namespace kpp;

extern "C" {

size_t kpp_kmeans_par_workspace_size(int64_t N, int32_t d, int64_t cand_cap)
{
    if (!shape_ok(N, d, cand_cap))
        return 0;
    const Layout L = layout(N, d, cand_cap);
    return L.lloyd_bytes ? L.bytes : 0;
}

kpp_status kpp_kmeans_par(const float *points, int64_t N, int32_t d, int32_t K, double ell,
                          int32_t rounds, uint64_t seed, uint64_t stream_id, int64_t cand_cap,
                          int64_t *idx_out, int64_t *cand_out, int64_t *n_cand_out,
                          int64_t *weights_out, int32_t *labels_out, float *d2_out,
                          double *phi_out, void *workspace, size_t workspace_bytes,
                          kpp_stream_t stream)
{
    if (!points || !idx_out || !cand_out || !n_cand_out || !shape_ok(N, d, cand_cap) || K < 1 ||
        K > N || rounds < 0 || !(ell > 0.0) || !(ell < 1e300))
        return KPP_ERR_INVALID_ARG;
    *n_cand_out = 0;
    const Layout L = layout(N, d, cand_cap);
    if (!L.lloyd_bytes || !workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 ||
        workspace_bytes < L.bytes)
        return KPP_ERR_WORKSPACE;
    char *ws = reinterpret_cast<char *>(workspace);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (sm_count() <= 0)
        return KPP_ERR_CUDA;
    Control *ctl = reinterpret_cast<Control *>(ws);
    Scalars *sc = reinterpret_cast<Scalars *>(ws + L.off_scal);
    float *D2 = reinterpret_cast<float *>(ws + L.off_d2);
    int32_t *lab = reinterpret_cast<int32_t *>(ws + L.off_lab);
    int32_t *pick = reinterpret_cast<int32_t *>(ws + L.off_tmp);
    uint8_t *flags = reinterpret_cast<uint8_t *>(ws + L.off_flags);
    long long *bcnt = reinterpret_cast<long long *>(ws + L.off_bcnt);
    long long *boff = reinterpret_cast<long long *>(ws + L.off_boff);
    Pair *part = reinterpret_cast<Pair *>(ws + L.off_part);
    float *cbuf = reinterpret_cast<float *>(ws + L.off_cbuf);
    auto *wts = reinterpret_cast<unsigned long long *>(ws + L.off_w);
    float *cT = reinterpret_cast<float *>(ws + L.off_ct);
    void *lws = ws + L.off_lloyd;
    const int kl = lloyd_k(N);
    auto launched = [] { return cudaGetLastError() == cudaSuccess; };

    auto init_fn = d <= 32 ? &kmpar_init_kernel<1> : d <= 64 ? &kmpar_init_kernel<2>
                                                             : &kmpar_init_kernel<4>;
    auto update_fn = d <= 32 ? &kmpar_min_update_kernel<1>
                             : d <= 64 ? &kmpar_min_update_kernel<2> : &kmpar_min_update_kernel<4>;
    kpp_status st = kpp_lloyd_prepare(points, N, d, kl, lws, L.lloyd_bytes, stream);
    if (st != KPP_OK)
        return st;
    // c_0, D^2 to it and phi, with both status words (this call's and the
    // assignment's) and the round state cleared
    auto start = [&]() -> kpp_status {
        if (cudaMemsetAsync(ws, 0, sizeof(Control), s) != cudaSuccess ||
            cudaMemsetAsync(lws, 0, sizeof(Control), s) != cudaSuccess ||
            cudaMemsetAsync(sc, 0, sizeof(Scalars), s) != cudaSuccess)
            return KPP_ERR_CUDA;
        init_fn<<<kGrid, kThreads, 0, s>>>(points, N, d, L.range, seed, stream_id, D2, lab,
                                           cand_out, cbuf, part, sc);
        kmpar_phi_kernel<<<1, 32, 0, s>>>(part, kGrid, sc);
        return launched() ? KPP_OK : KPP_ERR_LAUNCH;
    };
    auto draw = [&](int r) {
        kmpar_sample_kernel<<<kGrid, kThreads, 0, s>>>(D2, N, L.range, sc, ell, seed, stream_id, r,
                                                       flags, bcnt);
        kmpar_scan_kernel<<<1, kGrid, 0, s>>>(bcnt, boff, sc, L.cap, kl, ctl);
        kmpar_compact_kernel<<<kGrid, kThreads, 0, s>>>(points, N, d, L.range, flags, boff, sc,
                                                        cand_out, cbuf, D2, lab);
    };
    Scalars hs;
    auto read_state = [&]() -> bool {
        return cudaMemcpyAsync(&hs, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s) ==
                   cudaSuccess &&
               cudaStreamSynchronize(s) == cudaSuccess;
    };

    // The rounds with their state on the device and no host round trip: each
    // round's first kl new candidates are searched (the count is read by the
    // kernels).  If a round drew more than kl, the rounds run again below with
    // the count read on the host each round and one search per kl chunk.
    if ((st = start()) != KPP_OK)
        return st;
    for (int r = 0; r < rounds; ++r) {
        draw(r);
        st = lloyd_assign_device_count(cbuf, &sc->base, &sc->n_chunk, kl, N, d, pick, lws,
                                       L.lloyd_bytes, s);
        if (st != KPP_OK)
            return st;
        update_fn<<<kGrid, kThreads, 0, s>>>(points, N, d, L.range, cbuf, sc, 0, kl, pick, D2, lab,
                                             part);
        kmpar_phi_kernel<<<1, 32, 0, s>>>(part, kGrid, sc);
        if (!launched())
            return KPP_ERR_LAUNCH;
    }
    if (!read_state())
        return KPP_ERR_CUDA;
    if (hs.max_new > kl) {
        if ((st = start()) != KPP_OK)
            return st;
        for (int r = 0; r < rounds; ++r) {
            draw(r);
            if (!launched() || !read_state())
                return KPP_ERR_CUDA;
            if (hs.stop)
                break;
            for (int64_t c0 = 0; c0 < hs.count; c0 += kl) {
                const int kc = (int)(hs.count - c0 < kl ? hs.count - c0 : kl);
                st = kpp_lloyd_assign(cbuf + (hs.base + c0) * d, N, d, kc, pick, lws,
                                      L.lloyd_bytes, stream);
                if (st != KPP_OK)
                    return st;
                update_fn<<<kGrid, kThreads, 0, s>>>(points, N, d, L.range, cbuf, sc, c0, kl, pick,
                                                     D2, lab, part);
            }
            kmpar_phi_kernel<<<1, 32, 0, s>>>(part, kGrid, sc);
            if (!launched())
                return KPP_ERR_LAUNCH;
        }
        if (!read_state())
            return KPP_ERR_CUDA;
    }
    const int64_t nc = hs.nc;
    if (hs.stop) {
        *n_cand_out = nc;
        return KPP_ERR_CAPACITY;
    }
    *n_cand_out = nc;
    if (cudaMemsetAsync(wts, 0, (size_t)nc * 8, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    kmpar_weights_kernel<<<kGrid, kThreads, 0, s>>>(lab, N, wts);
    RecShape rs;
    if (!rec_shape(nc, d, rec_max_cluster(), &rs))
        return KPP_ERR_UNSUPPORTED;
    kmpar_transpose_kernel<<<(int)((nc * d + 255) / 256 < 4096 ? (nc * d + 255) / 256 : 4096), 256,
                             0, s>>>(cbuf, nc, d, L.ldc, cT);
    RecArgs ra;
    ra.cT = cT;
    ra.ldc = L.ldc;
    ra.cbuf = cbuf;
    ra.nc = nc;
    ra.d = d;
    ra.K = K;
    ra.slice = rs.S;
    ra.run = rs.R;
    ra.staged = rs.staged ? 1 : 0;
    ra.w = wts;
    ra.seed = seed;
    ra.stream = stream_id;
    ra.cand = cand_out;
    ra.idx_out = idx_out;
    ra.ctl = ctl;
    if (rec_launch(rs, ra, s) != cudaSuccess)
        return KPP_ERR_LAUNCH;
    if (weights_out)
        kmpar_weights_out_kernel<<<(int)((nc + 255) / 256), 256, 0, s>>>(wts, nc, weights_out);
    if (!launched())
        return KPP_ERR_LAUNCH;
    if ((labels_out && cudaMemcpyAsync(labels_out, lab, (size_t)N * 4, cudaMemcpyDeviceToDevice,
                                       s) != cudaSuccess) ||
        (d2_out &&
         cudaMemcpyAsync(d2_out, D2, (size_t)N * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) ||
        (phi_out && cudaMemcpyAsync(phi_out, &sc->phi, sizeof(double), cudaMemcpyDeviceToDevice,
                                    s) != cudaSuccess))
        return KPP_ERR_CUDA;
    int32_t status[2] = {0, 0};
    if (cudaMemcpyAsync(&status[0], &ctl->status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&status[1], lws, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (status[1] != KPP_OK)
        return (kpp_status)status[1];
    return (kpp_status)status[0];
}

} // extern "C"

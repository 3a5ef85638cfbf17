// kpp_kmpar.cu -- k-means|| on the GPU: the oversampling initialisation of
// Bahmani et al., which the paper's introduction cites beside k-means++.
//
//   * c_0 is the first k-means++ seed; D^2 is the FP32 difference-form
//     distance to it (the seeding pass's arithmetic), phi its FP64 sum.
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
//     K and small (a few thousand candidates): one CTA of 1024 threads, each
//     owning a contiguous run of candidates, FP32 distances, FP64 values
//     w_c D^2_c, a block scan for the inverse CDF.
//
// Per-CTA sums are FP64 over a fixed partition of the points and combined in
// CTA order, so a run is deterministic.
#include <cuda_runtime.h>

#include <cstring>

#include "kpp.h"
#include "kpp_device.cuh"

namespace kpp {
namespace {

constexpr int kThreads = 256;      // per-point kernels
constexpr int kGrid = 1024;        // their CTAs; each owns a contiguous range of points
constexpr int kChunk = 4096;       // candidates per tensor-core assignment (its K limit)
constexpr int kMaxD = 128;
constexpr int kRecThreads = 1024;  // recluster CTA
constexpr int kRowsInFlight = 4;   // rows a warp loads before reducing
constexpr size_t kAlign = 256;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Scalars {
    double phi;
    long long count; // new candidates of the current round
    long long pad_[30];
};

struct Layout {
    int64_t range; // points per CTA
    int64_t cap;   // candidates the workspace holds
    size_t off_scal, off_d2, off_lab, off_tmp, off_flags, off_bcnt, off_boff, off_part, off_cbuf,
        off_w, off_rd2, off_rval, off_lloyd, lloyd_bytes, bytes;
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
    L.off_rd2 = off = round_up(off, kAlign);
    off += (size_t)L.cap * 4;
    L.off_rval = off = round_up(off, kAlign);
    off += (size_t)L.cap * 8;
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
__device__ __forceinline__ float lane_sq(const float (&xv)[4], const float *c, int d, int lane)
{
    float s = 0.f;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
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

__device__ __forceinline__ void load_row(const float *x, int64_t row, int d, int lane, bool ok,
                                         float (&xv)[4])
{
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int j = lane + 32 * v;
        xv[v] = (ok && j < d) ? __ldcs(x + row * d + j) : 0.f;
    }
}

// The CTA's FP64 sum of per-warp FP64 partials, combined in warp order.
__device__ __forceinline__ double cta_sum_ordered(double v, double *sh)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            s += sh[w];
    return s;
}

// ---------------------------------------------------------------------------
// Step 1: c_0, D^2 to it, labels 0.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) kmpar_init_kernel(const float *x, int64_t N, int d,
                                                              int64_t range, uint64_t seed,
                                                              uint64_t stream, float *D2,
                                                              int32_t *lab, int64_t *cand,
                                                              float *cbuf, double *part)
{
    __shared__ float c[kMaxD];
    __shared__ double sh[kThreads / 32];
    const double u0 = philox_uniform(seed, stream, 0);
    int64_t c0 = (int64_t)floor(u0 * (double)N);
    c0 = c0 < N - 1 ? c0 : N - 1;
    for (int j = threadIdx.x; j < d; j += blockDim.x)
        c[j] = x[c0 * d + j];
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0)
            cand[0] = c0;
        for (int j = threadIdx.x; j < d; j += blockDim.x)
            cbuf[j] = x[c0 * d + j];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t lo = blockIdx.x * range, hi = lo + range < N ? lo + range : N;
    double acc = 0.0;
    for (int64_t r0 = lo + (int64_t)warp * kRowsInFlight; r0 < hi; r0 += (int64_t)nw * kRowsInFlight) {
        float xv[kRowsInFlight][4];
#pragma unroll
        for (int q = 0; q < kRowsInFlight; ++q)
            load_row(x, r0 + q, d, lane, r0 + q < hi, xv[q]);
#pragma unroll
        for (int q = 0; q < kRowsInFlight; ++q) {
            const int64_t row = r0 + q;
            const float s = lane_sq(xv[q], c, d, lane);
            if (row < hi) {
                if (lane == 0) {
                    D2[row] = s;
                    lab[row] = 0;
                }
                acc += (double)s;
            }
        }
    }
    const double t = cta_sum_ordered(acc, sh);
    if (threadIdx.x == 0)
        part[blockIdx.x] = t;
}

// phi = sum of the CTA partials in CTA order
__global__ void kmpar_phi_kernel(const double *part, int n, Scalars *sc)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < n; ++b)
            s += part[b];
        sc->phi = s;
    }
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
    const int64_t lo = blockIdx.x * range, hi = lo + range < N ? lo + range : N;
    int n = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double p = phi > 0.0 ? ell * (double)D2[i] / phi : 0.0;
        const double u = philox_uniform_ctr(seed, stream, (uint64_t)i, (uint64_t)r + 1, 0, 0);
        const uint8_t f = u < p ? 1 : 0;
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
__global__ void __launch_bounds__(kGrid) kmpar_scan_kernel(const long long *bcnt, long long *boff,
                                                           Scalars *sc)
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
        if (lane == 31)
            sc->count = wi;
    }
    __syncthreads();
    boff[t] = ws[warp] + inc - v;
}

// Step 2c: ordered compaction.  The round's candidates go to positions
// base + (chosen points before them); each takes D^2 = 0 and its own
// position as nearest candidate (a point is at distance 0 from itself).
__global__ void __launch_bounds__(kThreads)
    kmpar_compact_kernel(const float *x, int64_t N, int d, int64_t range, const uint8_t *flags,
                         const long long *boff, int64_t base, int64_t *cand, float *cbuf,
                         float *D2, int32_t *lab)
{
    __shared__ int wc[kThreads / 32 + 1];
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
// position.  Writes the CTA's FP64 sum of the resulting D^2.
__global__ void __launch_bounds__(kThreads)
    kmpar_min_update_kernel(const float *x, int64_t N, int d, int64_t range, const float *cbuf,
                            int64_t base, int32_t n, const int32_t *pick, float *D2, int32_t *lab,
                            double *part)
{
    __shared__ double sh[kThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t lo = blockIdx.x * range, hi = lo + range < N ? lo + range : N;
    double acc = 0.0;
    for (int64_t r0 = lo + (int64_t)warp * kRowsInFlight; r0 < hi; r0 += (int64_t)nw * kRowsInFlight) {
        float xv[kRowsInFlight][4];
        int64_t pos[kRowsInFlight];
#pragma unroll
        for (int q = 0; q < kRowsInFlight; ++q) {
            const bool ok = r0 + q < hi;
            load_row(x, r0 + q, d, lane, ok, xv[q]);
            // (a label outside the chunk -- only possible if the assignment
            // gave up on a timeout, which the host reports -- reads row 0)
            const int32_t pk = ok ? pick[r0 + q] : 0;
            pos[q] = base + ((unsigned)pk < (unsigned)n ? pk : 0);
        }
#pragma unroll
        for (int q = 0; q < kRowsInFlight; ++q) {
            const int64_t row = r0 + q;
            const float s = lane_sq(xv[q], cbuf + pos[q] * d, d, lane);
            if (row < hi) {
                float cur = D2[row];
                const int32_t l = lab[row];
                if (s < cur || (s == cur && pos[q] < l)) {
                    cur = s;
                    if (lane == 0) {
                        D2[row] = s;
                        lab[row] = (int32_t)pos[q];
                    }
                }
                acc += (double)cur;
            }
        }
    }
    const double t = cta_sum_ordered(acc, sh);
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
// Step 4: weighted k-means++ over the nc candidates, one CTA.  Thread t owns
// candidates [t S, t S + S); per centre m it updates their D^2 to the last
// centre (FP32 difference form) and values w D^2 (FP64), sums them in order,
// and a block scan gives every thread the FP64 prefix before its run.  The
// pick is the earliest candidate whose running prefix exceeds t = v_m T (the
// last candidate with a positive value if rounding leaves none).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_incl_scan(double v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += y;
    }
    return v;
}

__global__ void __launch_bounds__(kRecThreads, 1)
    kmpar_recluster_kernel(const float *cbuf, int64_t nc, int d, const unsigned long long *w,
                           int K, uint64_t seed, uint64_t stream, const int64_t *cand, float *rd2,
                           double *rval, int64_t *idx_out, Control *ctl)
{
    __shared__ float cen[kMaxD];
    __shared__ double wsum[kRecThreads / 32], wex[kRecThreads / 32];
    __shared__ double s_T;
    __shared__ unsigned long long s_pick;
    __shared__ long long s_last;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t S = (nc + kRecThreads - 1) / kRecThreads;
    const int64_t c_lo = (int64_t)t * S < nc ? (int64_t)t * S : nc;
    const int64_t c_hi = c_lo + S < nc ? c_lo + S : nc;
    for (int m = 0; m < K; ++m) {
        // this thread's run: D^2 to the last centre, values, their sum in order
        double seg = 0.0;
        long long last = -1;
        for (int64_t c = c_lo; c < c_hi; ++c) {
            double v;
            if (m == 0) {
                rd2[c] = __int_as_float(0x7f800000);
                v = (double)w[c];
            } else {
                float s = 0.f;
                for (int j = 0; j < d; ++j) {
                    const float q = cbuf[c * d + j] - cen[j];
                    s = fmaf(q, q, s);
                }
                float cur = rd2[c];
                if (s < cur) {
                    cur = s;
                    rd2[c] = s;
                }
                v = (double)w[c] * (double)cur;
            }
            rval[c] = v;
            seg += v;
            if (v > 0.0)
                last = (long long)c;
        }
        // block scan of the run sums: in-warp, then over the warp totals
        const double inc = warp_incl_scan(seg);
        double ex = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0)
            ex = 0.0;
        if (lane == 31)
            wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const double wi = warp_incl_scan(wsum[lane]);
            double we = __shfl_up_sync(0xffffffffu, wi, 1);
            wex[lane] = lane == 0 ? 0.0 : we;
            if (lane == 31)
                s_T = wi;
            if (lane == 0) {
                s_pick = ~0ull;
                s_last = -1;
            }
        }
        __syncthreads();
        const double T = s_T;
        if (!(T > 0.0)) {
            // fewer than K candidates carry weight: degenerate stop
            if (t == 0)
                atomicCAS(&ctl->status, KPP_OK, KPP_ERR_DEGENERATE);
            for (int k = m + t; k < K; k += blockDim.x)
                idx_out[k] = -1;
            return;
        }
        const double th = philox_uniform_ctr(seed, stream, (uint64_t)m, 0, 1, 0) * T;
        double P = wex[warp] + ex;
        for (int64_t c = c_lo; c < c_hi; ++c) {
            P += rval[c];
            if (P > th) {
                atomicMin(&s_pick, (unsigned long long)c);
                break;
            }
        }
        if (last >= 0)
            atomicMax(&s_last, last);
        __syncthreads();
        const int64_t pick = s_pick != ~0ull ? (int64_t)s_pick : (int64_t)s_last;
        if (t < d)
            cen[t] = cbuf[pick * d + t];
        if (t == 0)
            idx_out[m] = cand[pick];
        __syncthreads();
    }
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
    double *part = reinterpret_cast<double *>(ws + L.off_part);
    float *cbuf = reinterpret_cast<float *>(ws + L.off_cbuf);
    auto *wts = reinterpret_cast<unsigned long long *>(ws + L.off_w);
    float *rd2 = reinterpret_cast<float *>(ws + L.off_rd2);
    double *rval = reinterpret_cast<double *>(ws + L.off_rval);
    void *lws = ws + L.off_lloyd;
    const int kl = lloyd_k(N);
    auto launched = [] { return cudaGetLastError() == cudaSuccess; };

    // both status words (this call's and the assignment's) start at KPP_OK
    if (cudaMemsetAsync(ws, 0, sizeof(Control), s) != cudaSuccess ||
        cudaMemsetAsync(lws, 0, sizeof(Control), s) != cudaSuccess)
        return KPP_ERR_CUDA;
    kpp_status st = kpp_lloyd_prepare(points, N, d, kl, lws, L.lloyd_bytes, stream);
    if (st != KPP_OK)
        return st;
    kmpar_init_kernel<<<kGrid, kThreads, 0, s>>>(points, N, d, L.range, seed, stream_id, D2, lab,
                                                 cand_out, cbuf, part);
    kmpar_phi_kernel<<<1, 32, 0, s>>>(part, kGrid, sc);
    if (!launched())
        return KPP_ERR_LAUNCH;
    int64_t nc = 1;
    for (int r = 0; r < rounds; ++r) {
        kmpar_sample_kernel<<<kGrid, kThreads, 0, s>>>(D2, N, L.range, sc, ell, seed, stream_id, r,
                                                       flags, bcnt);
        kmpar_scan_kernel<<<1, kGrid, 0, s>>>(bcnt, boff, sc);
        if (!launched())
            return KPP_ERR_LAUNCH;
        long long n_new = 0;
        if (cudaMemcpyAsync(&n_new, &sc->count, sizeof(n_new), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return KPP_ERR_CUDA;
        if (nc + n_new > L.cap) {
            *n_cand_out = nc;
            return KPP_ERR_CAPACITY;
        }
        if (n_new == 0)
            continue;
        kmpar_compact_kernel<<<kGrid, kThreads, 0, s>>>(points, N, d, L.range, flags, boff, nc,
                                                        cand_out, cbuf, D2, lab);
        if (!launched())
            return KPP_ERR_LAUNCH;
        for (int64_t c0 = 0; c0 < n_new; c0 += kl) {
            const int kc = (int)(n_new - c0 < kl ? n_new - c0 : kl);
            st = kpp_lloyd_assign(cbuf + (nc + c0) * d, N, d, kc, pick, lws, L.lloyd_bytes, stream);
            if (st != KPP_OK)
                return st;
            kmpar_min_update_kernel<<<kGrid, kThreads, 0, s>>>(points, N, d, L.range, cbuf,
                                                               nc + c0, kc, pick, D2, lab,
                                                               part);
        }
        kmpar_phi_kernel<<<1, 32, 0, s>>>(part, kGrid, sc);
        if (!launched())
            return KPP_ERR_LAUNCH;
        nc += n_new;
    }
    *n_cand_out = nc;
    if (cudaMemsetAsync(wts, 0, (size_t)nc * 8, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    kmpar_weights_kernel<<<kGrid, kThreads, 0, s>>>(lab, N, wts);
    kmpar_recluster_kernel<<<1, kRecThreads, 0, s>>>(cbuf, nc, d, wts, K, seed, stream_id,
                                                     cand_out, rd2, rval, idx_out, ctl);
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

// kpp_device.cuh -- device building blocks of the seeding kernels:
// Philox draws, streaming loads, stored-format decode, FP32 two-sum
// accumulation, block-level FP64 scan-and-find for the inverse-CDF draw.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kpp.h"

namespace kpp {

constexpr int kWarp = 32;

// ---------------------------------------------------------------------------
// Workspace control block (first 256 bytes of every workspace).
// ---------------------------------------------------------------------------
struct Control {
    int32_t status;     // kpp_status written by the device (0 = OK)
    uint32_t ticket;    // streamed form: CTAs finished with the current pass
    uint32_t bar_count; // persistent form: grid barrier arrivals
    uint32_t bar_gen;   // persistent form: grid barrier generation
    int64_t pick;       // index drawn by the last pass (published to all CTAs)
    uint32_t timeout_where;
    uint32_t pad_[57];
};
static_assert(sizeof(Control) == 256, "control block is 256 bytes");

// Everything a seeding kernel needs about one problem.
struct Problem {
    const void *points;
    const float *scales; // FP8 row scales or nullptr
    int64_t N;
    int32_t d;
    int32_t K;
    uint64_t seed;
    uint64_t stream_id;
    const int64_t *forced;
    int32_t n_forced;
    int32_t nblocks; // number of contiguous row blocks (one per CTA)
    int64_t chunk;   // rows per block (last block may be shorter)
    int64_t *idx;
    float *d2;
    double *phi;
    Control *ctl;
    double *block_sums; // [nblocks]
};

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 64x64
// multiplies with the published multipliers, key bumped by the published Weyl
// constants between rounds.  u_m takes the top 53 bits of output word 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t stream, uint64_t m)
{
    uint64_t x0 = m, x1 = 0, x2 = 0, x3 = 0;
    uint64_t k0 = seed, k1 = stream;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t a = 0xD2E7470EE14C6C93ull, b = 0xCA5A826395121157ull;
        uint64_t hi_a = __umul64hi(a, x0), lo_a = a * x0;
        uint64_t hi_b = __umul64hi(b, x2), lo_b = b * x2;
        uint64_t y0 = hi_b ^ x1 ^ k0;
        uint64_t y2 = hi_a ^ x3 ^ k1;
        x0 = y0;
        x1 = lo_b;
        x2 = y2;
        x3 = lo_a;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    return (double)(x0 >> 11) * 0x1.0p-53;
}

// First seed: min(floor(u_0 * N), N - 1), or the forced index.
__device__ __forceinline__ int64_t first_seed(const Problem &p)
{
    if (p.n_forced > 0)
        return p.forced[0];
    double u = philox_uniform(p.seed, p.stream_id, 0);
    int64_t i = (int64_t)floor(u * (double)p.N);
    return i < p.N - 1 ? i : p.N - 1;
}

// ---------------------------------------------------------------------------
// Loads.
// ---------------------------------------------------------------------------
// 16-byte streaming load through the read-only path, not kept in L1.
// volatile: never speculated past the bounds check that guards it.
__device__ __forceinline__ uint4 ld_stream16(const void *ptr)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr));
    return v;
}

// Coherent-at-L2 loads for data written by other CTAs of the same launch.
__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Stored formats.
// ---------------------------------------------------------------------------
template <int DT> struct Fmt;
template <> struct Fmt<KPP_F32> {
    static constexpr int bytes = 4, per16 = 4;
};
template <> struct Fmt<KPP_BF16> {
    static constexpr int bytes = 2, per16 = 8;
};
template <> struct Fmt<KPP_FP8_E4M3> {
    static constexpr int bytes = 1, per16 = 16;
};

__device__ __forceinline__ void unpack_bf16x2(uint32_t w, float &lo, float &hi)
{
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xffff0000u);
}

__device__ __forceinline__ void unpack_e4m3x2(uint32_t w16, float &lo, float &hi)
{
    __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w16 & 0xffffu), __NV_E4M3);
    float2 f = __half22float2(*reinterpret_cast<__half2 *>(&h));
    lo = f.x;
    hi = f.y;
}

// Decode one 16-byte vector into Fmt<DT>::per16 floats.  For FP8 the value
// is scale * decode(q), rounded once to FP32 (never fused into a later
// subtraction, so a point and the same point used as a centre decode alike).
template <int DT>
__device__ __forceinline__ void decode16(uint4 v, float scale, float *out)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    if constexpr (DT == KPP_F32) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            out[i] = __uint_as_float(w[i]);
    } else if constexpr (DT == KPP_BF16) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            unpack_bf16x2(w[i], out[2 * i], out[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            unpack_e4m3x2(w[i], out[4 * i], out[4 * i + 1]);
            unpack_e4m3x2(w[i] >> 16, out[4 * i + 2], out[4 * i + 3]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
            out[i] = __fmul_rn(scale, out[i]);
    }
}

// Decode a single stored element (generic / scalar paths).
template <int DT>
__device__ __forceinline__ float decode1(const void *points, int64_t k, float scale)
{
    if constexpr (DT == KPP_F32) {
        return __ldg(reinterpret_cast<const float *>(points) + k);
    } else if constexpr (DT == KPP_BF16) {
        uint16_t h = __ldg(reinterpret_cast<const unsigned short *>(points) + k);
        return __uint_as_float((uint32_t)h << 16);
    } else {
        uint8_t q = __ldg(reinterpret_cast<const unsigned char *>(points) + k);
        float lo, hi;
        unpack_e4m3x2(q, lo, hi);
        return __fmul_rn(scale, lo);
    }
}

// ---------------------------------------------------------------------------
// FP32 two-sum accumulator: hi + lo equals the exact running sum up to
// rounding in lo (Knuth's TwoSum, 6 flops, no FP64 on the per-row path).
// ---------------------------------------------------------------------------
struct Acc2 {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float s = __fadd_rn(hi, x);
        float bb = __fsub_rn(s, hi);
        float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------------------
// Block reductions and scans (deterministic association).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of one double per thread over the block, in a fixed order; result on
// all threads.  `sh` needs NT/32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0)
        sh[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w)
        t += sh[w];
    return t;
}

// Exclusive prefix of one double per thread, in thread order; also returns
// the total.  `sh` needs NT/32 + 1 doubles.
template <int NT>
__device__ __forceinline__ double block_exclusive_scan(double v, double *sh, double &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    double prev = __shfl_up_sync(0xffffffffu, incl, 1);
    __syncthreads();
    if (lane == 31)
        sh[warp] = incl;
    __syncthreads();
    double before = 0.0, all = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        if (w < warp)
            before += sh[w];
        all += sh[w];
    }
    total = all;
    return lane ? before + prev : before;
}

template <int NT>
__device__ __forceinline__ int64_t block_min_i64(int64_t v, int64_t *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t y = __shfl_xor_sync(0xffffffffu, v, o);
        v = y < v ? y : v;
    }
    __syncthreads();
    if (lane == 0)
        sh[warp] = v;
    __syncthreads();
    int64_t r = sh[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w)
        r = sh[w] < r ? sh[w] : r;
    return r;
}

template <int NT>
__device__ __forceinline__ int64_t block_max_i64(int64_t v, int64_t *sh)
{
    return -block_min_i64<NT>(-v, sh);
}

// Ordered FP64 total of n values: contiguous per-thread slices summed in
// order, slice totals summed in thread order (the association block_find
// uses for its total).
template <int NT, class Get>
__device__ double block_ordered_total(int64_t n, Get get, double *shd)
{
    const int64_t per = (n + NT - 1) / NT;
    const int64_t b = (int64_t)threadIdx.x * per;
    const int64_t e = b + per < n ? b + per : n;
    double own = 0.0;
    for (int64_t k = b; k < e; ++k)
        own += get(k);
    double total;
    block_exclusive_scan<NT>(own, shd, total);
    return total;
}

struct FindResult {
    int64_t index;  // first k with base + prefix_k > t, or -1
    double before;  // base + prefix up to k-1 (valid if index >= 0)
    double total;   // base + sum of all n values
    int64_t last_positive; // largest k with value > 0, or -1
};

// Block-cooperative inverse-CDF search over n values v_k = get(k):
// thread t sums the contiguous slice [t*per, (t+1)*per) in order, slice
// totals are prefix-summed in thread order, and every slice is walked again
// from its exclusive prefix.  The threshold is t = u * (base + total) when
// `u_mode` is set, else `u_or_t` itself.  All threads return the same result.
template <int NT, class Get>
__device__ FindResult block_find(int64_t n, Get get, double base, double u_or_t, bool u_mode,
                                 double *shd, int64_t *shi, double *t_out = nullptr)
{
    const int64_t per = (n + NT - 1) / NT;
    const int64_t b = (int64_t)threadIdx.x * per;
    const int64_t e = b + per < n ? b + per : n;
    double own = 0.0;
    int64_t lastpos = -1;
    for (int64_t k = b; k < e; ++k) {
        double v = get(k);
        own += v;
        if (v > 0.0)
            lastpos = k;
    }
    double total;
    double excl = block_exclusive_scan<NT>(own, shd, total);
    const double t = u_mode ? u_or_t * (base + total) : u_or_t;
    if (t_out)
        *t_out = t;
    double run = base + excl;
    int64_t cand = INT64_MAX;
    double cand_before = 0.0;
    // First crossing of t within the slice; a zero weight never crosses.
    for (int64_t k = b; k < e; ++k) {
        double v = get(k);
        double next = run + v;
        if (v > 0.0 && next > t) {
            cand = k;
            cand_before = run;
            break;
        }
        run = next;
    }
    FindResult r;
    r.total = base + total;
    r.index = block_min_i64<NT>(cand, shi);
    r.last_positive = block_max_i64<NT>(lastpos, shi);
    __syncthreads();
    if (cand == r.index && cand != INT64_MAX)
        shd[0] = cand_before;
    __syncthreads();
    r.before = shd[0];
    if (r.index == INT64_MAX)
        r.index = -1;
    __syncthreads();
    return r;
}

// The draw of seed m (m >= 1) from per-block FP64 sums and per-point FP32
// D^2, by one thread block: find the block whose running FP64 sum first
// exceeds t = u_m * T, then rescan only that block's points from the
// block's exclusive prefix.  Returns the drawn index, or -1 if T == 0
// (degenerate).  `T_out` gets T on all threads.
template <int NT>
__device__ int64_t hierarchical_draw(const double *block_sums, int nblocks, const float *d2,
                                     int64_t N, int64_t chunk, double u, double *shd,
                                     int64_t *shi, double *T_out)
{
    double t;
    FindResult r1 = block_find<NT>(
        nblocks, [&](int64_t k) { return ld_cg(block_sums + k); }, 0.0, u, true, shd, shi, &t);
    *T_out = r1.total;
    if (!(r1.total > 0.0))
        return -1;
    int64_t blk = r1.index;
    double base = r1.before;
    double thr = t;
    if (blk < 0) { // rounding left no block above t: last block with weight
        blk = r1.last_positive;
        thr = INFINITY;
        base = 0.0;
    }
    const int64_t row0 = blk * chunk;
    const int64_t n2 = (N - row0) < chunk ? (N - row0) : chunk;
    FindResult r2 = block_find<NT>(
        n2, [&](int64_t k) { return (double)ld_cg(d2 + row0 + k); }, base, thr, false, shd, shi);
    if (r2.index >= 0)
        return row0 + r2.index;
    // rounding inside the block: its last point with weight (one exists,
    // since the block's sum is positive)
    return row0 + (r2.last_positive >= 0 ? r2.last_positive : 0);
}

} // namespace kpp

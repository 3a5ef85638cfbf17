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
    int32_t status;          // kpp_status written by the device (0 = OK)
    uint32_t ticket;         // streamed form: CTAs finished with the current pass
    unsigned long long mail; // persistent form: (drawn index << 32) | (pass + 1)
    uint32_t timeout_where;  // persistent form: pass whose wait gave up
    uint32_t bounds_site;    // debug build: site of the first index out of bounds
    uint32_t pad_[58];
};

// ---------------------------------------------------------------------------
// Debug build (KPP_DEBUG=1): index checks before the memory accesses of the
// hot kernels.  A check that fails records KPP_ERR_BOUNDS and its site in the
// status block (the first one wins) and tells the caller to skip the access;
// the release build compiles every check to `true`.
// ---------------------------------------------------------------------------
#ifndef KPP_DEBUG
#define KPP_DEBUG 0
#endif

__device__ __forceinline__ bool kpp_check(Control *ctl, bool ok, uint32_t site)
{
#if KPP_DEBUG
    if (!ok && ctl && atomicCAS(&ctl->status, KPP_OK, KPP_ERR_BOUNDS) == KPP_OK)
        atomicExch(&ctl->bounds_site, site);
    return ok;
#else
    (void)ctl;
    (void)site;
    return true;
#endif
}

// One tagged block sum per 32-byte slot, so the slots polled by every CTA
// sit in different sectors.
constexpr int kSlotWords = 4;
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
    int32_t nseg;    // segments per block (one per warp)
    int64_t chunk;   // rows per block (last block may be shorter)
    int64_t sw;      // rows per warp super-iteration; segments are whole ones
    int64_t *idx;
    float *d2;
    double *phi;
    Control *ctl;
    float2 *block_sums; // streamed form: [nblocks] pair sums of the pass
    float2 *seg_sums;   // streamed form: [nblocks * nseg] pair sums of the pass
    unsigned long long *slots; // persistent form: [2][nblocks * kSlotWords] tagged block sums
    unsigned long long *mail;  // persistent form: the drawn index, tagged with its pass
    int32_t recompute;         // streamed form: every pass rebuilds D^2 from all chosen seeds
    int32_t exact_draws;       // every draw decision in FP64 (the near-tie path), for testing
    // point-sharded seeding (one contiguous row range of a larger problem):
    // the centre of the pass comes from the exchange buffer `xchg` (global
    // index, row scale, stored row), indices are global (< n_global), and a
    // pass ends with the shard's D^2 total in `shard_total` instead of a draw
    const long long *xchg;
    float *shard_total;
    int64_t n_global;
};

// Exchange buffer of point-sharded seeding, in 64-bit words: [0] the global
// index of the centre, [1] its FP8 row scale (low 32 bits), [2..] its stored
// row (d * bytes, padded to 16 bytes).  Sharded processes sum their buffers
// (the owner's words plus zeros), so every word is its owner's bit pattern.
__host__ __device__ __forceinline__ int64_t xchg_words(int d, int elem_bytes)
{
    return 2 + 2 * (((int64_t)d * elem_bytes + 15) / 16);
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 64x64
// multiplies with the published multipliers, key bumped by the published Weyl
// constants between rounds.  A uniform takes the top 53 bits of output word
// 0; the k-means++ draw u_m uses the counter {m, 0, 0, 0}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double philox_uniform_ctr(uint64_t seed, uint64_t stream, uint64_t c0,
                                                     uint64_t c1, uint64_t c2, uint64_t c3)
{
    uint64_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
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

__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t stream, uint64_t m)
{
    return philox_uniform_ctr(seed, stream, m, 0, 0, 0);
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

// Decode one 16-byte vector into Fmt<DT>::per16 floats.  FP32 and BF16 give
// the stored values exactly; FP8 gives the unscaled E4M3 values q (exact in
// FP32) -- the row scale is applied inside the distance (see diff_fp8).
template <int DT>
__device__ __forceinline__ void decode16(uint4 v, float *out)
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
    }
}

// Decode a single stored element (generic / scalar paths); FP8 unscaled.
template <int DT>
__device__ __forceinline__ float decode1(const void *points, int64_t k)
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
        return lo;
    }
}

// An FP8 centre coordinate c = s_c * q_c (exact in FP64, not in FP32) is held
// as an unevaluated pair c_hi + c_lo with c_hi = RN(s_c * q_c) and c_lo the
// exact rounding error.  A point coordinate x = s * q then differs from it by
//   x - c = fma(s, q, -c_hi) - c_lo,
// rounded about once relative to the difference itself, so cancellation near
// the centre costs no accuracy and the centre's own distance is exactly 0.
__device__ __forceinline__ void split_fp8_centre(float s, float q, float &hi, float &lo)
{
    hi = __fmul_rn(s, q);
    lo = __fmaf_rn(s, q, -hi);
}

__device__ __forceinline__ float diff_fp8(float s, float q, float c_hi, float c_lo)
{
    return __fsub_rn(__fmaf_rn(s, q, -c_hi), c_lo);
}

// ---------------------------------------------------------------------------
// FP32 two-sum pairs: hi + lo holds a running sum with about 48 significant
// bits (Knuth's error-free TwoSum), so D^2 sums need no FP64 on the per-row
// path (GB300's FP64 rate is a small fraction of its FP32 rate).  Integer
// sums are exact while the error terms stay below 2^24.
// ---------------------------------------------------------------------------
struct Pair {
    float hi, lo; // trivial type (usable in shared memory); value-initialise with Pair{}

    __device__ __forceinline__ void add(float x)
    {
        float s = __fadd_rn(hi, x);
        float bb = __fsub_rn(s, hi);
        float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    // pair + pair; the exact error term makes this commutative, so butterfly
    // reductions leave the same value on every lane
    __device__ __forceinline__ void add(const Pair &o)
    {
        float s = __fadd_rn(hi, o.hi);
        float bb = __fsub_rn(s, hi);
        float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(o.hi, bb));
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, o.lo), err);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Butterfly sum of a pair over the 32 lanes (same result on every lane).
__device__ __forceinline__ Pair warp_pair_sum(Pair p)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Pair q;
        q.hi = __shfl_xor_sync(0xffffffffu, p.hi, o);
        q.lo = __shfl_xor_sync(0xffffffffu, p.lo, o);
        p.add(q);
    }
    return p;
}

__device__ __forceinline__ Pair shfl_pair(Pair p, int src)
{
    Pair q;
    q.hi = __shfl_sync(0xffffffffu, p.hi, src);
    q.lo = __shfl_sync(0xffffffffu, p.lo, src);
    return q;
}

__device__ __forceinline__ Pair pair_sum(Pair a, const Pair &b)
{
    a.add(b);
    return a;
}

// Inclusive prefix over lanes (Hillis-Steele); `excl` gets the exclusive one.
__device__ __forceinline__ Pair warp_pair_scan(Pair v, Pair &excl)
{
    const int lane = threadIdx.x & 31;
    Pair incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Pair y;
        y.hi = __shfl_up_sync(0xffffffffu, incl.hi, o);
        y.lo = __shfl_up_sync(0xffffffffu, incl.lo, o);
        if (lane >= o) {
            y.add(incl); // y precedes incl: keep the order of association
            incl = y;
        }
    }
    Pair e;
    e.hi = __shfl_up_sync(0xffffffffu, incl.hi, 1);
    e.lo = __shfl_up_sync(0xffffffffu, incl.lo, 1);
    excl = lane ? e : Pair{};
    return incl;
}

// ---------------------------------------------------------------------------
// The draw's threshold t = u * T.  Decisions "prefix > t" are taken on an
// FP32 pair approximation of t (relative error below 2^-44) whenever the
// prefix is farther than tol = 2^-40 * t from it -- then the answer is
// certain -- and otherwise (a near tie, rare) in FP64 against the exact
// t = fl64(u * T), the value the FP64 oracle uses.  FP64 is slow on this GPU
// (a dependent add costs ~64 cycles against ~5 for FP32), so the common case
// avoids it entirely.
// ---------------------------------------------------------------------------
// Exact FP64 decision of a near tie: (P.hi + P.lo) > u * (T.hi + T.lo).
// Out of line so that the compiler branches around it instead of computing
// it (predicated) on every comparison.
static __device__ __noinline__ bool pair_gt_exact(float phi, float plo, double u, float Thi, float Tlo)
{
    return (double)phi + (double)plo > u * ((double)Thi + (double)Tlo);
}

struct Thresh {
    float hi, lo; // approximation of t
    float tol;
    float uh, ul; // u split into two floats
    double u;
    Pair T;
    int inf;   // t = +infinity: no prefix exceeds it
    int all_exact; // every decision in FP64 (tol = +infinity)

    __device__ __forceinline__ double exact() const
    {
        return u * ((double)T.hi + (double)T.lo);
    }
    // prefix P > t ?
    __device__ __forceinline__ bool gt(const Pair &P) const
    {
        if (inf)
            return false;
        const float d = __fadd_rn(__fsub_rn(P.hi, hi), __fsub_rn(P.lo, lo));
        if (d > tol)
            return true;
        if (d < -tol)
            return false;
        return pair_gt_exact(P.hi, P.lo, u, T.hi, T.lo);
    }
};

// u and its float split; the FP64 work here is off the draw's critical path.
// `exact`: no decision is left to the FP32 estimate (the near-tie path is
// taken at every comparison).
__device__ __forceinline__ Thresh thresh_for_u(double u, int exact = 0)
{
    Thresh th;
    th.all_exact = exact;
    th.u = u;
    th.uh = (float)u;
    th.ul = (float)(u - (double)th.uh);
    th.hi = th.lo = th.tol = 0.f;
    th.T = Pair{0.f, 0.f};
    th.inf = 0;
    return th;
}

// The same threshold from a draw whose float split was computed ahead.
__device__ __forceinline__ Thresh thresh_for_split(double u, float uh, float ul, int exact = 0)
{
    Thresh th;
    th.all_exact = exact;
    th.u = u;
    th.uh = uh;
    th.ul = ul;
    th.hi = th.lo = th.tol = 0.f;
    th.T = Pair{0.f, 0.f};
    th.inf = 0;
    return th;
}

// Completes a threshold once T is known: t ~ uh*T.hi + (exact error of that
// product) + uh*T.lo + ul*T.hi, all in FP32.
__device__ __forceinline__ void thresh_set_total(Thresh &th, const Pair &T)
{
    th.T = T;
    const float p = __fmul_rn(th.uh, T.hi);
    const float e = __fmaf_rn(th.uh, T.hi, -p);
    th.hi = p;
    th.lo = __fadd_rn(e, __fmaf_rn(th.uh, T.lo, __fmul_rn(th.ul, T.hi)));
    th.tol = th.all_exact ? __int_as_float(0x7f800000) : fabsf(p) * 0x1.0p-40f + 0x1.0p-126f;
}

__device__ __forceinline__ Thresh thresh_inf()
{
    Thresh th = thresh_for_u(0.0);
    th.inf = 1;
    return th;
}

// ---------------------------------------------------------------------------
// Warp-level inverse-CDF search (the draw) over n values v_k >= 0 (get(k)
// returns a Pair), in FP32 two-sum pairs.  Lane l sums the contiguous slice
// [l*per, (l+1)*per) in order; slice sums are prefix-summed over lanes; the
// first lane whose running total exceeds t is walked element by element, one
// element per lane.  The result is the first k with v_k > 0 and
// base + prefix_k > t.  With `u_mode`, the threshold's total is first set to
// base + (sum of all values).  Every lane returns the same result.
// n <= 1024.
// ---------------------------------------------------------------------------
struct PFind {
    int64_t index;         // first crossing, or -1
    int64_t last_positive; // largest k with v_k > 0, or -1
    Pair before;           // base + prefix before the crossing
    Pair total;            // base + sum of all values
    Thresh th;             // the threshold used
};

__device__ __forceinline__ bool pair_gt(const Pair &p, double t)
{
    return (double)p.hi + (double)p.lo > t;
}

template <class Get>
__device__ __forceinline__ PFind warp_pfind(int n, Get get, Pair base, const Thresh &th_in,
                                            bool u_mode)
{
    const int lane = threadIdx.x & 31;
    const int per = (n + 31) >> 5;
    const int b = lane * per;
    const int e = b + per < n ? b + per : n;
    Pair own{};
    for (int k = b; k < e; ++k)
        own.add(get(k));
    Pair excl;
    const Pair incl = warp_pair_scan(own, excl);
    PFind r;
    r.before = Pair{};
    r.total = pair_sum(base, shfl_pair(incl, 31));
    r.th = th_in;
    if (u_mode)
        thresh_set_total(r.th, r.total);
    const Pair start = pair_sum(base, excl);
    const unsigned cross = __ballot_sync(0xffffffffu, b < e && r.th.gt(pair_sum(base, incl)));
    r.index = -1;
    r.last_positive = -1;
    if (cross) {
        // the first lane whose running total passes t walks its own slice;
        // rounding can leave that walk short of t: then the slice's last point
        // with weight
        const int L = __ffs(cross) - 1;
        int idx = -1;
        Pair before{};
        if (lane == L) {
            Pair run = start;
            int lastpos = -1;
            Pair lastpos_before{};
            for (int k = b; k < e; ++k) {
                const Pair v = get(k);
                const Pair next = pair_sum(run, v);
                if (v.hi > 0.f) {
                    if (r.th.gt(next)) {
                        idx = k;
                        before = run;
                        break;
                    }
                    lastpos = k;
                    lastpos_before = run;
                }
                run = next;
            }
            if (idx < 0) {
                idx = lastpos;
                before = lastpos_before;
            }
        }
        r.index = __shfl_sync(0xffffffffu, idx, L);
        r.before = shfl_pair(before, L);
    }
    if (r.index < 0) { // no crossing: the last value with weight (rare)
        int lp = -1;
        for (int k = b; k < e; ++k)
            if (get(k).hi > 0.f)
                lp = k;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int y = __shfl_xor_sync(0xffffffffu, lp, o);
            lp = y > lp ? y : lp;
        }
        r.last_positive = lp;
    }
    return r;
}

// Rows [first, last) of segment `seg` of a block of `rows` rows starting at
// `row0`: the block's super-iterations of `sw` rows are split evenly over
// `nseg` segments, segment w taking [w * ns / nseg, (w + 1) * ns / nseg).
__host__ __device__ __forceinline__ void segment_rows(int64_t row0, int64_t rows, int64_t sw,
                                                      int nseg, int seg, int64_t *first,
                                                      int64_t *last)
{
    const int64_t ns = (rows + sw - 1) / sw;
    const int64_t sb = (int64_t)seg * ns / nseg, se = (int64_t)(seg + 1) * ns / nseg;
    *first = row0 + sb * sw;
    const int64_t e = row0 + se * sw;
    *last = e < row0 + rows ? e : row0 + rows;
}

constexpr int kStage = 1024; // values staged in shared memory per round

// One-value-per-lane search (n <= 32): the first lane k < n with v_k > 0 and
// base + prefix_k > t, and the prefix before it; if none, the last lane with
// weight (index -1 if none at all).  Every lane returns the same result.
struct Find32 {
    int index;
    Pair before;
};

__device__ __forceinline__ Find32 warp_find32(int n, Pair v, Pair base, const Thresh &th)
{
    const int lane = threadIdx.x & 31;
    if (lane >= n)
        v = Pair{0.f, 0.f};
    Pair ex;
    const Pair in = warp_pair_scan(v, ex);
    const bool pos = lane < n && v.hi > 0.f;
    const unsigned hit = __ballot_sync(0xffffffffu, pos && th.gt(pair_sum(base, in)));
    Find32 r;
    if (hit) {
        r.index = __ffs(hit) - 1;
    } else {
        const unsigned any = __ballot_sync(0xffffffffu, pos);
        r.index = any ? 31 - __clz(any) : -1;
    }
    r.before = pair_sum(base, shfl_pair(ex, r.index < 0 ? 0 : r.index));
    return r;
}

// Point-level search of a draw by one warp over rows [first, last) whose D^2
// are read by `get_d2(row)`: lane l sums, in order, the rows of its slice of
// whole 32-row chunks; the slice sums are prefix-summed over lanes; then the
// chunks of the first slice whose running total passes t are scanned one at
// a time with one row per lane.  Returns the first row with D^2 > 0 whose
// prefix (from `base`) exceeds t -- or, when rounding leaves none, the last
// row with weight in the crossing slice (the last in the range if t.inf) --
// and `first` if no row has weight.  All lanes return the same row.
template <class GetD2>
__device__ int64_t warp_rows_find(int64_t first, int64_t last, GetD2 get_d2, Pair base,
                                  const Thresh &th)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = last - first;
    const int64_t nch = (n + 31) / 32;
    const int64_t pc = (nch + 31) / 32; // chunks per lane
    const int64_t sb = first + (int64_t)lane * pc * 32;
    const int64_t se_ = sb + pc * 32;
    const int64_t se = se_ < last ? se_ : last;
    Pair own{};
#pragma unroll 8
    for (int64_t r = sb; r < se; ++r)
        own.add(get_d2(r));
    Pair excl;
    const Pair incl = warp_pair_scan(own, excl);
    unsigned cross = __ballot_sync(0xffffffffu, sb < se && th.gt(pair_sum(base, incl)));
    int L;
    if (cross) {
        L = __ffs(cross) - 1;
    } else { // no slice passes t: the last slice with weight
        const unsigned pos = __ballot_sync(0xffffffffu, sb < se && own.hi > 0.f);
        if (!pos)
            return first;
        L = 31 - __clz(pos);
    }
    Pair run = pair_sum(base, shfl_pair(excl, L));
    const int64_t lb = first + (int64_t)L * pc * 32;
    const int64_t le_ = lb + pc * 32;
    const int64_t le = le_ < last ? le_ : last;
    int64_t lastpos = -1;
    for (int64_t c = lb; c < le; c += 32) {
        const int64_t row = c + lane;
        const float v = row < le ? get_d2(row) : 0.f;
        Pair vex;
        const Pair vin = warp_pair_scan(Pair{v, 0.f}, vex);
        const unsigned hit = __ballot_sync(0xffffffffu, v > 0.f && th.gt(pair_sum(run, vin)));
        if (hit)
            return c + (__ffs(hit) - 1);
        const unsigned pos = __ballot_sync(0xffffffffu, v > 0.f);
        if (pos)
            lastpos = c + (31 - __clz(pos));
        run = pair_sum(run, shfl_pair(vin, 31));
    }
    return lastpos >= 0 ? lastpos : first;
}

// ---------------------------------------------------------------------------
// Tagged words for the persistent form's grid-wide exchange.  Every exchanged
// value fits one 64-bit word, written and read with single-copy-atomic
// relaxed accesses, and carries its own pass tag, so a reader needs no fence:
//   block-sum slot:  (bits(lo) << 32) | bits(hi) with the sign bit of hi
//                    (hi >= 0) replaced by the tag of the pass;
//   mailbox:         (index << 32) | (pass + 1).
// The slot of pass m lives in buffer m & 1, and its tag bit is
// ((m >> 1) + 1) & 1: it flips between two uses of the same buffer, and a
// zeroed buffer never matches the first use.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t slot_tag(int m) { return (uint32_t)(((m >> 1) + 1) & 1); }

__device__ __forceinline__ unsigned long long pack_slot(const Pair &p, int m)
{
    const uint32_t hi = (__float_as_uint(p.hi) & 0x7fffffffu) | (slot_tag(m) << 31);
    return ((unsigned long long)__float_as_uint(p.lo) << 32) | hi;
}

__device__ __forceinline__ Pair unpack_slot(unsigned long long w)
{
    return Pair{__uint_as_float((uint32_t)w & 0x7fffffffu), __uint_as_float((uint32_t)(w >> 32))};
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *a, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *a)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}

// ---------------------------------------------------------------------------
// Bounded waits (persistent form, cooperative launch only).  A wait that
// outlasts its deadline records KPP_ERR_TIMEOUT (and the pass) in the status
// word and returns false instead of hanging; any other error recorded by
// another CTA also ends the wait.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool give_up(Control *ctl, uint64_t t0, uint64_t timeout_ns,
                                        uint32_t it, uint32_t where)
{
    if ((it & 63u) == 0 && *(volatile int32_t *)&ctl->status != KPP_OK)
        return true;
    if (global_ns() - t0 > timeout_ns) {
        if (atomicCAS(&ctl->status, KPP_OK, KPP_ERR_TIMEOUT) == KPP_OK)
            ctl->timeout_where = where;
        return true;
    }
    return false;
}

// Waits until slot `a` carries the tag of pass m; returns false on give-up.
__device__ __forceinline__ bool wait_slot(const unsigned long long *a, int m, Control *ctl,
                                          uint64_t timeout_ns, Pair *out)
{
    const uint32_t tag = slot_tag(m);
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        const unsigned long long w = ld_relaxed_u64(a);
        if (((uint32_t)w >> 31) == tag) {
            *out = unpack_slot(w);
            return true;
        }
        if (give_up(ctl, t0, timeout_ns, it, (uint32_t)m))
            return false;
    }
}

// One warp waits for slots [0, n) of pass m (n <= 32 * 8 per call), storing
// the unpacked pairs in `out`.  Each lane owns slots lane, lane + 32, ...; all
// its pending loads are issued before any is checked, so a round costs one
// memory round trip however many slots a lane owns.  Returns false (on all
// lanes) if a wait gave up.
__device__ __forceinline__ bool warp_wait_slots(const unsigned long long *slots, int n, int m,
                                                Control *ctl, uint64_t timeout_ns, float2 *out)
{
    constexpr int kPer = 8;
    const int lane = threadIdx.x & 31;
    const uint32_t tag = slot_tag(m);
    unsigned pending = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j)
        if (lane + 32 * j < n)
            pending |= 1u << j;
    const uint64_t t0 = global_ns();
    bool ok = true;
    for (uint32_t it = 1; pending; ++it) {
        unsigned long long w[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j)
            w[j] = (pending >> j) & 1u ? ld_relaxed_u64(slots + (size_t)(lane + 32 * j) * kSlotWords)
                                       : 0ull;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            if (((pending >> j) & 1u) && ((uint32_t)w[j] >> 31) == tag) {
                const Pair v = unpack_slot(w[j]);
                out[lane + 32 * j] = make_float2(v.hi, v.lo);
                pending &= ~(1u << j);
            }
        }
        if (pending && give_up(ctl, t0, timeout_ns, it, (uint32_t)m)) {
            ok = false;
            break;
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// Waits until the mailbox carries pass m's index; returns it, or -1.
__device__ __forceinline__ int64_t wait_mail(const unsigned long long *mail, Control *ctl, int m,
                                             uint64_t timeout_ns)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        const unsigned long long w = ld_relaxed_u64(mail);
        if ((uint32_t)w == (uint32_t)(m + 1))
            return (int64_t)(w >> 32);
        if (give_up(ctl, t0, timeout_ns, it, (uint32_t)m))
            return -1;
    }
}

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

} // namespace kpp

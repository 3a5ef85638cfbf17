// kpp_pass.cuh -- the per-point work of one seeding pass, shared by the
// streamed and persistent forms (Algorithm 2: the per-point loop run in
// parallel over contiguous partitions of the points):
//   - distance of every point of the CTA's row range to the newest centre,
//     d_{m,l} = d(H_m, n_l), in the difference form with FP32 FMAs;
//   - the min-update of the nearest squared distance d_sn (D^2);
//   - the D^2 sum of each warp's contiguous segment of rows, accumulated per
//     lane as FP32 two-sum pairs and reduced across the warp once per pass,
//     and the CTA's sum of its segments.
#pragma once

#include "kpp_device.cuh"

namespace kpp {

// Geometry of one (dtype, d, lanes-per-row) specialisation.
//   WIDE rows (>= 16 bytes): L lanes share a row, each lane reading VPL
//     16-byte vectors of it; a warp covers 32 rows per super-iteration and
//     lane (g, l) ends up owning row base + l * (32 / L) + g.
//   Narrow rows (< 16 bytes): one 16-byte vector holds RPV whole rows; a
//     lane owns RPV consecutive rows and a warp covers 32 * RPV rows.
// Each warp walks a contiguous run of super-iterations (its segment).
template <int DT, int D, int L_>
struct Geom {
    static constexpr int EB = Fmt<DT>::bytes;
    static constexpr int EPV = Fmt<DT>::per16;
    static constexpr int RB = D * EB;
    static constexpr bool WIDE = RB >= 16;
    static constexpr int VPR = WIDE ? RB / 16 : 1;
    static constexpr int L = WIDE ? L_ : 1;
    static constexpr int VPL = WIDE ? VPR / L : 1;
    static constexpr int RPV = WIDE ? 1 : 16 / RB;
    static constexpr int SW = WIDE ? 32 : 32 * RPV; // rows per warp super-iteration
    static constexpr int CREG = WIDE ? VPL * EPV : EPV;
    // slots per batch: 8 vectors per lane per batch (4 for FP8, whose decoded
    // vectors are 4x wider); two batches are in flight with the pipelining
    static constexpr int VB = (DT == KPP_FP8_E4M3) ? 4 : 8;
    static constexpr int JB = WIDE ? ((VB / VPL) < 1 ? 1 : ((VB / VPL) > L ? L : (VB / VPL))) : 1;
    static_assert(!WIDE || (RB % 16 == 0), "wide rows are whole vectors");
    static_assert(!WIDE || (VPR % L == 0 && L >= 1 && L <= 32 && (L & (L - 1)) == 0),
                  "lanes per row must divide the row's vectors");
    static_assert(WIDE || (16 % RB == 0), "narrow rows tile a vector");
    static_assert(!WIDE || (L % JB == 0), "slot batches tile the slots");
    // batches kept in flight by the software pipeline: about 16 vectors per
    // lane whatever the row size (FP8: 8); narrow rows, which also carry
    // RPV prefetched D^2 values per batch, 8 batches at most
    static constexpr int VPB = WIDE ? JB * VPL : 1; // vectors per batch
    static constexpr int PD0 = (2 * VB) / VPB;
    static constexpr int PDW = PD0 < 2 ? 2 : (PD0 > 16 ? 16 : PD0);
    static constexpr int PD = WIDE ? PDW : (RPV <= 2 ? 8 : (RPV == 4 ? 4 : 2));
};

// Packed FP32 pairs for the Blackwell FP32x2 instructions.
using F2 = unsigned long long;

__device__ __forceinline__ F2 f2(float lo, float hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_split(F2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ F2 f2_sub(F2 a, F2 b)
{
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Per-lane slice of the newest centre, decoded to FP32 once per pass.  For
// FP8 each coordinate is the pair (c_hi, c_lo) of split_fp8_centre.
template <int DT, int D, int L_>
struct CentreRegs {
    using G = Geom<DT, D, L_>;
    static constexpr int NLO = (DT == KPP_FP8_E4M3) ? G::CREG : 1;
    float c[G::CREG];
    float clo[NLO];

    __device__ __forceinline__ void set(int k, float s, float raw)
    {
        if constexpr (DT == KPP_FP8_E4M3)
            split_fp8_centre(s, raw, c[k], clo[k]);
        else
            c[k] = raw;
    }

    __device__ __forceinline__ void load(const void *points, const float *scales, int64_t ci)
    {
        const int lane = threadIdx.x & 31;
        const float sc = (DT == KPP_FP8_E4M3) ? __ldg(scales + ci) : 1.0f;
        const char *row = reinterpret_cast<const char *>(points) + ci * (int64_t)G::RB;
        if constexpr (G::WIDE) {
            const int l = lane % G::L;
#pragma unroll
            for (int v = 0; v < G::VPL; ++v) {
                uint4 x = *reinterpret_cast<const uint4 *>(row + (v * G::L + l) * 16);
                float f[G::EPV];
                decode16<DT>(x, f);
#pragma unroll
                for (int e = 0; e < G::EPV; ++e)
                    set(v * G::EPV + e, sc, f[e]);
            }
        } else {
            float tmp[D];
#pragma unroll
            for (int k = 0; k < D; ++k)
                tmp[k] = decode1<DT>(points, ci * D + k);
#pragma unroll
            for (int e = 0; e < G::EPV; ++e)
                set(e, sc, tmp[e % D]);
        }
    }

    // Adds sum_e (x_e - c_{k0+e})^2 of one decoded vector into (a0, a1):
    // even elements into a0, odd into a1, with packed FP32x2 instructions
    // (each lane of a packed op rounds exactly like the scalar op).
    // `s` is the row scale (FP8 only).
    template <int N>
    __device__ __forceinline__ void accum(const float *f, int k0, float s, float &a0,
                                          float &a1) const
    {
        F2 acc = f2(a0, a1);
#pragma unroll
        for (int e = 0; e < N; e += 2) {
            F2 t;
            if constexpr (DT == KPP_FP8_E4M3) {
                const F2 x = f2_fma(f2(s, s), f2(f[e], f[e + 1]),
                                    f2(-c[k0 + e], -c[k0 + e + 1]));
                t = f2_sub(x, f2(clo[k0 + e], clo[k0 + e + 1]));
            } else {
                t = f2_sub(f2(f[e], f[e + 1]), f2(c[k0 + e], c[k0 + e + 1]));
            }
            acc = f2_fma(t, t, acc);
        }
        f2_split(acc, a0, a1);
    }
};

// Where D^2 lives during a pass.
enum D2Mode {
    D2_INPLACE = 0, // the global D^2 array, read and written in place
    D2_SMEM = 1     // shared memory (copied out to the global array when asked)
};

struct PassIO {
    int64_t r0, r1;        // this CTA's rows
    bool first;            // pass 0: D^2 starts at +infinity
    bool reverse;          // walk each segment last super-iteration first
    const char *gpts;      // points in global memory
    const float *scales;   // FP8 row scales
    char *cache;           // shared-memory copy of the first `cache_supers`
    int64_t cache_supers;  //   super-iterations of every warp's segment, or null
    bool fill_cache;       // this pass loads the cached rows and stores them
    float *d2;             // D2_INPLACE: the global D^2 array
    float *d2_out;         // D2_SMEM: also store this pass's D^2 here, or null
    float *d2s;            // D2_SMEM: shared memory, indexed by row - r0
    float2 *segs;          // segment sums of this CTA, one per warp (global or smem)
    uint64_t policy;       // L2 cache policy of global point loads (0: none)
    Control *ctl;          // status block (debug build: index checks report here)
};

__device__ __forceinline__ uint4 ld_global_hint(const void *ptr, uint64_t policy)
{
    uint4 v;
    asm volatile(
        "ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr), "l"(policy));
    return v;
}

__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 16-byte shared-memory accesses by explicit shared-window address (the
// cache pointer is chosen at run time between shared and global memory, so
// the compiler could not prove the address space by itself).
__device__ __forceinline__ uint4 lds16(const void *p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a));
    return v;
}

__device__ __forceinline__ void sts16(void *p, uint4 v)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// One 16-byte vector of row data: from the shared-memory cache slot of the
// super-iteration (if cached and not being filled), else from global memory.
__device__ __forceinline__ uint4 load_vec(const PassIO &io, const char *cslot, int64_t rb,
                                          int64_t row, int byte_in_row, int RB)
{
    // the 16 bytes read lie within this CTA's rows (a narrow-row vector
    // covers several whole rows)
    if (!kpp_check(io.ctl,
                   row * RB + byte_in_row >= io.r0 * RB &&
                       row * RB + byte_in_row + 16 <= io.r1 * RB,
                   101))
        return make_uint4(0, 0, 0, 0);
    if (cslot)
        return lds16(cslot + (row - rb) * RB + byte_in_row);
    const char *g = io.gpts + row * RB + byte_in_row;
    return io.policy ? ld_global_hint(g, io.policy) : ld_stream16(g);
}

// The previous D^2 of an owned row, for D2_INPLACE prefetched together with
// the row's points (an L2 round trip that would otherwise stall the warp once
// per super-iteration); unused in pass 0 and for D2_SMEM.
template <int MODE>
__device__ __forceinline__ float prefetch_d2(const PassIO &io, int64_t row, bool in_range)
{
    if (MODE != D2_INPLACE || io.first || !in_range)
        return 0.f;
    if (!kpp_check(io.ctl, row >= io.r0 && row < io.r1, 102))
        return 0.f;
    return __ldcg(io.d2 + row);
}

// min-update of one owned row; returns the row's new D^2.  `pre` is the
// prefetched previous D^2 (D2_INPLACE).
template <int MODE>
__device__ __forceinline__ float update_d2(const PassIO &io, int64_t row, float v, float pre)
{
    if (!kpp_check(io.ctl, row >= io.r0 && row < io.r1, 103))
        return 0.f;
    float *slot = (MODE == D2_INPLACE) ? io.d2 + row : io.d2s + (row - io.r0);
    if (io.first) {
        *slot = v;
    } else {
        const float old = (MODE == D2_INPLACE) ? pre : *slot;
        if (v < old)
            *slot = v;
        else
            v = old;
    }
    if (MODE == D2_SMEM && io.d2_out)
        io.d2_out[row] = v;
    return v;
}

// One pass over rows [r0, r1) by all warps of the CTA, each over its own
// segment.  Loads are software-pipelined: the vectors of the next batch of
// rows are requested before the current batch is computed, so every warp
// keeps memory requests in flight continuously.  Writes the warp's segment
// sum and returns it (identical on all lanes of the warp).
template <int DT, int D, int L_, int MODE>
__device__ __forceinline__ Pair pass_rows(const PassIO &io, const CentreRegs<DT, D, L_> &cr)
{
    using G = Geom<DT, D, L_>;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int64_t seg_first, seg_last;
    segment_rows(io.r0, io.r1 - io.r0, G::SW, nwarps, warp, &seg_first, &seg_last);
    const int64_t nsup = (seg_last - seg_first + G::SW - 1) / G::SW;
    Pair lacc{};

    // super-iteration j of this warp: first row and shared-memory cache slot
    auto super_at = [&](int64_t j, int64_t &rb, char *&slot) {
        const int64_t jj = io.reverse ? (nsup - 1 - j) : j;
        rb = seg_first + jj * G::SW;
        slot = (io.cache != nullptr && jj < io.cache_supers)
                   ? io.cache + ((int64_t)warp * io.cache_supers + jj) * G::SW * G::RB
                   : nullptr;
    };

    if constexpr (G::WIDE) {
        // batch bi = slots [jb, jb + JB) of super-iteration bi / NB
        constexpr int NB = G::L / G::JB;
        const int g = lane / G::L, l = lane % G::L;
        const int64_t nbatch = nsup * NB;
        using Vecs = uint4[G::JB][G::VPL];
        using Scales = float[G::JB];
        auto issue = [&](int64_t bi, Vecs &x, Scales &sc, float &pre) {
            int64_t rb;
            char *slot;
            super_at(bi / NB, rb, slot);
            const int jb = (int)(bi % NB) * G::JB;
            const char *from = io.fill_cache ? nullptr : slot;
            const int64_t row0 = rb + (int64_t)jb * (32 / G::L) + g; // row of slot jb
            constexpr int QB = (32 / G::L) * G::RB;                   // bytes between slots
            pre = 0.f;
            if (jb + G::JB == G::L) { // last batch: the own row's previous D^2
                const int64_t own_row = rb + (int64_t)l * (32 / G::L) + g;
                pre = prefetch_d2<MODE>(io, own_row, own_row < seg_last);
            }
            if (rb + G::SW <= seg_last &&
                kpp_check(io.ctl,
                          row0 >= io.r0 && row0 + (int64_t)(G::JB - 1) * (32 / G::L) < io.r1, 104)) {
                // whole super-iteration in range: no bounds checks, one base
                // address and immediate offsets
                if (from) {
                    const char *p0 = from + (row0 - rb) * G::RB + l * 16;
#pragma unroll
                    for (int q = 0; q < G::JB; ++q)
#pragma unroll
                        for (int v = 0; v < G::VPL; ++v)
                            x[q][v] = lds16(p0 + q * QB + v * G::L * 16);
                } else {
                    const char *p0 = io.gpts + row0 * G::RB + l * 16;
#pragma unroll
                    for (int q = 0; q < G::JB; ++q)
#pragma unroll
                        for (int v = 0; v < G::VPL; ++v)
                            x[q][v] = io.policy ? ld_global_hint(p0 + q * QB + v * G::L * 16, io.policy)
                                                : ld_stream16(p0 + q * QB + v * G::L * 16);
                }
#pragma unroll
                for (int q = 0; q < G::JB; ++q)
                    sc[q] = (DT == KPP_FP8_E4M3) ? __ldg(io.scales + row0 + q * (32 / G::L)) : 1.0f;
                return;
            }
            if (rb + G::SW <= seg_last) { // only after a failed debug check
#pragma unroll
                for (int q = 0; q < G::JB; ++q) {
                    sc[q] = 1.0f;
#pragma unroll
                    for (int v = 0; v < G::VPL; ++v)
                        x[q][v] = make_uint4(0, 0, 0, 0);
                }
                return;
            }
#pragma unroll
            for (int q = 0; q < G::JB; ++q) {
                const int64_t row = row0 + (int64_t)q * (32 / G::L);
                const bool ok = row < seg_last;
                sc[q] = (DT == KPP_FP8_E4M3 && ok) ? __ldg(io.scales + row) : 1.0f;
#pragma unroll
                for (int v = 0; v < G::VPL; ++v)
                    x[q][v] = ok ? load_vec(io, from, rb, row, (v * G::L + l) * 16, G::RB)
                                 : make_uint4(0, 0, 0, 0);
            }
        };
        float mine = 0.f;
        auto consume = [&](int64_t bi, const Vecs &x, const Scales &sc, float pre) {
            int64_t rb;
            char *slot;
            super_at(bi / NB, rb, slot);
            const int jb = (int)(bi % NB) * G::JB;
            if (io.fill_cache && slot) {
#pragma unroll
                for (int q = 0; q < G::JB; ++q) {
                    const int64_t row = rb + (int64_t)(jb + q) * (32 / G::L) + g;
                    if (row < seg_last) {
#pragma unroll
                        for (int v = 0; v < G::VPL; ++v)
                            sts16(slot + (row - rb) * G::RB + (v * G::L + l) * 16, x[q][v]);
                    }
                }
            }
            float part[G::JB];
#pragma unroll
            for (int q = 0; q < G::JB; ++q) {
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int v = 0; v < G::VPL; ++v) {
                    float f[G::EPV];
                    decode16<DT>(x[q][v], f);
                    cr.template accum<G::EPV>(f, v * G::EPV, sc[q], a0, a1);
                }
                part[q] = a0 + a1;
            }
            if constexpr (G::JB == G::L) {
                // every slot of the row group is in this batch: reduce-scatter
                // over the L lanes sharing the rows -- halving the live slots
                // at each step, each lane keeping the half its bit selects --
                // leaves slot l's sum on lane l.  Each lane adds the same
                // partials in the same pairs as the butterfly below, so the
                // sums are bit-identical to it, with log2(L) shuffle rounds
                // for all L rows instead of log2(L) per row.
#pragma unroll
                for (int o = G::L / 2, n = G::JB; o > 0; o >>= 1, n >>= 1) {
                    const bool up = (l & o) != 0;
#pragma unroll
                    for (int i = 0; i < n / 2; ++i) {
                        const float send = up ? part[i] : part[i + n / 2];
                        const float keep = up ? part[i + n / 2] : part[i];
                        part[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                    }
                }
                mine = part[0];
            } else {
#pragma unroll
                for (int q = 0; q < G::JB; ++q) {
                    float sum = part[q];
#pragma unroll
                    for (int o = G::L / 2; o > 0; o >>= 1)
                        sum += __shfl_xor_sync(0xffffffffu, sum, o);
                    if (l == jb + q)
                        mine = sum;
                }
            }
            if (jb + G::JB == G::L) { // last batch of the super-iteration
                const int64_t own_row = rb + (int64_t)l * (32 / G::L) + g;
                if (own_row < seg_last)
                    lacc.add(update_d2<MODE>(io, own_row, mine, pre));
            }
        };
        // ring of PD batches: batch bi + PD - 1 is requested before batch bi
        // is computed
        constexpr int P = G::PD;
        Vecs x[P];
        Scales sc[P];
        float pre[P];
#pragma unroll
        for (int q = 0; q < P - 1; ++q)
            if (q < nbatch)
                issue(q, x[q], sc[q], pre[q]);
        for (int64_t bi = 0; bi < nbatch; bi += P) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int qn = (q + P - 1) % P;
                if (bi + q + P - 1 < nbatch)
                    issue(bi + q + P - 1, x[qn], sc[qn], pre[qn]);
                if (bi + q < nbatch)
                    consume(bi + q, x[q], sc[q], pre[q]);
            }
        }
    } else {
        // narrow rows: one 16-byte vector (RPV rows) per lane and super-iteration
        using Pre = float[G::RPV];
        auto issue = [&](int64_t j, uint4 &x, Pre &pre) {
            int64_t rb;
            char *slot;
            super_at(j, rb, slot);
            const int64_t own = rb + (int64_t)lane * G::RPV;
            x = (own + G::RPV <= seg_last)
                    ? load_vec(io, io.fill_cache ? nullptr : slot, rb, own, 0, G::RB)
                    : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int r = 0; r < G::RPV; ++r)
                pre[r] = prefetch_d2<MODE>(io, own + r, own + r < seg_last);
        };
        auto consume = [&](int64_t j, const uint4 &x, const Pre &pre) {
            int64_t rb;
            char *slot;
            super_at(j, rb, slot);
            const int64_t own_row = rb + (int64_t)lane * G::RPV;
            float f[G::EPV];
            float sc[G::RPV];
            if (own_row + G::RPV <= seg_last) {
                if (io.fill_cache && slot)
                    sts16(slot + (own_row - rb) * G::RB, x);
                decode16<DT>(x, f);
#pragma unroll
                for (int r = 0; r < G::RPV; ++r)
                    sc[r] = (DT == KPP_FP8_E4M3) ? __ldg(io.scales + own_row + r) : 1.0f;
            } else {
                // ragged tail of the segment: element loads from global memory,
                // never past its end (these rows are never cached)
#pragma unroll
                for (int r = 0; r < G::RPV; ++r) {
                    const int64_t row = own_row + r;
                    const bool ok = row < seg_last && kpp_check(io.ctl, row >= io.r0 && row < io.r1, 105);
                    sc[r] = (DT == KPP_FP8_E4M3 && ok) ? __ldg(io.scales + row) : 1.0f;
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        f[r * D + k] = ok ? decode1<DT>(io.gpts, row * D + k) : 0.f;
                }
            }
#pragma unroll
            for (int r = 0; r < G::RPV; ++r) {
                float a0 = 0.f, a1 = 0.f;
                cr.template accum<D>(f + r * D, r * D, sc[r], a0, a1);
                const int64_t row = own_row + r;
                if (row < seg_last)
                    lacc.add(update_d2<MODE>(io, row, a0 + a1, pre[r]));
            }
        };
        constexpr int P = G::PD;
        uint4 x[P];
        Pre pre[P];
#pragma unroll
        for (int q = 0; q < P - 1; ++q)
            if (q < nsup)
                issue(q, x[q], pre[q]);
        for (int64_t j = 0; j < nsup; j += P) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int qn = (q + P - 1) % P;
                if (j + q + P - 1 < nsup)
                    issue(j + q + P - 1, x[qn], pre[qn]);
                if (j + q < nsup)
                    consume(j + q, x[q], pre[q]);
            }
        }
    }
    const Pair seg = warp_pair_sum(lacc);
    if (lane == 0)
        io.segs[warp] = make_float2(seg.hi, seg.lo);
    return seg;
}

// The CTA's D^2 sum: warp pairs added in warp order, rounded once to FP64.
// All threads return it.  `sh` holds 2 floats per warp.
__device__ __forceinline__ double cta_sum(const Pair &wacc, float *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[2 * warp] = wacc.hi;
        sh[2 * warp + 1] = wacc.lo;
    }
    __syncthreads();
    Pair t{};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        Pair q;
        q.hi = sh[2 * w];
        q.lo = sh[2 * w + 1];
        t.add(q);
    }
    return t.value();
}

// Generic pass for any d and any row alignment: one thread per row, element
// loads, centre in shared memory (c_sh[0..d) = c_hi, c_sh[d..2d) = c_lo for
// FP8).  Segments as in pass_rows with 32-row super-iterations.
template <int DT>
__device__ __forceinline__ Pair pass_rows_generic(const PassIO &io, int d, const float *c_sh)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int64_t seg_first, seg_last;
    segment_rows(io.r0, io.r1 - io.r0, 32, nwarps, warp, &seg_first, &seg_last);
    Pair lacc{};
    for (int64_t row = seg_first + lane; row < seg_last; row += 32) {
        const float sc = (DT == KPP_FP8_E4M3) ? __ldg(io.scales + row) : 1.0f;
        float a0 = 0.f, a1 = 0.f;
        int k = 0;
        for (; k + 1 < d; k += 2) {
            float q0 = decode1<DT>(io.gpts, row * d + k);
            float q1 = decode1<DT>(io.gpts, row * d + k + 1);
            float t0, t1;
            if constexpr (DT == KPP_FP8_E4M3) {
                t0 = diff_fp8(sc, q0, c_sh[k], c_sh[d + k]);
                t1 = diff_fp8(sc, q1, c_sh[k + 1], c_sh[d + k + 1]);
            } else {
                t0 = q0 - c_sh[k];
                t1 = q1 - c_sh[k + 1];
            }
            a0 = fmaf(t0, t0, a0);
            a1 = fmaf(t1, t1, a1);
        }
        if (k < d) {
            float q0 = decode1<DT>(io.gpts, row * d + k);
            float t0 = (DT == KPP_FP8_E4M3) ? diff_fp8(sc, q0, c_sh[k], c_sh[d + k])
                                            : q0 - c_sh[k];
            a0 = fmaf(t0, t0, a0);
        }
        lacc.add(update_d2<D2_INPLACE>(io, row, a0 + a1, prefetch_d2<D2_INPLACE>(io, row, true)));
    }
    const Pair seg = warp_pair_sum(lacc);
    if (lane == 0)
        io.segs[warp] = make_float2(seg.hi, seg.lo);
    return seg;
}

template <int DT>
__device__ __forceinline__ void load_centre_smem(const void *points, const float *scales,
                                                 int64_t ci, int d, float *c_sh)
{
    const float s = (DT == KPP_FP8_E4M3) ? __ldg(scales + ci) : 1.0f;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        const float q = decode1<DT>(points, ci * d + k);
        if constexpr (DT == KPP_FP8_E4M3)
            split_fp8_centre(s, q, c_sh[k], c_sh[d + k]);
        else
            c_sh[k] = q;
    }
}

} // namespace kpp

// kpp_pass.cuh -- the per-point work of one seeding pass, shared by the
// streamed and persistent forms: distance of every point of a contiguous
// row range to the newest centre (difference form, FP32 FMA), in-place
// min-update of D^2, and the range's D^2 sum (FP32 two-sum per lane, FP64
// across lanes).  Algorithm 1/2: d_{m,l} = d(H_m, n_l), d_sn = min over
// seeds of the squared distance.
#pragma once

#include "kpp_device.cuh"

namespace kpp {

// Geometry of one (dtype, d, lanes-per-row) specialisation.
//   WIDE rows (>= 16 bytes): L lanes share a row, each lane reading VPL
//     16-byte vectors of it; a warp covers 32 rows per super-iteration and
//     lane (g, l) ends up owning row base + l * (32 / L) + g.
//   Narrow rows (< 16 bytes): one 16-byte vector holds RPV whole rows; a
//     lane owns RPV consecutive rows and a warp covers 32 * RPV rows.
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
    // slots per unrolled batch, so at most 8 vectors per lane are in flight
    static constexpr int JB = WIDE ? ((8 / VPL) < 1 ? 1 : ((8 / VPL) > L ? L : (8 / VPL))) : 1;
    static_assert(!WIDE || (RB % 16 == 0), "wide rows are whole vectors");
    static_assert(!WIDE || (VPR % L == 0 && L >= 1 && L <= 32 && (L & (L - 1)) == 0),
                  "lanes per row must divide the row's vectors");
    static_assert(WIDE || (16 % RB == 0), "narrow rows tile a vector");
    static_assert(!WIDE || (L % JB == 0), "slot batches tile the slots");
};

// Per-lane slice of the newest centre, decoded to FP32 once per pass.
template <int DT, int D, int L_>
struct CentreRegs {
    using G = Geom<DT, D, L_>;
    float c[G::CREG];

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
                decode16<DT>(x, sc, c + v * G::EPV);
            }
        } else {
            float tmp[D];
#pragma unroll
            for (int k = 0; k < D; ++k)
                tmp[k] = decode1<DT>(points, ci * D + k, sc);
#pragma unroll
            for (int e = 0; e < G::EPV; ++e)
                c[e] = tmp[e % D];
        }
    }
};

// One pass over rows [row_begin, row_end) by all warps of the CTA.
// m == 0 writes D^2 (the initial infinity makes the min a plain store);
// m > 0 stores only where D^2 decreases.  Returns this thread's share of
// the range's D^2 sum.
template <int DT, int D, int L_>
__device__ __forceinline__ Acc2 pass_rows(const void *points, const float *scales, float *d2,
                                          int64_t row_begin, int64_t row_end, bool first_pass,
                                          const CentreRegs<DT, D, L_> &cr)
{
    using G = Geom<DT, D, L_>;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const char *base_ptr = reinterpret_cast<const char *>(points);
    Acc2 acc;

    for (int64_t rb = row_begin + (int64_t)warp * G::SW; rb < row_end;
         rb += (int64_t)nwarps * G::SW) {
        float mine[G::RPV];
        int64_t own_row;
        if constexpr (G::WIDE) {
            const int g = lane / G::L, l = lane % G::L;
            mine[0] = 0.f;
#pragma unroll 1
            for (int jb = 0; jb < G::L; jb += G::JB) {
                uint4 x[G::JB][G::VPL];
                float sc[G::JB];
#pragma unroll
                for (int jj = 0; jj < G::JB; ++jj) {
                    const int64_t row = rb + (int64_t)(jb + jj) * (32 / G::L) + g;
                    const bool ok = row < row_end;
                    sc[jj] = (DT == KPP_FP8_E4M3 && ok) ? __ldg(scales + row) : 1.0f;
#pragma unroll
                    for (int v = 0; v < G::VPL; ++v)
                        x[jj][v] = ok ? ld_stream16(base_ptr + row * G::RB + (v * G::L + l) * 16)
                                      : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int jj = 0; jj < G::JB; ++jj) {
                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                    for (int v = 0; v < G::VPL; ++v) {
                        float f[G::EPV];
                        decode16<DT>(x[jj][v], sc[jj], f);
#pragma unroll
                        for (int e = 0; e < G::EPV; e += 2) {
                            float t0 = f[e] - cr.c[v * G::EPV + e];
                            float t1 = f[e + 1] - cr.c[v * G::EPV + e + 1];
                            a0 = fmaf(t0, t0, a0);
                            a1 = fmaf(t1, t1, a1);
                        }
                    }
                    float part = a0 + a1;
#pragma unroll
                    for (int o = G::L / 2; o > 0; o >>= 1)
                        part += __shfl_xor_sync(0xffffffffu, part, o);
                    if (l == jb + jj)
                        mine[0] = part;
                }
            }
            own_row = rb + (int64_t)l * (32 / G::L) + g;
        } else {
            own_row = rb + (int64_t)lane * G::RPV;
            float f[G::EPV];
            if (own_row + G::RPV <= row_end) {
                uint4 x = ld_stream16(base_ptr + own_row * G::RB);
                decode16<DT>(x, 1.0f, f);
                if constexpr (DT == KPP_FP8_E4M3) {
#pragma unroll
                    for (int r = 0; r < G::RPV; ++r) {
                        const float s = __ldg(scales + own_row + r);
#pragma unroll
                        for (int k = 0; k < D; ++k)
                            f[r * D + k] = __fmul_rn(s, f[r * D + k]);
                    }
                }
            } else {
                // ragged tail: element loads, never past row_end
#pragma unroll
                for (int r = 0; r < G::RPV; ++r) {
                    const int64_t row = own_row + r;
                    const float s = (DT == KPP_FP8_E4M3 && row < row_end) ? __ldg(scales + row) : 1.0f;
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        f[r * D + k] = row < row_end ? decode1<DT>(points, row * D + k, s) : 0.f;
                }
            }
#pragma unroll
            for (int r = 0; r < G::RPV; ++r) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    float t = f[r * D + k] - cr.c[r * D + k];
                    a = fmaf(t, t, a);
                }
                mine[r] = a;
            }
        }
        // min-update of the rows this lane owns, and their sum
#pragma unroll
        for (int r = 0; r < G::RPV; ++r) {
            const int64_t row = own_row + r;
            if (row < row_end) {
                float v = mine[r];
                if (first_pass) {
                    d2[row] = v;
                } else {
                    const float old = d2[row];
                    if (v < old)
                        d2[row] = v;
                    else
                        v = old;
                }
                acc.add(v);
            }
        }
    }
    return acc;
}

// Generic pass for any d and any row alignment: one thread per row, element
// loads, centre in shared memory (`c_sh`, d floats).  Used when no
// specialisation for (dtype, d) is built.
template <int DT>
__device__ __forceinline__ Acc2 pass_rows_generic(const void *points, const float *scales,
                                                  float *d2, int64_t row_begin, int64_t row_end,
                                                  int d, bool first_pass, const float *c_sh)
{
    Acc2 acc;
    for (int64_t row = row_begin + threadIdx.x; row < row_end; row += blockDim.x) {
        const float s = (DT == KPP_FP8_E4M3) ? __ldg(scales + row) : 1.0f;
        float a0 = 0.f, a1 = 0.f;
        int k = 0;
        for (; k + 1 < d; k += 2) {
            float t0 = decode1<DT>(points, row * d + k, s) - c_sh[k];
            float t1 = decode1<DT>(points, row * d + k + 1, s) - c_sh[k + 1];
            a0 = fmaf(t0, t0, a0);
            a1 = fmaf(t1, t1, a1);
        }
        if (k < d) {
            float t0 = decode1<DT>(points, row * d + k, s) - c_sh[k];
            a0 = fmaf(t0, t0, a0);
        }
        float v = a0 + a1;
        if (first_pass) {
            d2[row] = v;
        } else {
            const float old = d2[row];
            if (v < old)
                d2[row] = v;
            else
                v = old;
        }
        acc.add(v);
    }
    return acc;
}

template <int DT>
__device__ __forceinline__ void load_centre_smem(const void *points, const float *scales,
                                                 int64_t ci, int d, float *c_sh)
{
    const float s = (DT == KPP_FP8_E4M3) ? __ldg(scales + ci) : 1.0f;
    for (int k = threadIdx.x; k < d; k += blockDim.x)
        c_sh[k] = decode1<DT>(points, ci * d + k, s);
}

} // namespace kpp

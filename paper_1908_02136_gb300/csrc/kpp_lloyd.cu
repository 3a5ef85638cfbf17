// kpp_lloyd.cu -- one Lloyd iteration on the GPU: the clustering stage the
// seeds are for (Section II: "the clustering part is implemented the same as
// the K-means algorithm", i.e. Lloyd's nearest-centre assignment followed by
// moving every centre to the mean of its points).
//
// Assignment is a dense contraction: the nearest centre of x minimises
// |c|^2 - 2 x.c, so the N x K dot products run on the tensor cores
// (tcgen05.mma, BF16 operands staged by TMA, FP32 accumulators in tensor
// memory).  To keep close to FP32 accuracy every operand is split into two
// BF16 planes, v = hi + lo with hi = bf16(v) and lo = bf16(v - hi), and the
// product is hi.hi + hi.lo + lo.hi (the dropped lo.lo term is ~2^-16 of the
// whole).  The epilogue reads the accumulators from tensor memory and keeps
// the running minimum of |c_k|^2 - 2 x.c_k per point (smallest k on ties).
// Two kernels compute it: one on pairs of SMs sharing each MMA (cta_group::2,
// 256 x 256 tiles; the default) and one on single SMs (128 x 128 tiles; where
// no cluster of two can be launched).
//
// The update reads the FP32 points again: the exact squared distance to the
// assigned centre in the same FP32 difference form as the seeding pass, the
// cost phi, and per-centre sums (FP32 per CTA in shared memory, FP64 across
// CTAs) and counts; centres with no point keep their position.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "kpp.h"
#include "kpp_internal.h"
#include "kpp_tc.cuh"

namespace kpp {
namespace {

constexpr int kBM = 128;      // points per tile: TMEM lanes of an accumulator
constexpr int kMT = 2;        // point tiles served by each pass over the centres
constexpr int kBN = 128;      // centres per tile: accumulator columns
constexpr int kBK = 64;       // features per chunk: one 128-byte swizzled row of BF16
constexpr int kMaxD = 128;    // d <= 128 (at most two chunks)
constexpr int kMaxK = 4096;   // centre norms stay in shared memory
constexpr int kThreads = 256; // warp 0 TMA, warp 1 MMA, warp 2 TMEM, warps 4-7 epilogue
constexpr int kMaxStages = 4; // centre-tile stages in flight
constexpr uint32_t kTmemCols = 2 * kMT * kBN; // [buffer][point tile] accumulators: 512
constexpr uint32_t kABytes = kBM * kBK * 2; // one plane, one chunk: 16 KB
constexpr uint32_t kBBytes = kBN * kBK * 2; // 16 KB
// The CTA-pair form: 256-point x 256-centre tiles over two SMs, each CTA
// holding 128 points and 128 centres (one kBBytes plane each) of a tile.
constexpr int kPN = 256;     // centres per tile: accumulator columns in each CTA
constexpr int kPNH = kPN / 2; // centres per tile held by each CTA
constexpr int kMaxStagesPair = 8;
constexpr size_t kAlign = 256;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    int dp;   // padded feature count (64 or 128)
    int grid; // CTAs of the per-point kernels
    size_t off_phi, off_plo, off_chi, off_clo, off_cn, off_sums, off_counts, off_partial, bytes;
};

bool shape_ok(int64_t N, int32_t d, int32_t K)
{
    return N >= 1 && N < (int64_t(1) << 31) && d >= 1 && d <= kMaxD && K >= 1 && K <= kMaxK &&
           K <= N;
}

Layout layout(int64_t N, int32_t d, int32_t K)
{
    Layout L;
    L.dp = d <= 64 ? 64 : 128;
    L.grid = 1024;
    size_t off = sizeof(Control);
    L.off_phi = off = round_up(off, kAlign);
    off += (size_t)N * L.dp * 2;
    L.off_plo = off = round_up(off, kAlign);
    off += (size_t)N * L.dp * 2;
    L.off_chi = off = round_up(off, kAlign);
    off += (size_t)K * L.dp * 2;
    L.off_clo = off = round_up(off, kAlign);
    off += (size_t)K * L.dp * 2;
    L.off_cn = off = round_up(off, kAlign);
    off += (size_t)K * 4;
    L.off_sums = off = round_up(off, kAlign);
    off += (size_t)K * d * 8;
    L.off_counts = off = round_up(off, kAlign);
    off += (size_t)K * 8;
    L.off_partial = off = round_up(off, kAlign);
    off += (size_t)L.grid * 8;
    L.bytes = round_up(off, kAlign);
    return L;
}

// ---------------------------------------------------------------------------
// Splitting into BF16 planes (zero-padded to dp features).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// A thread per (row, group of 8 features): eight FP32 loads, one 16-byte
// store per plane.  dp / 8 is 8 or 16, so the indexing is shifts and masks.
__device__ __forceinline__ void split_rows_body(const float *x, int64_t rows, int d, int dp,
                                                __nv_bfloat16 *hi, __nv_bfloat16 *lo)
{
    const int sh = dp == 64 ? 3 : 4;
    const int64_t n = rows << sh;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = g >> sh;
        const int j0 = (int)(g & ((1 << sh) - 1)) << 3;
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = j0 + u;
            split_bf16(j < d ? x[r * d + j] : 0.f, h[u], l[u]);
        }
        *reinterpret_cast<uint4 *>(hi + r * dp + j0) = *reinterpret_cast<const uint4 *>(h);
        *reinterpret_cast<uint4 *>(lo + r * dp + j0) = *reinterpret_cast<const uint4 *>(l);
    }
}

__global__ void split_rows_kernel(const float *x, int64_t rows, int d, int dp, __nv_bfloat16 *hi,
                                  __nv_bfloat16 *lo)
{
    split_rows_body(x, rows, d, dp, hi, lo);
}

// The same for rows [*row0, *row0 + *rows) of `base`, counts read on the device.
__global__ void split_rows_dev_kernel(const float *base, const long long *row0,
                                      const int32_t *rows, int d, int dp, __nv_bfloat16 *hi,
                                      __nv_bfloat16 *lo)
{
    split_rows_body(base + *row0 * d, *rows, d, dp, hi, lo);
}

// |c_k|^2 in FP32 (one thread per centre); the device-count form reads K and
// the first row from device memory.
__device__ __forceinline__ void centre_norm(const float *c, int k, int d, float *cn)
{
    float s = 0.f;
    for (int j = 0; j < d; ++j)
        s = fmaf(c[(int64_t)k * d + j], c[(int64_t)k * d + j], s);
    cn[k] = s;
}

__global__ void centre_norms_kernel(const float *c, int K, int d, float *cn)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K)
        centre_norm(c, k, d, cn);
}

__global__ void centre_norms_dev_kernel(const float *base, const long long *row0,
                                        const int32_t *K, int d, float *cn)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < *K)
        centre_norm(base + *row0 * d, k, d, cn);
}

// ---------------------------------------------------------------------------
// Assignment on the tensor cores.
// ---------------------------------------------------------------------------
struct AssignArgs {
    int64_t N;
    int32_t K;
    const int32_t *Kdev; // if set, K is read here (written by an earlier launch)
    int32_t nk;     // feature chunks (dp / 64)
    int32_t stages; // centre-tile stages in shared memory
    int32_t abufs;  // point-tile buffers (2: the next group's load overlaps this one)
    const float *cn;
    int32_t *labels;
    Control *ctl;
    uint64_t timeout_ns;
};

// The smallest of 32 scores and its position, the first one on ties: a
// tournament in which the later of two entries wins only when strictly
// smaller.  Depth 5 instead of a 32-long chain of dependent compares, so the
// four epilogue warps keep their issue slots busy.
__device__ __forceinline__ float block_argmin32(float (&w)[32], int &wi)
{
    int id[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const bool p = w[2 * j + 1] < w[2 * j];
        w[j] = p ? w[2 * j + 1] : w[2 * j];
        id[j] = 2 * j + (p ? 1 : 0);
    }
#pragma unroll
    for (int n = 8; n >= 1; n >>= 1) {
#pragma unroll
        for (int j = 0; j < n; ++j) {
            const bool p = w[2 * j + 1] < w[2 * j];
            w[j] = p ? w[2 * j + 1] : w[2 * j];
            id[j] = p ? id[2 * j + 1] : id[2 * j];
        }
    }
    wi = id[0];
    return w[0];
}

// The 32 scores |c_k|^2 - 2 x.c_k of a block from the accumulators `acc`
// (x.c_k, FP32 bits) and the norms `n4` (eight float4), two per packed FP32
// fma (each lane rounded as fmaf(-2, x.c, |c|^2)).
__device__ __forceinline__ void block_scores32(const uint32_t (&acc)[32], const float4 *n4,
                                               float (&w)[32])
{
    const uint64_t m2 = 0xC0000000C0000000ull; // {-2.f, -2.f}
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const float4 n = n4[v];
        uint64_t a01, a23, n01, n23, s01, s23;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a01) : "r"(acc[4 * v + 0]), "r"(acc[4 * v + 1]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(a23) : "r"(acc[4 * v + 2]), "r"(acc[4 * v + 3]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(n01) : "f"(n.x), "f"(n.y));
        asm("mov.b64 %0, {%1, %2};" : "=l"(n23) : "f"(n.z), "f"(n.w));
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(s01) : "l"(m2), "l"(a01), "l"(n01));
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(s23) : "l"(m2), "l"(a23), "l"(n23));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(w[4 * v + 0]), "=f"(w[4 * v + 1]) : "l"(s01));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(w[4 * v + 2]), "=f"(w[4 * v + 3]) : "l"(s23));
    }
}

__device__ __forceinline__ uint32_t dynamic_smem_bytes()
{
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void fail(Control *ctl, volatile int *abort_flag)
{
    *abort_flag = 1;
    atomicCAS(&ctl->status, KPP_OK, KPP_ERR_TIMEOUT);
}

// Persistent over groups of kMT 128-point tiles.  Per group the producer
// loads both BF16 planes of its points once, then streams both planes of
// every 128-centre tile, one 64-feature chunk at a time, through a ring of
// shared-memory stages; each stage feeds the MMAs of all kMT point tiles, so
// a centre byte read from L2 serves 256 points.  The MMA thread accumulates
// hi.hi + hi.lo + lo.hi into one of two sets of tensor-memory accumulators;
// the four epilogue warps turn a finished set into running argmins (a
// tournament per 32-column block, then one compare per block) while the
// next one fills.  Every wait is bounded: on a timeout the kernel records
// KPP_ERR_TIMEOUT, lets the copies and MMAs already issued finish (again
// bounded), frees its tensor memory and returns.
__global__ void __launch_bounds__(kThreads, 1)
    lloyd_assign_kernel(const __grid_constant__ CUtensorMap map_phi,
                        const __grid_constant__ CUtensorMap map_plo,
                        const __grid_constant__ CUtensorMap map_chi,
                        const __grid_constant__ CUtensorMap map_clo, AssignArgs a)
{
    using namespace tc;
    const int K = a.Kdev ? *a.Kdev : a.K;
    if (K <= 0)
        return; // nothing to assign (every thread leaves before any setup)
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    const int NS = a.stages;
    const uint32_t abytes = kMT * 2 * a.nk * kABytes; // one group's point tiles
    uint8_t *sA = smem;                              // [buffer][tile][plane][chunk] 16 KB each
    uint8_t *sB = smem + a.abufs * abytes;           // [stage][plane] 16 KB each
    float *s_cn = reinterpret_cast<float *>(sB + NS * 2 * kBBytes);
    // debug build: the host's plan fits this launch (every thread, before
    // any barrier or tensor memory is set up)
    if (!kpp_check(a.ctl,
                   NS >= 2 && NS <= kMaxStages && (a.abufs == 1 || a.abufs == 2) &&
                       (size_t)(reinterpret_cast<uint8_t *>(s_cn) - smem_raw) +
                               (size_t)((K + kBN - 1) / kBN) * kBN * 4 <=
                           dynamic_smem_bytes(),
                   501))
        return;
    __shared__ uint64_t a_full[2], a_empty[2], b_full[kMaxStages], b_empty[kMaxStages], acc_full[2],
        acc_empty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    auto a_tile = [&](uint32_t b, int t, int plane, int k) {
        return sA + b * abytes + ((t * 2 + plane) * a.nk + k) * kABytes;
    };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        for (int s = 0; s < NS; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], kBM);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    // centre norms, padded with +infinity up to whole centre tiles (those
    // columns can never win)
    const int n_ct = (K + kBN - 1) / kBN;
    for (int k = threadIdx.x; k < n_ct * kBN; k += blockDim.x)
        s_cn[k] = k < K ? a.cn[k] : __int_as_float(0x7f800000);
    if (warp == 2)
        tmem_alloc(&tmem_base, kTmemCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();

    const int64_t n_mt = (a.N + kBM - 1) / kBM;
    const int64_t n_grp = (n_mt + kMT - 1) / kMT;
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- producer ----
        uint32_t it = 0, g = 0;
        uint32_t a_pending[2] = {}; // 1 + use of the last point load per buffer
        uint32_t b_pending[kMaxStages] = {}; // 1 + use of the last centre load per stage
        for (int64_t gp = blockIdx.x; gp < n_grp && !abort_flag; gp += gridDim.x, ++it) {
            const uint32_t ab = it % a.abufs, ause = it / a.abufs;
            if (ause > 0 && !mbar_wait(&a_empty[ab], (ause - 1) & 1, a.timeout_ns)) {
                fail(a.ctl, &abort_flag);
                break;
            }
            mbar_expect_tx(&a_full[ab], abytes);
            for (int t = 0; t < kMT; ++t) {
                const int y = (int)((gp * kMT + t) * kBM);
                for (int k = 0; k < a.nk; ++k) {
                    tma_load_2d(a_tile(ab, t, 0, k), &map_phi, &a_full[ab], k * kBK, y);
                    tma_load_2d(a_tile(ab, t, 1, k), &map_plo, &a_full[ab], k * kBK, y);
                }
            }
            a_pending[ab] = ause + 1;
            for (int ct = 0; ct < n_ct && !abort_flag; ++ct) {
                for (int k = 0; k < a.nk; ++k, ++g) {
                    const uint32_t s = g % NS, use = g / NS;
                    if (use > 0 && !mbar_wait(&b_empty[s], (use - 1) & 1, a.timeout_ns)) {
                        fail(a.ctl, &abort_flag);
                        break;
                    }
                    mbar_expect_tx(&b_full[s], 2 * kBBytes);
                    tma_load_2d(sB + (s * 2 + 0) * kBBytes, &map_chi, &b_full[s], k * kBK, ct * kBN);
                    tma_load_2d(sB + (s * 2 + 1) * kBBytes, &map_clo, &b_full[s], k * kBK, ct * kBN);
                    b_pending[s] = use + 1;
                }
            }
        }
        if (abort_flag) {
            // let the copies already issued land before the CTA exits
            for (int b = 0; b < 2; ++b)
                if (a_pending[b])
                    mbar_wait(&a_full[b], (a_pending[b] - 1) & 1, a.timeout_ns);
            for (int s = 0; s < NS; ++s)
                if (b_pending[s])
                    mbar_wait(&b_full[s], (b_pending[s] - 1) & 1, a.timeout_ns);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        const uint32_t idesc = idesc_bf16_f32(kBM, kBN);
        uint32_t it = 0, g = 0, t = 0;
        bool issued = false;
        for (int64_t gp = blockIdx.x; gp < n_grp && !abort_flag; gp += gridDim.x, ++it) {
            const uint32_t ab = it % a.abufs, ause = it / a.abufs;
            if (!mbar_wait(&a_full[ab], ause & 1, a.timeout_ns)) {
                fail(a.ctl, &abort_flag);
                break;
            }
            fence_after_sync();
            for (int ct = 0; ct < n_ct && !abort_flag; ++ct, ++t) {
                const uint32_t buf = t & 1, ause = t >> 1;
                if (ause > 0 && !mbar_wait(&acc_empty[buf], (ause - 1) & 1, a.timeout_ns)) {
                    fail(a.ctl, &abort_flag);
                    break;
                }
                fence_after_sync();
                for (int k = 0; k < a.nk; ++k, ++g) {
                    const uint32_t s = g % NS, use = g / NS;
                    if (!mbar_wait(&b_full[s], use & 1, a.timeout_ns)) {
                        fail(a.ctl, &abort_flag);
                        break;
                    }
                    fence_after_sync();
                    const uint32_t bh = smem_u32(sB + (s * 2 + 0) * kBBytes);
                    const uint32_t bl = smem_u32(sB + (s * 2 + 1) * kBBytes);
#pragma unroll
                    for (int mt = 0; mt < kMT; ++mt) {
                        const uint32_t d_tmem = tmem + (buf * kMT + mt) * kBN;
                        const uint32_t ah = smem_u32(a_tile(ab, mt, 0, k));
                        const uint32_t al = smem_u32(a_tile(ab, mt, 1, k));
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            // one MMA covers 16 features = 32 bytes of the swizzled row
                            const uint32_t o = kk * 32;
                            mma_bf16(d_tmem, sdesc_k_sw128(ah + o), sdesc_k_sw128(bh + o), idesc,
                                     (k | kk) ? 1u : 0u);
                            mma_bf16(d_tmem, sdesc_k_sw128(ah + o), sdesc_k_sw128(bl + o), idesc, 1u);
                            mma_bf16(d_tmem, sdesc_k_sw128(al + o), sdesc_k_sw128(bh + o), idesc, 1u);
                        }
                    }
                    issued = true;
                    mma_commit(&b_empty[s]); // stage s is free once these are done
                }
                if (abort_flag)
                    break;
                mma_commit(&acc_full[buf]);
            }
            if (abort_flag)
                break;
            mma_commit(&a_empty[ab]);
        }
        // every MMA issued has completed before the tensor memory is freed
        if (issued) {
            mma_commit(&done);
            mbar_wait(&done, 0, a.timeout_ns);
        }
    } else if (warp >= 4) {
        // ---- epilogue: argmin of |c|^2 - 2 x.c over the centres ----
        const int q = warp & 3; // this warp's quarter of the TMEM lanes
        const int row_local = q * 32 + lane;
        uint32_t t = 0;
        for (int64_t gp = blockIdx.x; gp < n_grp && !abort_flag; gp += gridDim.x) {
            float best[kMT];
            int bk[kMT];
#pragma unroll
            for (int mt = 0; mt < kMT; ++mt) {
                best[mt] = __int_as_float(0x7f800000);
                bk[mt] = 0;
            }
            for (int ct = 0; ct < n_ct; ++ct, ++t) {
                const uint32_t buf = t & 1, use = t >> 1;
                if (!mbar_wait(&acc_full[buf], use & 1, a.timeout_ns)) {
                    fail(a.ctl, &abort_flag);
                    break;
                }
                fence_after_sync();
                const float4 *cn4 = reinterpret_cast<const float4 *>(s_cn + ct * kBN);
#pragma unroll
                for (int mt = 0; mt < kMT; ++mt) {
                    const uint32_t base = tmem + (buf * kMT + mt) * kBN + ((uint32_t)(q * 32) << 16);
                    // the tile's 128 columns, two loads in flight at a time
#pragma unroll 1
                    for (int h = 0; h < 4; h += 2) {
                        uint32_t r[2][32];
                        tmem_ld32_async(base + h * 32, r[0]);
                        tmem_ld32_async(base + h * 32 + 32, r[1]);
                        tmem_ld_wait();
                        tmem_regs_ready(r[0]);
                        tmem_regs_ready(r[1]);
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            float w[32];
                            block_scores32(r[c], cn4 + (h + c) * 8, w);
                            int wi;
                            const float m = block_argmin32(w, wi);
                            if (m < best[mt]) { // earlier blocks win ties
                                best[mt] = m;
                                bk[mt] = ct * kBN + (h + c) * 32 + wi;
                            }
                        }
                    }
                }
                fence_before_sync();
                mbar_arrive(&acc_empty[buf]);
            }
            if (abort_flag)
                break;
#pragma unroll
            for (int mt = 0; mt < kMT; ++mt) {
                const int64_t row = (gp * kMT + mt) * kBM + row_local;
                if (row < a.N)
                    a.labels[row] = bk[mt];
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 2) {
        fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// The same assignment on CTA pairs (clusters of two CTAs on neighbouring
// SMs).  One thread of the even CTA issues tcgen05.mma.cta_group::2 with
// M = N = 256: A is the two CTAs' own 128-point tiles, B a 256-centre tile of
// which each CTA holds half (centres 0-127 of the tile in the even CTA,
// 128-255 in the odd one), and each CTA's tensor memory receives its points'
// 256 scores.  Per SM every MMA then does 128 x 256 x 16 multiply-adds from
// 8 KB of shared-memory operands (the one-SM form's 128 x 128 x 16 MMAs
// read as much for half the work), and half as many MMAs are issued.
//
// Protocol: both CTAs' loads complete on the even CTA's full barriers (which
// its producer arms with the pair's byte count); each MMA commit arrives on
// the barrier at the same offset in both CTAs (stage free, accumulator
// ready, point buffer free); each epilogue warp of either CTA releases an
// accumulator with one arrival on the even CTA's barrier.  Every wait is
// bounded; after a timeout the MMAs already issued are drained, loads in
// flight are given 200 us to land, and the pair frees its tensor memory
// together.
__global__ void __launch_bounds__(kThreads, 1)
    lloyd_assign_pair_kernel(const __grid_constant__ CUtensorMap map_phi,
                             const __grid_constant__ CUtensorMap map_plo,
                             const __grid_constant__ CUtensorMap map_chi,
                             const __grid_constant__ CUtensorMap map_clo, AssignArgs a)
{
    using namespace tc;
    const int K = a.Kdev ? *a.Kdev : a.K;
    if (K <= 0)
        return; // nothing to assign (every thread of every CTA leaves before any setup)
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    const int NS = a.stages;
    const uint32_t abytes = 2 * a.nk * kABytes; // this CTA's point tile, both planes
    uint8_t *sA = smem;                         // [buffer][plane][chunk] 16 KB each
    uint8_t *sB = smem + a.abufs * abytes;      // [stage][plane] 16 KB each
    float *s_cn = reinterpret_cast<float *>(sB + NS * 2 * kBBytes);
    // debug build: the host's plan fits this launch (every thread of both
    // CTAs takes the same branch, before any cluster barrier or allocation)
    if (!kpp_check(a.ctl,
                   NS >= 2 && NS <= kMaxStagesPair && (a.abufs == 1 || a.abufs == 2) &&
                       (size_t)(reinterpret_cast<uint8_t *>(s_cn) - smem_raw) +
                               (size_t)((K + kPN - 1) / kPN) * kPN * 4 <=
                           dynamic_smem_bytes(),
                   502))
        return;
    __shared__ uint64_t a_full[2], a_empty[2], b_full[kMaxStagesPair], b_empty[kMaxStagesPair],
        acc_full[2], acc_empty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    auto a_tile = [&](uint32_t b, int plane, int k) {
        return sA + b * abytes + (plane * a.nk + k) * kABytes;
    };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank(); // 0 issues the MMAs
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 2 * 4); // each epilogue warp of both CTAs
        }
        for (int s = 0; s < NS; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    const int n_ct = (K + kPN - 1) / kPN;
    for (int k = threadIdx.x; k < n_ct * kPN; k += blockDim.x)
        s_cn[k] = k < K ? a.cn[k] : __int_as_float(0x7f800000);
    // both CTAs running with their barriers initialised before any signal
    // crosses between them and before they allocate tensor memory together
    cluster_sync();
    if (warp == 2)
        tmem_alloc_pair(&tmem_base, kTmemCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();

    const int64_t n_mt = (a.N + kBM - 1) / kBM;
    const int64_t n_grp = (n_mt + 1) / 2; // 256-point groups of the pair
    const int64_t cl0 = cluster_id_x(), ncl = n_clusters_x();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- producer (both CTAs): own point tile, own half of each centre tile ----
        uint32_t it = 0, g = 0;
        for (int64_t gp = cl0; gp < n_grp && !abort_flag; gp += ncl, ++it) {
            const uint32_t ab = it % a.abufs, ause = it / a.abufs;
            if (ause > 0 && !mbar_wait_cluster(&a_empty[ab], (ause - 1) & 1, a.timeout_ns)) {
                fail(a.ctl, &abort_flag);
                break;
            }
            if (rank == 0)
                mbar_expect_tx(&a_full[ab], 2 * abytes);
            const uint32_t fa = mapa(smem_u32(&a_full[ab]), 0);
            const int y = (int)((gp * 2 + rank) * kBM);
            for (int k = 0; k < a.nk; ++k) {
                tma_load_2d_pair(a_tile(ab, 0, k), &map_phi, fa, k * kBK, y);
                tma_load_2d_pair(a_tile(ab, 1, k), &map_plo, fa, k * kBK, y);
            }
            for (int ct = 0; ct < n_ct && !abort_flag; ++ct) {
                for (int k = 0; k < a.nk; ++k, ++g) {
                    const uint32_t s = g % NS, use = g / NS;
                    if (use > 0 && !mbar_wait_cluster(&b_empty[s], (use - 1) & 1, a.timeout_ns)) {
                        fail(a.ctl, &abort_flag);
                        break;
                    }
                    if (rank == 0)
                        mbar_expect_tx(&b_full[s], 2 * 2 * kBBytes);
                    const uint32_t fb = mapa(smem_u32(&b_full[s]), 0);
                    const int yc = ct * kPN + (int)rank * kPNH;
                    tma_load_2d_pair(sB + (s * 2 + 0) * kBBytes, &map_chi, fb, k * kBK, yc);
                    tma_load_2d_pair(sB + (s * 2 + 1) * kBBytes, &map_clo, fb, k * kBK, yc);
                }
            }
        }
        if (abort_flag) {
            // this CTA's loads complete on the even CTA's barriers, which
            // this thread cannot wait on: give those in flight time to land
            const uint64_t t0 = gtimer();
            while (gtimer() - t0 < 200000ull)
                __nanosleep(1000);
        }
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // ---- MMA issuer (even CTA) ----
        const uint32_t idesc = idesc_bf16_f32(2 * kBM, kPN);
        uint32_t it = 0, g = 0, t = 0;
        bool issued = false;
        for (int64_t gp = cl0; gp < n_grp && !abort_flag; gp += ncl, ++it) {
            const uint32_t ab = it % a.abufs, ause = it / a.abufs;
            if (!mbar_wait_cluster(&a_full[ab], ause & 1, a.timeout_ns)) {
                fail(a.ctl, &abort_flag);
                break;
            }
            fence_after_sync();
            for (int ct = 0; ct < n_ct && !abort_flag; ++ct, ++t) {
                const uint32_t buf = t & 1, use_acc = t >> 1;
                if (use_acc > 0 &&
                    !mbar_wait_cluster(&acc_empty[buf], (use_acc - 1) & 1, a.timeout_ns)) {
                    fail(a.ctl, &abort_flag);
                    break;
                }
                fence_after_sync();
                const uint32_t d_tmem = tmem + buf * kPN;
                for (int k = 0; k < a.nk; ++k, ++g) {
                    const uint32_t s = g % NS, use = g / NS;
                    if (!mbar_wait_cluster(&b_full[s], use & 1, a.timeout_ns)) {
                        fail(a.ctl, &abort_flag);
                        break;
                    }
                    fence_after_sync();
                    const uint32_t bh = smem_u32(sB + (s * 2 + 0) * kBBytes);
                    const uint32_t bl = smem_u32(sB + (s * 2 + 1) * kBBytes);
                    const uint32_t ah = smem_u32(a_tile(ab, 0, k));
                    const uint32_t al = smem_u32(a_tile(ab, 1, k));
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint32_t o = kk * 32;
                        mma_bf16_pair(d_tmem, sdesc_k_sw128(ah + o), sdesc_k_sw128(bh + o), idesc,
                                      (k | kk) ? 1u : 0u);
                        mma_bf16_pair(d_tmem, sdesc_k_sw128(ah + o), sdesc_k_sw128(bl + o), idesc,
                                      1u);
                        mma_bf16_pair(d_tmem, sdesc_k_sw128(al + o), sdesc_k_sw128(bh + o), idesc,
                                      1u);
                    }
                    issued = true;
                    mma_commit_pair(&b_empty[s], 0x3); // both halves of stage s are free
                }
                if (abort_flag)
                    break;
                mma_commit_pair(&acc_full[buf], 0x3);
            }
            if (abort_flag)
                break;
            mma_commit_pair(&a_empty[ab], 0x3);
        }
        if (issued) { // every MMA issued completes before the pair frees its tensor memory
            mma_commit_pair(&done, 0x1);
            mbar_wait_cluster(&done, 0, a.timeout_ns);
        }
    } else if (warp >= 4) {
        // ---- epilogue (both CTAs): its own 128 rows of each accumulator ----
        const int q = warp & 3;
        const int row_local = q * 32 + lane;
        uint32_t t = 0;
        for (int64_t gp = cl0; gp < n_grp && !abort_flag; gp += ncl) {
            float best = __int_as_float(0x7f800000);
            int bk = 0;
            for (int ct = 0; ct < n_ct; ++ct, ++t) {
                const uint32_t buf = t & 1, use = t >> 1;
                if (!mbar_wait_cluster(&acc_full[buf], use & 1, a.timeout_ns)) {
                    fail(a.ctl, &abort_flag);
                    break;
                }
                fence_after_sync();
                const float4 *cn4 = reinterpret_cast<const float4 *>(s_cn + ct * kPN);
                // four rounds of 64 columns; the next round's loads are in
                // flight while this one is scored
                const uint32_t base = tmem + buf * kPN + ((uint32_t)(q * 32) << 16);
                uint32_t r[2][2][32];
                tmem_ld32_async(base, r[0][0]);
                tmem_ld32_async(base + 32, r[0][1]);
                tmem_ld_wait();
                tmem_regs_ready(r[0][0]);
                tmem_regs_ready(r[0][1]);
#pragma unroll
                for (int j = 0; j < kPN / 64; ++j) {
                    const int slot = j & 1, h = 2 * j;
                    if (j + 1 < kPN / 64) {
                        tmem_ld32_async(base + (h + 2) * 32, r[slot ^ 1][0]);
                        tmem_ld32_async(base + (h + 3) * 32, r[slot ^ 1][1]);
                    } else {
                        // every column of the accumulator is in registers:
                        // release it before scoring the last 64
                        fence_before_sync();
                        __syncwarp();
                        if (lane == 0)
                            mbar_arrive_cluster(mapa(smem_u32(&acc_empty[buf]), 0));
                    }
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        float w[32];
                        block_scores32(r[slot][c], cn4 + (h + c) * 8, w);
                        int wi;
                        const float m = block_argmin32(w, wi);
                        if (m < best) { // earlier blocks win ties
                            best = m;
                            bk = ct * kPN + (h + c) * 32 + wi;
                        }
                    }
                    if (j + 1 < kPN / 64) {
                        tmem_ld_wait();
                        tmem_regs_ready(r[slot ^ 1][0]);
                        tmem_regs_ready(r[slot ^ 1][1]);
                    }
                }
            }
            if (abort_flag)
                break;
            const int64_t row = (gp * 2 + rank) * kBM + row_local;
            if (row < a.N)
                a.labels[row] = bk;
        }
    }
    // the pair's MMAs drained (the even CTA waited for them) and both
    // epilogues done before either CTA frees tensor memory or exits
    fence_before_sync();
    __syncthreads();
    cluster_sync();
    if (warp == 2) {
        fence_after_sync();
        tmem_dealloc_pair(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// Update: exact D^2 to the assigned centre, phi, per-centre sums and counts.
// ---------------------------------------------------------------------------
constexpr int kUpdThreads = 512;
constexpr size_t kUpdSmem = 200 * 1024; // per-CTA FP32 sums of one centre tile

// centres per tile of the update's shared-memory sums
__host__ __device__ inline int update_tile(int K, int d)
{
    const int t = (int)((kUpdSmem - 4 * 1024) / ((size_t)d * 4 + 4));
    return t < K ? t : K;
}

// Every CTA owns a contiguous range of points and walks it once per tile of
// TK centres.  A warp takes ROWS points at a time (16 for d <= 64, 8 above):
// their labels in one load, then all their features (lane j holds features
// j, j+32, ...), so the loads of a batch are in flight together; each point's
// features are added into the CTA's FP32 sums of its centre in shared memory.
// Walks after the first load only the points whose centre is in the tile.
// The tile's sums then go to the FP64 totals in global memory with one atomic
// per (centre, feature).  The first walk also takes the FP32 difference-form
// D^2 to the assigned centre and the CTA's cost: per lane the squares of its
// features (even features in one accumulator, odd in another), then the
// batch's per-lane partials are reduce-scattered across the warp (point r
// ends in lane r * 32 / ROWS); costs are FP32 two-sum pairs.
template <int VEC, int ROWS> // features per lane and point: ceil(d / 32); points per batch
__global__ void __launch_bounds__(kUpdThreads, 1)
    lloyd_update_kernel(const float *x, int64_t N, int d, int K, const float *c,
                        const int32_t *labels, float *d2_out, double *sums,
                        unsigned long long *counts, double *partial)
{
    static_assert(ROWS == 8 || ROWS == 16, "8 or 16 points per batch");
    constexpr int kStages = ROWS == 16 ? 4 : 3; // reduce-scatter halvings
    extern __shared__ float u_smem[];
    __shared__ float2 wsum[kUpdThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int TK = update_tile(K, d);
    float *acc = u_smem;                                                   // [TK x d]
    unsigned *cnt = reinterpret_cast<unsigned *>(u_smem + (size_t)TK * d); // [TK]
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per;
    const int64_t r1 = (r0 + per) < N ? (r0 + per) : N;
    Pair mine{}; // the cost of this lane's points
    for (int k0 = 0; k0 < K; k0 += TK) {
        const int tk = (K - k0) < TK ? (K - k0) : TK;
        for (int e = threadIdx.x; e < tk * d; e += blockDim.x)
            acc[e] = 0.f;
        for (int e = threadIdx.x; e < tk; e += blockDim.x)
            cnt[e] = 0u;
        __syncthreads();
        for (int64_t b = r0 + (int64_t)warp * ROWS; b < r1; b += (int64_t)nwarps * ROWS) {
            const int nr = (r1 - b) < ROWS ? (int)(r1 - b) : ROWS;
            const int my_label = lane < nr ? labels[b + lane] : 0;
            // points of this batch to load: all on the first walk (for D^2),
            // then only those whose centre is in the tile
            // (on the first walk the row loads do not wait for the labels)
            unsigned need = (1u << nr) - 1u;
            if (k0 > 0) {
                need = __ballot_sync(0xffffffffu, lane < nr && my_label >= k0 && my_label < k0 + tk);
                if (need == 0)
                    continue;
            }
            float xv[ROWS][VEC];
#pragma unroll
            for (int q = 0; q < ROWS; ++q)
#pragma unroll
                for (int t = 0; t < VEC; ++t) {
                    const int j = lane + 32 * t;
                    xv[q][t] = (((need >> q) & 1u) && j < d) ? x[(b + q) * d + j] : 0.f;
                }
            if (k0 == 0) {
                // the assigned centres' features, all in flight, then the
                // per-lane partial squared distances of the batch's points
                float part[ROWS];
#pragma unroll
                for (int q = 0; q < ROWS; ++q) {
                    const int k = __shfl_sync(0xffffffffu, my_label, q);
                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                    for (int t = 0; t < VEC; ++t) {
                        const int j = lane + 32 * t;
                        const float cj = (q < nr && j < d) ? c[(int64_t)k * d + j] : 0.f;
                        const float u = xv[q][t] - cj;
                        if (j & 1)
                            a1 = fmaf(u, u, a1);
                        else
                            a0 = fmaf(u, u, a0);
                    }
                    part[q] = a0 + a1;
                }
                // reduce-scatter: lane bits 4, 3, ... select the point, the
                // remaining low bits are summed last
#pragma unroll
                for (int h = 0; h < kStages; ++h) {
                    const int m = 16 >> h;          // 16, 8, 4 (, 2)
                    const int w = (ROWS / 2) >> h;  // values kept
                    const bool up = (lane & m) != 0;
#pragma unroll
                    for (int i = 0; i < w; ++i) {
                        const float send = up ? part[i] : part[i + w];
                        const float keep = up ? part[i + w] : part[i];
                        part[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
                    }
                }
                float v = part[0];
#pragma unroll
                for (int o = (16 >> kStages); o >= 1; o >>= 1)
                    v += __shfl_xor_sync(0xffffffffu, v, o);
                int r = 0;
#pragma unroll
                for (int h = 0; h < kStages; ++h)
                    r |= ((lane >> (4 - h)) & 1) << (kStages - 1 - h);
                if ((lane & ((32 / ROWS) - 1)) == 0 && r < nr) {
                    if (d2_out)
                        d2_out[b + r] = v;
                    mine.add(v);
                }
            }
#pragma unroll
            for (int q = 0; q < ROWS; ++q) {
                if (q >= nr)
                    break;
                const int k = __shfl_sync(0xffffffffu, my_label, q);
                if (k >= k0 && k < k0 + tk) {
                    float *ak = acc + (size_t)(k - k0) * d;
#pragma unroll
                    for (int t = 0; t < VEC; ++t) {
                        const int j = lane + 32 * t;
                        if (j < d)
                            atomicAdd(ak + j, xv[q][t]);
                    }
                    if (lane == 0)
                        atomicAdd(cnt + (k - k0), 1u);
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < tk * d; e += blockDim.x) {
            const float v = acc[e];
            if (v != 0.f)
                atomicAdd(sums + (size_t)k0 * d + e, (double)v);
        }
        for (int e = threadIdx.x; e < tk; e += blockDim.x)
            if (cnt[e])
                atomicAdd(counts + k0 + e, (unsigned long long)cnt[e]);
        __syncthreads();
    }
    // the CTA's cost: lanes, then warps, in a fixed order
    const Pair wt = warp_pair_sum(mine);
    if (lane == 0)
        wsum[warp] = make_float2(wt.hi, wt.lo);
    __syncthreads();
    if (threadIdx.x == 0) {
        Pair t{};
        for (int w = 0; w < nwarps; ++w)
            t.add(Pair{wsum[w].x, wsum[w].y});
        partial[blockIdx.x] = (double)t.hi + (double)t.lo;
    }
}

using UpdateFn = void (*)(const float *, int64_t, int, int, const float *, const int32_t *,
                          float *, double *, unsigned long long *, double *);

UpdateFn update_fn(int d)
{
    if (d <= 32)
        return &lloyd_update_kernel<1, 16>;
    if (d <= 64)
        return &lloyd_update_kernel<2, 16>;
    return &lloyd_update_kernel<4, 8>;
}

__global__ void lloyd_finalize_kernel(const float *c_in, int K, int d, const double *sums,
                                      const unsigned long long *counts, float *c_out,
                                      int64_t *counts_out, const double *partial, int nparts,
                                      double *phi_out)
{
    const int64_t n = (int64_t)K * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / d);
        const unsigned long long m = counts[k];
        c_out[e] = m ? (float)(sums[e] / (double)m) : c_in[e];
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; counts_out && k < K;
         k += gridDim.x * blockDim.x)
        counts_out[k] = (int64_t)counts[k];
    if (blockIdx.x == 0 && threadIdx.x == 0 && phi_out) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b)
            s += partial[b];
        *phi_out = s;
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// [rows x dp] BF16, 128-byte swizzled boxes of 64 features x box_rows rows;
// rows past the end read as zero
bool make_map(CUtensorMap *m, const void *base, int64_t rows, int dp, int box_rows)
{
    auto enc = encode_fn();
    if (!enc)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)dp * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// centre-tile stages that fit beside the point tiles and the centre norms
int padded_k(int K) { return (K + kBN - 1) / kBN * kBN; }

int assign_stages(int nk, int K, int abufs)
{
    const long long budget = 227LL * 1024 - 1024 - 8 * 1024 -
                             (long long)abufs * kMT * 2 * nk * kABytes - (long long)padded_k(K) * 4;
    const int s = budget > 0 ? (int)(budget / (2 * kBBytes)) : 0;
    return s < kMaxStages ? s : kMaxStages;
}

// Two point-tile buffers when that still leaves kMinStagesTwoA centre stages.
constexpr int kMinStagesTwoA = 2;
int assign_abufs(int nk, int K) { return assign_stages(nk, K, 2) >= kMinStagesTwoA ? 2 : 1; }

// The CTA-pair form's centre stages (half a 256-centre tile each) and point
// buffers (one 128-point tile each).
int padded_k_pair(int K) { return (K + kPN - 1) / kPN * kPN; }
int assign_stages_pair(int nk, int K, int abufs)
{
    const long long budget = 227LL * 1024 - 1024 - 8 * 1024 -
                             (long long)abufs * 2 * nk * kABytes - (long long)padded_k_pair(K) * 4;
    const int s = budget > 0 ? (int)(budget / (2 * kBBytes)) : 0;
    return s < kMaxStagesPair ? s : kMaxStagesPair;
}
constexpr int kMinStagesTwoAPair = 3;
int assign_abufs_pair(int nk, int K)
{
    return assign_stages_pair(nk, K, 2) >= kMinStagesTwoAPair ? 2 : 1;
}
size_t assign_smem_pair(int nk, int K)
{
    const int ab = assign_abufs_pair(nk, K);
    return 1024 + (size_t)ab * 2 * nk * kABytes + (size_t)assign_stages_pair(nk, K, ab) * 2 * kBBytes +
           (size_t)padded_k_pair(K) * 4;
}

// Which assignment kernel: the CTA-pair form wherever a cluster of two fits
// (measured on 10^7 points, K = 1024: 2.89 against 3.10 ms at d = 64, 4.65
// against 5.55 ms at d = 128); the one-SM form otherwise.  KPP_LLOYD_PAIR=0
// or 1 forces one of them; both give the same labels.
bool use_pair_form()
{
    const char *e = std::getenv("KPP_LLOYD_PAIR");
    return !(e && e[0] == '0');
}

size_t assign_smem(int nk, int K)
{
    const int ab = assign_abufs(nk, K);
    return 1024 + (size_t)ab * kMT * 2 * nk * kABytes + (size_t)assign_stages(nk, K, ab) * 2 * kBBytes +
           (size_t)padded_k(K) * 4;
}

int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

// The assignment of N prepared points to K centres.  With row0 and kdev set,
// the centres are rows [*row0, *row0 + *kdev) of `centres` and K is only the
// largest count the launch is sized for; both are read on the device.
kpp_status assign_impl(const float *centres, const long long *row0, const int32_t *kdev, int32_t K,
                       int64_t N, int32_t d, int32_t *labels_out, void *workspace,
                       size_t workspace_bytes, cudaStream_t s)
{
    const Layout L = layout(N, d, K);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 ||
        workspace_bytes < L.bytes)
        return KPP_ERR_WORKSPACE;
    char *ws = reinterpret_cast<char *>(workspace);
    const int sms = sm_count();
    if (sms <= 0)
        return KPP_ERR_CUDA;
    auto *phi = reinterpret_cast<__nv_bfloat16 *>(ws + L.off_phi);
    auto *plo = reinterpret_cast<__nv_bfloat16 *>(ws + L.off_plo);
    auto *chi = reinterpret_cast<__nv_bfloat16 *>(ws + L.off_chi);
    auto *clo = reinterpret_cast<__nv_bfloat16 *>(ws + L.off_clo);
    float *cn = reinterpret_cast<float *>(ws + L.off_cn);
    CUtensorMap m_phi, m_plo, m_chi, m_clo;
    if (!make_map(&m_phi, phi, N, L.dp, kBM) || !make_map(&m_plo, plo, N, L.dp, kBM) ||
        !make_map(&m_chi, chi, K, L.dp, kBN) || !make_map(&m_clo, clo, K, L.dp, kBN))
        return KPP_ERR_CUDA;
    const int nk = L.dp / kBK;
    const size_t smem = assign_smem(nk, K);
    if (cudaFuncSetAttribute(lloyd_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return KPP_ERR_CUDA;
    AssignArgs a;
    a.N = N;
    a.K = K;
    a.Kdev = kdev;
    a.nk = nk;
    a.abufs = assign_abufs(nk, K);
    a.stages = assign_stages(nk, K, a.abufs);
    a.cn = cn;
    a.labels = labels_out;
    a.ctl = reinterpret_cast<Control *>(ws);
    a.timeout_ns = 2000000000ull;
    if (a.stages < 2)
        return KPP_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(ws, 0, sizeof(Control), s) != cudaSuccess)
        return KPP_ERR_CUDA;
    if (kdev) {
        split_rows_dev_kernel<<<(K * L.dp / 8 + 255) / 256, 256, 0, s>>>(centres, row0, kdev, d,
                                                                         L.dp, chi, clo);
        centre_norms_dev_kernel<<<(K + 127) / 128, 128, 0, s>>>(centres, row0, kdev, d, cn);
    } else {
        split_rows_kernel<<<(K * L.dp / 8 + 255) / 256, 256, 0, s>>>(centres, K, d, L.dp, chi,
                                                                     clo);
        centre_norms_kernel<<<(K + 127) / 128, 128, 0, s>>>(centres, K, d, cn);
    }
    if (use_pair_form()) {
        // CTA pairs: persistent, as many clusters of two as fit at once
        AssignArgs a2 = a;
        a2.abufs = assign_abufs_pair(nk, K);
        a2.stages = assign_stages_pair(nk, K, a2.abufs);
        const size_t smem2 = assign_smem_pair(nk, K);
        if (a2.stages >= 2 &&
            cudaFuncSetAttribute(lloyd_assign_pair_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem2) == cudaSuccess) {
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2, 1, 1);
            cfg.blockDim = dim3(kThreads, 1, 1);
            cfg.dynamicSmemBytes = smem2;
            cfg.stream = s;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int ncl = 0;
            if (cudaOccupancyMaxActiveClusters(&ncl, lloyd_assign_pair_kernel, &cfg) ==
                    cudaSuccess &&
                ncl >= 1) {
                const int64_t n_grp2 = ((N + kBM - 1) / kBM + 1) / 2;
                const int64_t clusters = n_grp2 < ncl ? n_grp2 : ncl;
                cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
                if (cudaLaunchKernelEx(&cfg, lloyd_assign_pair_kernel, m_phi, m_plo, m_chi, m_clo,
                                       a2) != cudaSuccess)
                    return KPP_ERR_LAUNCH;
                return cudaGetLastError() == cudaSuccess ? KPP_OK : KPP_ERR_LAUNCH;
            }
        }
        (void)cudaGetLastError(); // no cluster fits: the one-SM form below
    }
    const int64_t n_grp = ((N + kBM - 1) / kBM + kMT - 1) / kMT;
    const int grid = (int)(n_grp < sms ? n_grp : sms);
    lloyd_assign_kernel<<<grid, kThreads, smem, s>>>(m_phi, m_plo, m_chi, m_clo, a);
    return cudaGetLastError() == cudaSuccess ? KPP_OK : KPP_ERR_LAUNCH;
}

} // namespace

kpp_status lloyd_assign_device_count(const float *centres, const long long *row0,
                                     const int32_t *kdev, int32_t kmax, int64_t N, int32_t d,
                                     int32_t *labels_out, void *workspace, size_t workspace_bytes,
                                     cudaStream_t stream)
{
    if (!centres || !row0 || !kdev || !labels_out || !shape_ok(N, d, kmax))
        return KPP_ERR_INVALID_ARG;
    return assign_impl(centres, row0, kdev, kmax, N, d, labels_out, workspace, workspace_bytes,
                       stream);
}

} // namespace kpp

using namespace kpp;

extern "C" {

size_t kpp_lloyd_workspace_size(int64_t N, int32_t d, int32_t K)
{
    if (!shape_ok(N, d, K))
        return 0;
    return layout(N, d, K).bytes;
}

kpp_status kpp_lloyd_prepare(const float *points, int64_t N, int32_t d, int32_t K, void *workspace,
                             size_t workspace_bytes, kpp_stream_t stream)
{
    if (!points || !shape_ok(N, d, K))
        return KPP_ERR_INVALID_ARG;
    const Layout L = layout(N, d, K);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 ||
        workspace_bytes < L.bytes)
        return KPP_ERR_WORKSPACE;
    char *ws = reinterpret_cast<char *>(workspace);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int sms = sm_count();
    if (sms <= 0)
        return KPP_ERR_CUDA;
    split_rows_kernel<<<sms * 8, 256, 0, s>>>(points, N, d, L.dp,
                                             reinterpret_cast<__nv_bfloat16 *>(ws + L.off_phi),
                                             reinterpret_cast<__nv_bfloat16 *>(ws + L.off_plo));
    return cudaGetLastError() == cudaSuccess ? KPP_OK : KPP_ERR_LAUNCH;
}

kpp_status kpp_lloyd_assign(const float *centres, int64_t N, int32_t d, int32_t K,
                            int32_t *labels_out, void *workspace, size_t workspace_bytes,
                            kpp_stream_t stream)
{
    if (!centres || !labels_out || !shape_ok(N, d, K))
        return KPP_ERR_INVALID_ARG;
    return assign_impl(centres, nullptr, nullptr, K, N, d, labels_out, workspace, workspace_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
}

kpp_status kpp_lloyd_step(const float *points, int64_t N, int32_t d, const float *centres,
                          int32_t K, int32_t *labels_out, float *d2_out, float *centres_out,
                          int64_t *counts_out, double *phi_out, void *workspace,
                          size_t workspace_bytes, kpp_stream_t stream)
{
    if (!points || !centres || !labels_out || !centres_out || !shape_ok(N, d, K))
        return KPP_ERR_INVALID_ARG;
    const Layout L = layout(N, d, K);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 ||
        workspace_bytes < L.bytes)
        return KPP_ERR_WORKSPACE;
    char *ws = reinterpret_cast<char *>(workspace);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int sms = sm_count();
    if (sms <= 0)
        return KPP_ERR_CUDA;
    double *sums = reinterpret_cast<double *>(ws + L.off_sums);
    auto *counts = reinterpret_cast<unsigned long long *>(ws + L.off_counts);
    double *partial = reinterpret_cast<double *>(ws + L.off_partial);
    const size_t usmem = (size_t)update_tile(K, d) * ((size_t)d * 4 + 4);
    const UpdateFn ufn = update_fn(d);
    if (cudaFuncSetAttribute(ufn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usmem) !=
        cudaSuccess)
        return KPP_ERR_CUDA;
    const kpp_status st =
        kpp_lloyd_assign(centres, N, d, K, labels_out, workspace, workspace_bytes, stream);
    if (st != KPP_OK)
        return st;
    if (cudaMemsetAsync(ws + L.off_sums, 0, L.off_partial - L.off_sums, s) != cudaSuccess)
        return KPP_ERR_CUDA;
    const int ugrid = sms < L.grid ? sms : L.grid;
    ufn<<<ugrid, kUpdThreads, usmem, s>>>(points, N, d, K, centres, labels_out, d2_out, sums,
                                          counts, partial);
    lloyd_finalize_kernel<<<(K * d + 255) / 256, 256, 0, s>>>(centres, K, d, sums, counts,
                                                              centres_out, counts_out, partial,
                                                              ugrid, phi_out);
    return cudaGetLastError() == cudaSuccess ? KPP_OK : KPP_ERR_LAUNCH;
}

} // extern "C"

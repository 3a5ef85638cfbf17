// kpp_quantize.cu -- precision forms of the point array (not in the paper):
// FP32 -> BF16 (round to nearest even) and FP32 -> FP8-E4M3 with one FP32
// scale per row, s_i = max_j |x_ij| / 448 (1 for an all-zero row), codes
// q_ij = RNE-saturating E4M3 of the FP32 quotient x_ij / s_i.  One
// streaming pass, done once per dataset before seeding.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kpp_internal.h"

namespace kpp {

namespace {

constexpr int kQThreads = 256;

// BF16: 8 elements per thread-iteration (two 16-byte loads, one store).
__global__ void __launch_bounds__(kQThreads)
    quantize_bf16_kernel(const float *__restrict__ x, uint16_t *__restrict__ out, int64_t n)
{
    const int64_t n8 = n / 8;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += stride) {
        float4 a = __ldcs(reinterpret_cast<const float4 *>(x) + 2 * i);
        float4 b = __ldcs(reinterpret_cast<const float4 *>(x) + 2 * i + 1);
        const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k]));
            uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k + 1]));
            w[k] = lo | (hi << 16);
        }
        __stcs(reinterpret_cast<uint4 *>(out) + i, make_uint4(w[0], w[1], w[2], w[3]));
    }
    // tail (n not a multiple of 8)
    for (int64_t i = n8 * 8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x[i]));
}

// FP8: one warp per row.
__global__ void __launch_bounds__(kQThreads)
    quantize_fp8_kernel(const float *__restrict__ x, uint8_t *__restrict__ q,
                        float *__restrict__ scales, int64_t N, int d)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); row < N;
         row += warps) {
        const float *xr = x + row * d;
        float mx = 0.f;
        for (int j = lane; j < d; j += 32)
            mx = fmaxf(mx, fabsf(__ldg(xr + j)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float s = mx > 0.f ? __fdiv_rn(mx, 448.0f) : 1.0f;
        if (lane == 0)
            scales[row] = s;
        uint8_t *qr = q + row * d;
        for (int j = lane; j < d; j += 32) {
            const float v = __fdiv_rn(xr[j], s);
            qr[j] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

int grid_for(int64_t work, int per_block)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (work + per_block - 1) / per_block;
    int64_t cap = (int64_t)sms * 8;
    if (want < 1)
        want = 1;
    return (int)(want < cap ? want : cap);
}

} // namespace

cudaError_t quantize_bf16(const float *x, int64_t n, uint16_t *out, cudaStream_t stream)
{
    quantize_bf16_kernel<<<grid_for(n / 8 + 1, kQThreads), kQThreads, 0, stream>>>(x, out, n);
    return cudaGetLastError();
}

cudaError_t quantize_fp8(const float *x, int64_t N, int d, uint8_t *q, float *scales,
                         cudaStream_t stream)
{
    quantize_fp8_kernel<<<grid_for(N, kQThreads / 32), kQThreads, 0, stream>>>(x, q, scales, N, d);
    return cudaGetLastError();
}

} // namespace kpp

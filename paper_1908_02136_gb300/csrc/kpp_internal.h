// kpp_internal.h -- declarations shared by the host-side translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kpp_device.cuh"

namespace kpp {

// One streamed-form specialisation chosen for (dtype, d, lanes).
struct StreamedKernel {
    const void *fn;
    int rows_align; // per-CTA row ranges are multiples of this
    int lanes;      // lanes per row (0 for the generic kernel)
    bool generic;
};

bool streamed_lookup(int dt, int d, int lanes, StreamedKernel *out);
int streamed_threads();
cudaError_t streamed_launch(const StreamedKernel &k, int grid, const Problem &p, int m,
                            cudaStream_t stream);

} // namespace kpp

namespace kpp {

cudaError_t quantize_bf16(const float *x, int64_t n, uint16_t *out, cudaStream_t stream);
cudaError_t quantize_fp8(const float *x, int64_t N, int d, uint8_t *q, float *scales,
                         cudaStream_t stream);

} // namespace kpp

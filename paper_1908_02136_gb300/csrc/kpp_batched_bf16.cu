// kpp_batched_bf16.cu -- batched-form kernel for BF16 points.
#include "kpp_batched.cuh"

namespace kpp {

BatchFn batched_kernel_bf16() { return &batched_kernel<KPP_BF16>; }

} // namespace kpp

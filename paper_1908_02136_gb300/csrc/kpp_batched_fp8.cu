// kpp_batched_fp8.cu -- batched-form kernel for FP8 points.
#include "kpp_batched.cuh"

namespace kpp {

BatchFn batched_kernel_fp8() { return &batched_kernel<KPP_FP8_E4M3>; }

} // namespace kpp

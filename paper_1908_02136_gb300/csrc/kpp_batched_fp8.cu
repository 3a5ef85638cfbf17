// kpp_batched_fp8.cu -- batched-form wave kernels for FP8 points, one per d.
#include "kpp_batched.cuh"

namespace kpp {

BatchFn batched_kernel_fp8(int d) { return batched_kernel_of<KPP_FP8_E4M3>(d); }

} // namespace kpp
